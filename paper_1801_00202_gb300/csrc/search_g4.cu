// Search kernel instantiations with 4 lane(s) per subtree.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH(4, 1)
MCE_DEFINE_SEARCH(4, 2)
