// Search kernel instantiations with 2 lane(s) per subtree.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH(2, 1)
MCE_DEFINE_SEARCH(2, 2)
