// Search kernel instantiations with 8 lane(s) per subtree.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH(8, 1)
MCE_DEFINE_SEARCH(8, 2)
