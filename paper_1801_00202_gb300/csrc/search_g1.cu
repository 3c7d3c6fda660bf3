// Search kernel instantiations with 1 lane(s) per subtree.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH(1, 1)
MCE_DEFINE_SEARCH(1, 2)
