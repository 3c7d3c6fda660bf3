// Search kernel instantiations with 16 lane(s) per subtree.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH(16, 1)
MCE_DEFINE_SEARCH(16, 2)
