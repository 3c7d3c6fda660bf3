// Search kernel instantiations with a whole warp per subtree.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH(32, 1)
MCE_DEFINE_SEARCH(32, 2)
MCE_DEFINE_SEARCH(32, 4)
