// Search kernels with 16 lane(s) per subtree and 4 word(s) per lane.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH(16, 4)
