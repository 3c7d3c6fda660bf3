// Search kernels with 8 lane(s) per subtree and 2 word(s) per lane.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH(8, 2)
