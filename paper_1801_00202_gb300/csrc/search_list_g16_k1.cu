// Listing variants of the search kernels with 16 lanes per subtree and 1 word per lane.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH_LIST(16, 1)
