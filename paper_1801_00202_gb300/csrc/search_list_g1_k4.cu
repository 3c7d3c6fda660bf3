// Listing variants of the search kernels with 1 lane per subtree and 4 words per lane.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH_LIST(1, 4)
