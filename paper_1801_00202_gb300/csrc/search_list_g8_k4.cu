// Listing variants of the search kernels with 8 lanes per subtree and 4 words per lane.
#include "search_inst.cuh"
MCE_DEFINE_SEARCH_LIST(8, 4)
