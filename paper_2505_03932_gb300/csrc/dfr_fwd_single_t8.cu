// Single-frame split forward kernels, tile height 8 (see dfr_fwd_inst.cuh).
#include "dfr_fwd_inst.cuh"

DFR_SPLIT_SET(split_single_t8, false, 8, false)
