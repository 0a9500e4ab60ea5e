// Single-frame split forward kernels, tile height 16 (see dfr_fwd_inst.cuh).
#include "dfr_fwd_inst.cuh"

DFR_SPLIT_SET(split_single_t16, false, 16, false)
