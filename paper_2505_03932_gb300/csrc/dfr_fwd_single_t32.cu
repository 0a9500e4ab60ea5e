// Single-frame split forward kernels, tile height 32 (see dfr_fwd_inst.cuh).
#include "dfr_fwd_inst.cuh"

DFR_SPLIT_SET(split_single_t32, false, 32, false)
