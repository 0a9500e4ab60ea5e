// Single-frame split forward kernels, tile height 8, with
// asynchronous-copy box staging (see dfr_fwd_inst.cuh).
#include "dfr_fwd_inst.cuh"

DFR_SPLIT_SET(split_single_sw_t8, false, 8, true)
