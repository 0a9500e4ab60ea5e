// Batched (frame table) split forward kernels, tile height 16 (see dfr_fwd_inst.cuh).
#include "dfr_fwd_inst.cuh"

DFR_SPLIT_SET(split_batch_t16, true, 16, false)
