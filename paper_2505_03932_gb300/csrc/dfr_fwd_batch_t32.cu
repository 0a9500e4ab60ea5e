// Batched (frame table) split forward kernels, tile height 32 (see dfr_fwd_inst.cuh).
#include "dfr_fwd_inst.cuh"

DFR_SPLIT_SET(split_batch_t32, true, 32, false)
