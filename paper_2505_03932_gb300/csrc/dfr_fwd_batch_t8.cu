// Batched (frame table) split forward kernels, tile height 8 (see dfr_fwd_inst.cuh).
#include "dfr_fwd_inst.cuh"

DFR_SPLIT_SET(split_batch_t8, true, 8, false)
