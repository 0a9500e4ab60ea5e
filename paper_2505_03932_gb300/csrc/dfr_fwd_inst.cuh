// Instantiation of the split forward kernels of one (launch form, tile height, staging): each set
// is its own translation unit, so that the sets compile in parallel. A unit defines
// NAME(order) -> kernel and the reader of its device status word, NAME_status. SW sets also
// compile the asynchronous-copy box staging for sources TMA cannot describe.
#pragma once

#include "dfr_fwd_kernels.cuh"

#define DFR_SPLIT_K(O, BATCH, TH, SW) \
  reinterpret_cast<const void*>(&fwd_split_kernel<O, BATCH, false, TH, SW>)

#define DFR_SPLIT_SET(NAME, BATCH, TH, SW)                                  \
  namespace dfr {                                                          \
  const void* NAME(int order) {                                           \
    switch (order) {                                                      \
      case DFR_NEAREST: return DFR_SPLIT_K(DFR_NEAREST, BATCH, TH, SW);   \
      case DFR_BILINEAR: return DFR_SPLIT_K(DFR_BILINEAR, BATCH, TH, SW); \
      case DFR_BICUBIC: return DFR_SPLIT_K(DFR_BICUBIC, BATCH, TH, SW);   \
      case DFR_LANCZOS3: return DFR_SPLIT_K(DFR_LANCZOS3, BATCH, TH, SW); \
      default: return DFR_SPLIT_K(DFR_BSPLINE3, BATCH, TH, SW);           \
    }                                                                     \
  }                                                                       \
  DFR_DEFINE_STATUS_READER(NAME##_status)                                 \
  }
