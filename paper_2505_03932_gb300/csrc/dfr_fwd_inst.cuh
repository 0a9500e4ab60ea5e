// Instantiation of the split forward kernels of one (launch form, tile height): each such set
// is its own translation unit, so that the sets compile in parallel. A unit defines
// NAME(order) -> kernel and the reader of its device status word, NAME_status.
#pragma once

#include "dfr_fwd_kernels.cuh"

#define DFR_SPLIT_SET(NAME, BATCH, TH)                                                      \
  namespace dfr {                                                                          \
  const void* NAME(int order) {                                                           \
    switch (order) {                                                                      \
      case DFR_NEAREST:                                                                   \
        return reinterpret_cast<const void*>(&fwd_split_kernel<DFR_NEAREST, BATCH, false, TH>); \
      case DFR_BILINEAR:                                                                  \
        return reinterpret_cast<const void*>(&fwd_split_kernel<DFR_BILINEAR, BATCH, false, TH>); \
      case DFR_BICUBIC:                                                                   \
        return reinterpret_cast<const void*>(&fwd_split_kernel<DFR_BICUBIC, BATCH, false, TH>); \
      case DFR_LANCZOS3:                                                                  \
        return reinterpret_cast<const void*>(&fwd_split_kernel<DFR_LANCZOS3, BATCH, false, TH>); \
      default:                                                                            \
        return reinterpret_cast<const void*>(&fwd_split_kernel<DFR_BSPLINE3, BATCH, false, TH>); \
    }                                                                                     \
  }                                                                                       \
  DFR_DEFINE_STATUS_READER(NAME##_status)                                                 \
  }
