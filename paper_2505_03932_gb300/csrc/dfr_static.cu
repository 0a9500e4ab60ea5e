// dfr_reproject_batch_noalloc: the batched forward launch with its frame table in a fixed,
// library-owned device array instead of memory from cudaMalloc.
//
// Who needs it: callers that must not allocate device memory themselves or let a library do
// it, e.g. a plug-in running inside a host framework whose own allocator owns all GPU memory,
// or a real-time loop where cudaMalloc's implicit device synchronisation and unbounded latency
// are not allowed. They still pass their own input and output buffers.
#include <mutex>

#include "dfr_internal.h"

namespace dfr {
namespace {

constexpr int kStaticFrames = 64;  // maximum frames per call
constexpr int kMaxDevices = 64;

struct StaticBatch {
  FwdPlan plans[kStaticFrames];
  int32_t tile_start[kStaticFrames + 1];
  int32_t counter;
};

// The scratch: about 300 KB (64 frame plans, the tile prefix table and the work counter).
// Every GPU that loads the library holds it until the process exits. Host code must not use
// the symbol as a pointer: it is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_batch[sizeof(StaticBatch)];

std::mutex g_mu;
StaticBatch* g_addr[kMaxDevices];          // device address of g_static_batch, per device
FwdPlan g_host_plans[kStaticFrames];       // host staging, static (no allocation)
int32_t g_host_starts[kStaticFrames + 1];
int g_sms[kMaxDevices];

}  // namespace
}  // namespace dfr

using namespace dfr;

extern "C" int dfr_reproject_batch_noalloc(const dfr_frame* frames, int32_t n,
                                           const dfr_wcs* tgt, int32_t order, uint32_t flags,
                                           void* stream) {
  if (n < 0) return report_error(DFR_ERR_INVALID_ARG, "negative frame count");
  if (n > kStaticFrames)
    return report_error(DFR_ERR_INVALID_ARG,
                        "dfr_reproject_batch_noalloc takes at most 64 frames per call");
  if (n == 0) return DFR_OK;
  if (!frames) return report_error(DFR_ERR_INVALID_ARG, "NULL frame array");
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return report_error(DFR_ERR_INVALID_ARG, "device index beyond the static table");
  if (!g_addr[dev]) {
    // once per device, with that device current: the device address of the static scratch
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_batch);
    if (e != cudaSuccess) return report_cuda_error(e, "cudaGetSymbolAddress");
    e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return report_cuda_error(e, "cudaDeviceGetAttribute");
    g_addr[dev] = static_cast<StaticBatch*>(p);
  }
  StaticBatch* S = g_addr[dev];
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  const int ideg = inverse_degree_for(frames, n);
  int64_t total = 0;
  int floats = 0;
  for (int f = 0; f < n; ++f) {
    int rc = plan_for_frame(frames[f], tgt, order, flags, ideg, g_host_plans[f]);
    if (rc != DFR_OK) return rc;
    g_host_starts[f] = int32_t(total);
    if (frames[f].w > 0 && frames[f].h > 0)
      total += batch_units(g_host_plans[f]);
    floats = std::max(floats, plan_box_floats(g_host_plans[f]));
  }
  if (total >= (int64_t(1) << 31)) return report_error(DFR_ERR_INVALID_ARG, "batch too large");
  g_host_starts[n] = int32_t(total);
  if (total == 0) return DFR_OK;

  // Pageable-memory copies return once the host data is staged, so the static host arrays
  // may be rewritten by the next call; the copies wait for earlier work on the stream.
  e = cudaMemcpyAsync(S->plans, g_host_plans, size_t(n) * sizeof(FwdPlan),
                      cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return report_cuda_error(e, "cudaMemcpyAsync(plans)");
  e = cudaMemcpyAsync(S->tile_start, g_host_starts, size_t(n + 1) * sizeof(int32_t),
                      cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return report_cuda_error(e, "cudaMemcpyAsync(tile_start)");
  e = cudaMemsetAsync(&S->counter, 0, sizeof(int32_t), s);  // the counter must start at 0
  if (e != cudaSuccess) return report_cuda_error(e, "cudaMemsetAsync(counter)");

  FwdLaunch L{};
  L.plans = S->plans;
  L.tile_start = S->tile_start;
  L.nframes = n;
  L.counter = &S->counter;
  L.box_floats = floats;
  const int smem = plan_smem_bytes(floats);
  const int threads = forward_threads_default();
  const FwdPlan head = batch_head(g_host_plans, n);
  int grid;
  if (head.flags & DFR_SPLIT) {
    grid = split_grid(head, int(total), L.split_from, L.split_k, true, smem);
  } else {
    const int per_sm = forward_max_blocks_per_sm(head, threads, smem);
    grid = std::max(1, std::min(int(total), g_sms[dev] * per_sm));
  }
  e = launch_forward(head, L, grid, threads, smem, s);
  if (e != cudaSuccess) return report_cuda_error(e, "dfr_reproject_batch_noalloc launch");
  return DFR_OK;
}
