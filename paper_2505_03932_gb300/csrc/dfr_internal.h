// Internal plan structures shared by the host plan builder (dfr_host.cpp) and the kernels
// (dfr_fwd.cu, dfr_bwd.cu). Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dfr.h"

namespace dfr {

// Coefficients of a 2-D polynomial of total degree <= N, packed row by row in p:
// P(u, v) = sum_p u^p C_p(v), C_p(v) = sum_{q <= N-p} c[off(p) + q] v^q, off(p) = p(N+1) - p(p-1)/2.
// The constant term c[0] is always 0 (SIP has no constant term).
constexpr int kMaxCoef = (DFR_MAX_SIP + 1) * (DFR_MAX_SIP + 2) / 2;  // 55

__host__ __device__ constexpr int poly_off(int p, int n) { return p * (n + 1) - p * (p - 1) / 2; }
__host__ __device__ constexpr int poly_ncoef(int n) { return (n + 1) * (n + 2) / 2; }

// Target tile: 32 x 8 pixels, relative to the bounding-box origin (the FP64 kernel's work unit
// and the adjoint's staged tile; lane = column).
constexpr int kTileW = 32;
constexpr int kTileH = 8;
constexpr int kTilePix = kTileW * kTileH;
// Cell of the split path: 32 x 64 pixels of the bounding box (cells tile it from its origin).
// The warp that owns a cell samples the map at a 4 x 4 grid of nodes and four check points in
// about 48-bit double-float arithmetic (FP64 with a target SIP), one point per lane, and each
// lane interpolates the cubic in the row that gives its column's source positions (cell_fit).
// The forward split kernel runs one warp (one cell) per CTA and stages the source in boxes of
// TH rows (a template parameter, 8, 16 or 32: the tile height the autotuner picks). The staged
// adjoint runs kBwdWarps warps per CTA, one cell each.
constexpr int kCellW = 32;
constexpr int kCellH = 64;
constexpr int kTilesPerCell = kCellH / kTileH;
constexpr int kFwdWarps = 1;
constexpr int kCellsPerCta = 1;
constexpr int kBwdWarps = 4;
constexpr int kBwdCellsPerCta = 4;
// Source-box row pitch of the split kernels, in floats: a multiple of 32, so that the 32 lanes
// of a warp (consecutive target columns) reading a tap from two adjacent source rows fall in
// distinct shared-memory banks. It is also the TMA box width.
constexpr int kBoxW = 64;
// Default tile height (box rows of target pixels) of the split forward kernel.
constexpr int kDefaultTileH = 16;

// Per-frame forward plan. Built on the host in FP64; read by every CTA of the launch.
struct FwdPlan {  // aligned (128 B) through its CUtensorMap member, as TMA requires
  CUtensorMap tmap;          // source image tile map (valid when use_tma != 0)
  // target bounding box and its tiling
  int32_t x0, y0, w, h;
  int32_t tiles_x, tiles_y;
  int32_t cells_x, cells_y;
  // outputs (device)
  float* out;
  float* fp;                 // nullable
  int64_t out_pitch;
  double* coords;            // nullable: 2 doubles per output pixel
  // source image (device)
  const float* img;
  int64_t pitch;
  int32_t W, H;
  int32_t use_tma, box_w, box_h;  // use_tma: source boxes staged in shared memory (by TMA,
                             // or, with stage_sw, by per-thread asynchronous copies)
  int32_t stage_sw;          // boxes staged by cp.async (a source whose row pitch TMA cannot
                             // describe: not a multiple of 16 bytes, or a base not 16-aligned)
  int32_t box_margin;        // px added around a tile's corner extent (covers map curvature)
  int32_t th;                // tile height (rows) the box and its tensor map are sized for
  int32_t tma_ok;            // box staging the source allows: 1 TMA, 2 asynchronous copies, 0 none
  float jac[4];              // host bounds of |dx/dX|, |dx/dY|, |dy/dX|, |dy/dY| (box sizing)
  float curv[3];             // host bounds of the map's second derivatives (xx, xy, yy)
  int32_t identity;          // the map is a translation: source and target WCS differ at
                             // most in CRPIX (same CRVAL, CD and distortion)
  double shift[2];           // then x_s = x_t + shift (source minus target CRPIX)
  // target WCS
  double crpix_t[2];         // CRPIX - 1 (0-based reference pixel)
  int32_t tsip_deg;          // 0 = no target SIP; else packed degree of A, B
  double tsip_d[2][kMaxCoef];
  float tsip_f[2][kMaxCoef];
  // split path: homography from target intermediate offsets (p, q) (after SIP, pixels) to
  // source intermediate offsets (U, V) (before inverse SIP, pixels), scaled so G[2][2] = 1
  double G[3][3];
  // the same G, CRPIX - 1 of the target and of the source as unevaluated float pairs
  // (hi, lo; hi = the nearest float, lo = the nearest float to the rest) for the
  // double-float arithmetic of the split path's anchors
  float G_ff[3][3][2];
  float crpix_t_ff[2][2];
  float crpix_s_ff[2][2];
  // source WCS
  double crpix_s[2];         // CRPIX - 1
  int32_t isip_deg;          // packed degree of AP, BP (0 = none)
  float isip_f[2][kMaxCoef];
  double isip_d[2][kMaxCoef];
  int32_t fsip_deg;          // packed degree of the source A, B (exact inverse; 0 = none)
  float fsip_f[2][kMaxCoef];
  double fsip_d[2][kMaxCoef];
  int32_t newton_iters;      // FP32 Newton steps in the split exact inverse
  // all-FP64 path constants
  double ra0_t, sd0_t, cd0_t;
  double cd_t[2][2];
  double ra0_s, sd0_s, cd0_s;
  double cdinv_s[2][2];
  double cd_s[2][2];
  int32_t flags;
  int32_t order;
};

// Launch description shared by the forward kernels.
struct FwdLaunch {
  const FwdPlan* plans;      // batch: device array of n plans (nullptr: single frame in p0)
  const int32_t* tile_start; // batch: device prefix sums of work units per frame (n + 1
                             // entries, the last is the total): tiles for the FP64 kernel,
                             // anchor cells for the split kernel
  int32_t nframes;
  int32_t total_tiles;       // single frame: work units (tiles or cells; batch reads
                             // tile_start[n])
  int32_t* counter;          // FP64 batch: device work counter of the persistent grid
  int32_t box_floats;        // floats of each warp's source-box buffer, a multiple of 32
  int32_t unit_begin;        // single-frame split launch: first work unit (a band of the box)
  int32_t split_from;        // single frame: cells from this one on are split into split_k
  int32_t split_k;           // units of kCellH / (TH split_k) tile rows each (1: no split)
  uint32_t tx_extra;         // fault injection for the timeout test: bytes added to every box
                             // load's expected count, so that its wait runs out (0 normally)
};

// Backward launch arguments. The kernel accumulates parameter gradients in a padded layout
// (6 + 2 * terms(fd)); pmap sends each padded entry to its dfr_reproject_backward index (-1:
// not a parameter of this WCS).
constexpr int kMaxParams = 6 + 2 * (kMaxCoef - 1);  // 114
struct BwdExtra {
  float* grad_src;           // nullable
  int64_t gs_pitch;
  const float* grad_out;
  int64_t go_pitch;
  double* grad_params;       // nullable: final, nout entries
  double* partials;          // scratch: grid x np per-block sums
  int32_t nout;              // dfr_num_params(src)
  int32_t fd;                // padded A/B degree of the parameter layout (0: A/B not live)
  int32_t grid;
  int32_t box_floats;        // split path: floats of each warp's source / gradient box (0: none)
  int16_t pmap[kMaxParams];
};

// Internal plan flag (never part of the public flags): the plan's kernel adds value x footprint
// and footprint into co-add sums instead of storing value and footprint.
constexpr uint32_t kFlagAccumulate = 1u << 16;

// Device status word: bit 0 = a bounded wait timed out, bit 1 = internal check failed.
enum : int32_t { kStatusTimeout = 1, kStatusCheck = 2 };

// Kernel launchers (dfr_fwd.cu / dfr_bwd.cu). Return cudaError_t.
cudaError_t launch_forward(const FwdPlan& p0, const FwdLaunch& L, int grid, int threads,
                           int smem_bytes, cudaStream_t s);
const void* forward_kernel(const FwdPlan& p0);
// split kernels by launch form, staging and tile height
// (dfr_fwd_{single,batch}[_sw]_t{8,16,32}.cu) and their status readers
#define DFR_SPLIT_DECL(NAME)    \
  const void* NAME(int order); \
  cudaError_t NAME##_status(int32_t* out, cudaStream_t s);
DFR_SPLIT_DECL(split_single_t8)
DFR_SPLIT_DECL(split_single_t16)
DFR_SPLIT_DECL(split_single_t32)
DFR_SPLIT_DECL(split_batch_t8)
DFR_SPLIT_DECL(split_batch_t16)
DFR_SPLIT_DECL(split_batch_t32)
DFR_SPLIT_DECL(split_single_sw_t8)
DFR_SPLIT_DECL(split_single_sw_t16)
DFR_SPLIT_DECL(split_single_sw_t32)
DFR_SPLIT_DECL(split_batch_sw_t8)
DFR_SPLIT_DECL(split_batch_sw_t16)
DFR_SPLIT_DECL(split_batch_sw_t32)
#undef DFR_SPLIT_DECL
cudaError_t launch_split_coords(const FwdPlan& p0, cudaStream_t s);
int forward_max_blocks_per_sm(const FwdPlan& p0, int threads, int smem_bytes, bool batch = true);
int forward_threads_default();
cudaError_t read_and_clear_status_fwd(int32_t* out, cudaStream_t s);
cudaError_t read_and_clear_status_bwd(int32_t* out, cudaStream_t s);
cudaError_t read_and_clear_status_bwd_tile(int32_t* out, cudaStream_t s);
cudaError_t read_and_clear_status_coadd(int32_t* out, cudaStream_t s);
cudaError_t launch_backward(const FwdPlan& p0, const BwdExtra& B, cudaStream_t s);
int backward_num_padded(int fd);
int backward_max_blocks_per_sm(const FwdPlan& p0, int fd, int smem_bytes);
int backward_smem_bytes(const FwdPlan& p0, int fd, int box_floats);
int backward_threads_for(const FwdPlan& p0, int fd);
const void* backward_tile_kernel(int order, int ideg, int fd);  // dfr_bwd_tile.cu
const void* coadd_kernel(const FwdPlan& p0);                      // dfr_coadd.cu
cudaError_t launch_bspline_prefilter(const float* img, int64_t pitch, int32_t w, int32_t h,
                                     float* coef, int64_t coef_pitch, cudaStream_t s);
cudaError_t launch_coadd_normalize(const float* sum_vf, const float* sum_f, int64_t pitch,
                                   int32_t w, int32_t h, float min_weight, float* mean,
                                   int64_t mean_pitch, cudaStream_t s);

// Box size and tensor map of a plan for tiles of th rows (dfr_host.cpp).
void set_tile_height(FwdPlan& P, int th);

// Plan-builder access for translation units other than dfr_host.cpp.
int plan_for_frame(const dfr_frame& fr, const dfr_wcs* tgt, int32_t order, uint32_t flags,
                   int ideg, FwdPlan& P);
int inverse_degree_for(const dfr_frame* frames, int n);
int plan_box_floats(const FwdPlan& P);
int batch_units(const FwdPlan& P);
FwdPlan batch_head(const FwdPlan* plans, int n);
int split_grid(const FwdPlan& P, int cells, int32_t& split_from, int32_t& split_k, bool batch,
               int smem);
int plan_smem_bytes(int floats);
int report_error(int code, const char* msg);
int report_cuda_error(cudaError_t e, const char* where);

}  // namespace dfr
