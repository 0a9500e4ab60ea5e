/* dfr — GB300-native TAN-SIP reprojection: public C ABI.
 *
 * The library reprojects a source image onto a target FITS-WCS pixel grid, per target pixel:
 *   target pixel -> (shift, SIP A/B, CD, gnomonic deprojection, native->celestial) -> (ra, dec)
 *   -> (celestial->native, gnomonic projection, CD^-1, inverse SIP AP/BP, shift) -> source
 *   pixel -> nearest / bilinear / bicubic interpolation normalised by the footprint.
 * This is dfreproject (arXiv 2505.03932) Sec. 3.1 steps 1-3, with the formulas of
 * Sec. 3.2.1 and Sec. 3.2.2, following the FITS WCS papers (Greisen & Calabretta 2002,
 * Calabretta & Greisen 2002) and the SIP convention (Shupe et al. 2005) the paper cites.
 *
 * Conventions shared by every call
 *   - Images are row-major float32, y (NAXIS2) rows of x (NAXIS1) pixels; `pitch` is the row
 *     stride in ELEMENTS. Pixel centres sit at integer 0-based coordinates (Sec. 3.2 shifts by
 *     one pixel from FITS' 1-based CRPIX).
 *   - A target bounding box (x0, y0, w, h) selects target pixels x0 .. x0+w-1, y0 .. y0+h-1;
 *     output element (i, j) holds target pixel (x0 + i, y0 + j).
 *   - Interpolation reads taps outside the source as zero and divides by the footprint, the
 *     in-bounds sum of the interpolation weights (Sec. 3.1, "identity tensor"). A target pixel
 *     whose source position lies outside [-0.5, W-0.5] x [-0.5, H-0.5], or whose sky position
 *     is on the far hemisphere of the source projection, gets value 0 and footprint 0.
 *   - SIP polynomials use the monomials u^p v^q with 1 <= p+q <= ORDER and are ADDED:
 *     u <- u + A(u, v), v <- v + B(u, v) (Shupe et al. 2005; the paper prints a minus sign,
 *     which does not match the convention it cites).
 *   - Device pointers are caller-owned CUDA device memory; `stream` is a cudaStream_t (NULL =
 *     legacy default stream). Calls that launch work are asynchronous on that stream.
 *   - Every call returns DFR_OK (0) or a negative DFR_ERR_* code; dfr_last_error() gives a
 *     thread-local message for the last failure on the calling thread. Argument errors are
 *     reported before anything is launched.
 */
#ifndef DFR_H_
#define DFR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DFR_ABI_VERSION 1

/* status codes */
#define DFR_OK                   0
#define DFR_ERR_INVALID_ARG     -1  /* null/ill-sized argument, bad order or flag          */
#define DFR_ERR_HEADER_PARSE    -2  /* malformed card or missing required keyword          */
#define DFR_ERR_UNSUPPORTED_WCS -3  /* CTYPE not RA---TAN/DEC--TAN[-SIP]                   */
#define DFR_ERR_SINGULAR_CD     -4  /* det(CD) == 0 or non-finite                          */
#define DFR_ERR_NO_INVERSE_SIP  -5  /* source has A/B but no AP/BP and no exact inverse    */
#define DFR_ERR_CUDA            -6  /* a CUDA runtime call failed                          */
#define DFR_ERR_TIMEOUT         -7  /* a bounded device-side wait gave up                  */
#define DFR_ERR_DEVICE          -8  /* a kernel reported a failed internal check           */

/* interpolation orders (Sec. 4.2 names three schemes) */
#define DFR_NEAREST  0
#define DFR_BILINEAR 1
#define DFR_BICUBIC  2   /* Keys cubic convolution, a = -0.5 */
#define DFR_LANCZOS3 3   /* Lanczos-3 (6x6 taps, weights normalised per axis)               */
#define DFR_BSPLINE3 4   /* cubic B-spline on prefiltered coefficients (dfr_bspline_prefilter), */
                         /* mirror boundary, footprint 1 where covered; forward only           */

/* flags */
#define DFR_FP64           0u  /* all-FP64 per pixel: the printed formulas, with libm trig   */
#define DFR_SPLIT          1u  /* the map exactly (sky rotation in ~48-bit double-float) at */
                               /* 20 points per 32x64 cell, per-column FP32 cubics between   */
#define DFR_EXACT_INVERSE  2u  /* source inverse = Newton solve of A/B (AP/BP as start)      */
#define DFR_NO_TMA         4u  /* gather straight from global memory instead of TMA tiles    */
#define DFR_NAN_MASK       8u  /* NaN source pixels are missing: no weight in value or        */
                               /* footprint (forward and co-add; not the adjoint)             */

#define DFR_MAX_SIP 9

/* WCS record. Plain data in host memory, owned by the caller. */
typedef struct dfr_wcs {
  int32_t naxis[2];       /* NAXIS1 (width, x), NAXIS2 (height, y)                          */
  double  crpix[2];       /* FITS 1-based reference pixel                                   */
  double  crval[2];       /* reference point (ra0, dec0), degrees                           */
  double  cd[2][2];       /* CDi_j (or PCi_j * CDELTi), degrees per pixel                   */
  int32_t a_order, b_order, ap_order, bp_order;        /* 0 = absent, at most DFR_MAX_SIP   */
  double  a[10][10], b[10][10], ap[10][10], bp[10][10]; /* [p][q]: coefficient of u^p v^q   */
} dfr_wcs;

/* One exposure of a batch. Device pointers are caller-owned. */
typedef struct dfr_frame {
  dfr_wcs      wcs;        /* source WCS                                                    */
  const float* img;        /* source image, wcs.naxis[1] rows of wcs.naxis[0] floats        */
  int64_t      pitch;      /* source row stride, elements (>= naxis[0])                     */
  float*       out;        /* reprojected values, h rows of w floats, row stride out_pitch  */
  float*       footprint;  /* footprint (same layout), may be NULL                          */
  int64_t      out_pitch;  /* output row stride, elements (>= w)                            */
  int32_t      x0, y0, w, h; /* target bounding box; use dfr_target_bbox to size it         */
} dfr_frame;

/* Thread-local text of the last error on this thread ("" if none). Never NULL. */
const char* dfr_last_error(void);

/* Library ABI version (DFR_ABI_VERSION). */
int dfr_abi_version(void);

/* Parse a FITS header into a WCS record (Sec. 2: header reading is a cheap host step;
 * Sec. 3.1 lists the keywords used). `cards` holds 80-character cards, either packed or
 * newline-separated; `nbytes` is its length. Keywords: NAXISn, CTYPEn (RA---TAN / DEC--TAN,
 * optional -SIP), CRPIXn, CRVALn, CDi_j or PCi_j with CDELTi (CD wins; CD = CDELT x PC,
 * Sec. 3.1) or, with neither CD nor PC, CDELTi with the legacy CROTA2 rotation
 * (CD = [[CDELT1 cos r, -CDELT2 sin r], [CDELT1 sin r, CDELT2 cos r]]), optional LONPOLE,
 * A_ORDER/A_p_q, B_*, AP_*, BP_*. The record has no LONPOLE field: the method's formulas fix
 * the native pole longitude at 180 deg (Sec. 3.2), and another LONPOLE (a rotation of the
 * native longitude, which for the zenithal TAN is a rotation of the intermediate plane after
 * CD) is folded into CD. Missing keywords -> DFR_ERR_HEADER_PARSE; other projections ->
 * DFR_ERR_UNSUPPORTED_WCS; singular CD -> DFR_ERR_SINGULAR_CD. `out` is fully written on
 * success, untouched on failure. */
int dfr_wcs_from_header(const char* cards, size_t nbytes, dfr_wcs* out);

/* Fit inverse SIP polynomials AP/BP of the given order (1..9) to the forward A/B of `wcs`
 * by least squares (Householder QR) on a grid over the frame plus a 5% margin, and store
 * them in `wcs` (host memory, in place). Sec. 3.1 names SIP_INV_A/B as header content;
 * this builds them when a header has only A/B. max_resid_px / rms_resid_px (nullable)
 * receive the round-trip residual over a 512x512 grid of the frame. */
int dfr_wcs_fit_inverse_sip(dfr_wcs* wcs, int32_t order, double* max_resid_px,
                            double* rms_resid_px);

/* Target-pixel bounding box of a source frame: the source boundary, sampled densely, mapped
 * into the target grid (FP64, host), widened by 2 px and clipped to the target. Writes
 * bbox = {x0, y0, w, h}; w = h = 0 when the frame misses the target. Host only. */
int dfr_target_bbox(const dfr_wcs* src, const dfr_wcs* tgt, int32_t bbox[4]);

/* Reproject one source image onto a bounding box of the target grid (Sec. 3.1 steps 1-3,
 * Sec. 3.2). src_img: device, src->naxis[1] rows, row stride src_pitch. out: device,
 * out_h rows of out_w values, row stride out_pitch. footprint: device, same layout, nullable.
 * order: DFR_NEAREST / DFR_BILINEAR / DFR_BICUBIC / DFR_LANCZOS3 / DFR_BSPLINE3 (src_img then
 * holds B-spline coefficients). flags: DFR_FP64 or DFR_SPLIT, optionally
 * | DFR_EXACT_INVERSE | DFR_NO_TMA | DFR_NAN_MASK. Without DFR_NAN_MASK, NaN source pixels
 * propagate into the values they touch. coords_out (nullable, device): 2*out_w*out_h doubles,
 * the source position (x then y per pixel, row-major) exactly as the kernel used it, NaN where
 * the projection is undefined. Asynchronous on `stream`; out/footprint are written in full.
 * Split-precision frames of at least 2^22 output pixels tune the kernel's tile height (8, 16
 * or 32 target rows per staged source box) on their first call per (order, flags, inverse
 * degree, size class) by timing the three on the caller's arguments (each writes the same
 * bits; that first call synchronises the stream); DFR_AUTOTUNE=0, or a stream being
 * captured, keeps 16, DFR_TILE_H=8|16|32 pins it. */
int dfr_reproject(const dfr_wcs* src, const dfr_wcs* tgt,
                  const float* src_img, int64_t src_pitch,
                  float* out, float* footprint, int64_t out_pitch,
                  int32_t x0, int32_t y0, int32_t out_w, int32_t out_h,
                  int32_t order, uint32_t flags, double* coords_out, void* stream);

/* dfr_reproject from HOST memory to HOST memory, with the copies overlapped with the work:
 * the bounding box is cut into bands of 64-pixel cell rows; each band's source rows go
 * host->device on one library stream (only rows no earlier band copied), its kernel runs on a
 * second stream once they are in, and its value / footprint rows go device->host on a third,
 * so both copy directions and the compute overlap. host_img: src->naxis[1] rows, stride
 * host_pitch; host_out / host_fp (nullable): out_h rows of out_w, stride out_pitch. The
 * library holds the device copies of source and outputs (cached per device, grown on demand).
 * Page-locked host buffers (cudaHostAlloc / cudaHostRegister) let the copies run
 * asynchronously; pageable memory works but serialises them. Returns once the outputs are in
 * host memory. The FP64 path, DFR_BSPLINE3 (prefilter first) and boxes of one band run as one
 * band. Same arithmetic, so the same bits, as dfr_reproject. */
int dfr_reproject_host(const dfr_wcs* src, const dfr_wcs* tgt, const float* host_img,
                       int64_t host_pitch, float* host_out, float* host_fp, int64_t out_pitch,
                       int32_t x0, int32_t y0, int32_t out_w, int32_t out_h, int32_t order,
                       uint32_t flags);

/* Reproject n exposures onto one target grid in one CUDA-graph launch (the paper's pipeline
 * stacks >1000 exposures, Sec. 2). Every frame's pixels are computed with exactly the
 * arithmetic of dfr_reproject for the same bounding box and flags, so results are equal bit
 * for bit. Frames with w or h == 0 are skipped. The graph is either the single-frame kernels
 * in parallel chains or one kernel over a frame table (library-owned pinned and device
 * memory; split precision: one CTA per anchor cell of every frame, all-FP64: a persistent
 * grid); a built-in autotuner picks the form, the chains or CTAs per SM, source-box staging
 * on or off and, for split precision, the tile height (8, 16 or 32 target rows per staged
 * source box) on the first call per (order, flags, SIP degree, log2 n), by timing the
 * candidates on the caller's data (DFR_AUTOTUNE=0: one chain, tile height 16, no timing;
 * DFR_BATCH_FORM=graph|table and DFR_TILE_H=8|16|32 restrict the search). Graphs are cached
 * and updated in place when only pointers change. */
int dfr_reproject_batch(const dfr_frame* frames, int32_t n, const dfr_wcs* tgt,
                        int32_t order, uint32_t flags, void* stream);

/* dfr_reproject_batch without any device allocation: the same frames, target and flags give
 * the same output bits as dfr_reproject_batch. The paper has no counterpart; this is for
 * callers that cannot call cudaMalloc or let a library do it (a plug-in inside a host
 * framework whose allocator owns all device memory; a real-time loop that must avoid
 * cudaMalloc's implicit synchronisation). Instead of allocated scratch it uses a fixed
 * library-owned device array of about 300 KB that every GPU loading the library keeps until
 * the process exits. At most 64 frames per call (more -> DFR_ERR_INVALID_ARG, nothing
 * launched). The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress). The frame table is
 * copied in from a static host buffer with a pageable cudaMemcpyAsync (which waits for the
 * stream's earlier work) and the work counter is cleared on every call. Every call shares the
 * one array per device: calls whose kernels overlap on the GPU (different streams, or several
 * host threads) race on it. No autotuning and no graph; caller-owned buffers as in
 * dfr_reproject_batch. */
int dfr_reproject_batch_noalloc(const dfr_frame* frames, int32_t n, const dfr_wcs* tgt,
                                int32_t order, uint32_t flags, void* stream);

/* Launch configurations the library last chose (a report for benchmarks and tuning; the paper
 * has no counterpart). out[5], host memory: [0] the tile height (rows of target pixels per
 * staged source box, 8, 16 or 32; 0: no staging) of the last split-precision dfr_reproject;
 * [1..4] of the last dfr_reproject_batch: form (1: a CUDA graph of single-frame kernels in
 * parallel chains, 0: one kernel over the frame table), chains or CTAs per SM, box staging
 * (0/1), tile height. Process-wide (the last call on any device or thread). DFR_ERR_INVALID_ARG if out is
 * NULL. */
int dfr_last_launch_config(int32_t* out);

/* Measured throughput of the arithmetic pipes on the current device (the denominators of the
 * all-FP64 path's roofline; the paper has no counterpart). out[4], host memory, operations
 * per second: [0] FP64 flops by fused multiply-add (2 per DFMA), [1] FP32 flops by scalar
 * FFMA, [2] FP32 flops by packed FP32x2 FMA (4 per instruction), [3] special-function results
 * per second (sin.approx.f32). Each from the best of three launches of a kernel of 8 independent
 * chains per thread filling every SM; synchronises `stream`; about 0.1 s. */
int dfr_measure_pipe_peaks(double* out, void* stream);

/* Cubic B-spline prefilter (the interpolation coefficients of DFR_BSPLINE3): per row, then per
 * column, the recursive filter with pole z = sqrt(3) - 2 and gain 6 (Unser, Aldroubi & Eden,
 * 1991; the causal start summed over a mirrored horizon, the anticausal start in closed form),
 * with mirror (whole-sample symmetric) boundaries, so that the cubic B-spline through the
 * coefficients passes through every source pixel. img / coef: device, h rows of w values, row
 * strides pitch / coef_pitch; coef may equal img (in place, same stride). A reprojection with
 * DFR_BSPLINE3 takes coef as its source image. Asynchronous on `stream`. */
int dfr_bspline_prefilter(const float* img, int64_t pitch, int32_t w, int32_t h, float* coef,
                          int64_t coef_pitch, void* stream);

/* Co-add (stack) n exposures onto one target grid: for every target pixel p covered by a
 * frame, sum_vf[p] += value_f(p) * footprint_f(p) and sum_f[p] += footprint_f(p), with value
 * and footprint exactly as dfr_reproject computes them (Sec. 3.1); combining reprojected
 * exposures is the use the paper builds the method for (Sec. 1). Frames are added in order,
 * one after another (one CUDA-graph launch), each as a single FP32 fused multiply-add per
 * pixel: the result is deterministic. sum_vf / sum_f: device, tgt->naxis[1] rows of
 * tgt->naxis[0] values, row stride `pitch` (>= NAXIS1); the caller zeroes them first (or keeps
 * accumulating across calls). A frame's out / footprint / out_pitch fields are ignored; its
 * bounding box must lie inside the target grid, and w = h = 0 asks the library to size it
 * (dfr_target_bbox). Pixels a frame does not cover are not touched. flags as dfr_reproject
 * (DFR_NO_TMA allowed). Frames share library-owned graph state with dfr_reproject_batch. */
int dfr_coadd(const dfr_frame* frames, int32_t n, const dfr_wcs* tgt, int32_t order,
              uint32_t flags, float* sum_vf, float* sum_f, int64_t pitch, void* stream);

/* Mean of a co-add: mean[p] = sum_vf[p] / sum_f[p] where sum_f[p] > min_weight, else 0 (the
 * value of uncovered pixels in dfr_reproject). Device buffers, h rows of w values, row strides
 * pitch (sums) and mean_pitch; mean may alias sum_vf when the strides agree. Asynchronous. */
int dfr_coadd_normalize(const float* sum_vf, const float* sum_f, int64_t pitch, int32_t w,
                        int32_t h, float min_weight, float* mean, int64_t mean_pitch,
                        void* stream);

/* Adjoint of dfr_reproject with respect to the source pixels and the source WCS.
 * Given grad_out = dL/d(out) (device, out_h rows, stride go_pitch) for the same arguments as a
 * forward call, accumulates grad_src += dL/d(src_img) (device, src->naxis[1] rows, stride
 * gs_pitch; nullable) by scattering grad * w / footprint through the interpolation weights,
 * and writes grad_params (device, nullable) = dL/d(theta) for the source parameters
 *   [CRVAL1, CRVAL2 (per degree), CD1_1, CD1_2, CD2_1, CD2_2,
 *    A_pq for 1 <= p+q <= A_ORDER (by p+q, then p descending), B_pq likewise],
 * i.e. 6 + n_terms(A) + n_terms(B) doubles. The paper has no gradient; this extension lets
 * alignment parameters be fitted by gradient descent. Source positions use the same
 * arithmetic as the forward call with the same flags. order: DFR_NEAREST, DFR_BILINEAR,
 * DFR_BICUBIC or DFR_LANCZOS3; DFR_BSPLINE3 and the DFR_NAN_MASK flag are refused
 * (DFR_ERR_INVALID_ARG). Asynchronous on `stream`. */
int dfr_reproject_backward(const dfr_wcs* src, const dfr_wcs* tgt,
                           const float* src_img, int64_t src_pitch,
                           const float* grad_out, int64_t go_pitch,
                           int32_t x0, int32_t y0, int32_t out_w, int32_t out_h,
                           int32_t order, uint32_t flags,
                           float* grad_src, int64_t gs_pitch,
                           double* grad_params, void* stream);

/* One frame of a batched adjoint: the arguments of one dfr_reproject_backward call. */
typedef struct dfr_bwd_frame {
  dfr_wcs      wcs;         /* source WCS                                                   */
  const float* img;         /* source image, wcs.naxis[1] rows of wcs.naxis[0] floats       */
  int64_t      pitch;       /* source row stride, elements                                  */
  const float* grad_out;    /* dL/d(out), h rows of w floats, row stride go_pitch           */
  int64_t      go_pitch;
  int32_t      x0, y0, w, h; /* target bounding box of the forward call                     */
  float*       grad_src;    /* accumulated dL/d(img) (same layout as img, stride gs_pitch);
                               may be NULL                                                  */
  int64_t      gs_pitch;
  double*      grad_params; /* dfr_num_params(&wcs) doubles, may be NULL                    */
} dfr_bwd_frame;

/* Batched adjoint: the n calls dfr_reproject_backward(frames[f], ...) with one target, order
 * and flags, issued at once. The frames run side by side on library-owned streams, after the
 * work enqueued on `stream` before the call and before the work enqueued after it (as if all
 * ran on `stream`). Each frame's kernels and arguments are those of its single call:
 * grad_params come out bit for bit equal to the single calls'; grad_src receives the same
 * terms, added by float atomics whose order (and so the last bits of a sum) may differ, as
 * between two single calls. Frames may share a grad_src buffer (their terms add up). Errors:
 * as dfr_reproject_backward, the message naming the frame; nothing is launched when a frame's
 * arguments are refused. Asynchronous. */
int dfr_reproject_backward_batch(const dfr_bwd_frame* frames, int32_t n, const dfr_wcs* tgt,
                                 int32_t order, uint32_t flags, void* stream);

/* Number of doubles dfr_reproject_backward writes to grad_params for this source WCS. */
int dfr_num_params(const dfr_wcs* src);

/* Read and clear the device status word that kernels set when a bounded wait gives up or an
 * internal check fails. Synchronises `stream`. Returns DFR_OK, DFR_ERR_TIMEOUT or
 * DFR_ERR_DEVICE. */
int dfr_device_status(void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DFR_H_ */
