"""GB300-native TAN-SIP reprojection (dfreproject, arXiv 2505.03932) — Python binding.

Thin ctypes marshalling over the C ABI in ``include/dfr.h`` (libdfr.so, built in place by
``paper_2505_03932_gb300.build``). Every step of the reprojection runs in the library's CUDA
kernels; PyTorch only supplies device memory, streams and autograd. There is no CPU fallback:
if libdfr.so is missing or no CUDA device is present, the calls raise.

WCS records are plain dicts with the fields of ``dfr_wcs``: naxis (W, H), crpix, crval (deg),
cd (2x2, deg/px), a_order/b_order/ap_order/bp_order and a/b/ap/bp (10x10 arrays,
[p][q] = coefficient of u^p v^q).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "DfrError", "lib", "wcs_from_header", "fit_inverse_sip", "target_bbox", "num_params",
    "reproject", "reproject_batch", "reproject_batch_noalloc", "reproject_backward",
    "reproject_backward_batch",
    "coadd", "coadd_normalize", "reproject_host", "calculate_reprojection", "last_launch_config",
    "measure_pipe_peaks",
    "Reproject", "device_status", "bspline_prefilter", "NEAREST", "BILINEAR", "BICUBIC",
    "LANCZOS3", "BSPLINE3", "FP64", "SPLIT",
    "EXACT_INVERSE", "NO_TMA", "NAN_MASK",
]

NEAREST, BILINEAR, BICUBIC, LANCZOS3, BSPLINE3 = 0, 1, 2, 3, 4
FP64, SPLIT, EXACT_INVERSE, NO_TMA, NAN_MASK = 0, 1, 2, 4, 8
ORDERS = {"nearest": NEAREST, "bilinear": BILINEAR, "bicubic": BICUBIC, "lanczos3": LANCZOS3,
          "bspline3": BSPLINE3}
_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.environ.get("DFR_LIBRARY") or os.path.join(_HERE, "libdfr.so")


class DfrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dfr error %d: %s" % (code, msg))
        self.code = code


_d2 = ctypes.c_double * 2
_i2 = ctypes.c_int32 * 2
_m2 = (ctypes.c_double * 2) * 2
_s10 = (ctypes.c_double * 10) * 10


class DfrWcs(ctypes.Structure):
    _fields_ = [("naxis", _i2), ("crpix", _d2), ("crval", _d2), ("cd", _m2),
                ("a_order", ctypes.c_int32), ("b_order", ctypes.c_int32),
                ("ap_order", ctypes.c_int32), ("bp_order", ctypes.c_int32),
                ("a", _s10), ("b", _s10), ("ap", _s10), ("bp", _s10)]


class DfrFrame(ctypes.Structure):
    _fields_ = [("wcs", DfrWcs), ("img", ctypes.c_void_p), ("pitch", ctypes.c_int64),
                ("out", ctypes.c_void_p), ("footprint", ctypes.c_void_p),
                ("out_pitch", ctypes.c_int64), ("x0", ctypes.c_int32), ("y0", ctypes.c_int32),
                ("w", ctypes.c_int32), ("h", ctypes.c_int32)]


class DfrBwdFrame(ctypes.Structure):
    _fields_ = [("wcs", DfrWcs), ("img", ctypes.c_void_p), ("pitch", ctypes.c_int64),
                ("grad_out", ctypes.c_void_p), ("go_pitch", ctypes.c_int64),
                ("x0", ctypes.c_int32), ("y0", ctypes.c_int32), ("w", ctypes.c_int32),
                ("h", ctypes.c_int32), ("grad_src", ctypes.c_void_p), ("gs_pitch", ctypes.c_int64),
                ("grad_params", ctypes.c_void_p)]


_LIB = None


def lib():
    """The loaded libdfr.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_LIBPATH):
            raise RuntimeError("libdfr.so is not built: run python -m paper_2505_03932_gb300.build")
        L = ctypes.CDLL(_LIBPATH)
        L.dfr_last_error.restype = ctypes.c_char_p
        L.dfr_abi_version.restype = ctypes.c_int
        L.dfr_wcs_from_header.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(DfrWcs)]
        L.dfr_wcs_fit_inverse_sip.argtypes = [ctypes.POINTER(DfrWcs), ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]
        L.dfr_target_bbox.argtypes = [ctypes.POINTER(DfrWcs), ctypes.POINTER(DfrWcs),
                                      ctypes.POINTER(ctypes.c_int32)]
        L.dfr_reproject.argtypes = [
            ctypes.POINTER(DfrWcs), ctypes.POINTER(DfrWcs), ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p,
            ctypes.c_void_p]
        L.dfr_reproject_batch.argtypes = [ctypes.POINTER(DfrFrame), ctypes.c_int32,
                                          ctypes.POINTER(DfrWcs), ctypes.c_int32,
                                          ctypes.c_uint32, ctypes.c_void_p]
        L.dfr_reproject_backward.argtypes = [
            ctypes.POINTER(DfrWcs), ctypes.POINTER(DfrWcs), ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
            ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p]
        L.dfr_reproject_batch_noalloc.argtypes = [ctypes.POINTER(DfrFrame), ctypes.c_int32,
                                                  ctypes.POINTER(DfrWcs), ctypes.c_int32,
                                                  ctypes.c_uint32, ctypes.c_void_p]
        L.dfr_coadd.argtypes = [ctypes.POINTER(DfrFrame), ctypes.c_int32, ctypes.POINTER(DfrWcs),
                                ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.dfr_coadd_normalize.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.dfr_bspline_prefilter.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_void_p]
        L.dfr_reproject_host.argtypes = [
            ctypes.POINTER(DfrWcs), ctypes.POINTER(DfrWcs), ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32]
        L.dfr_reproject_backward_batch.argtypes = [ctypes.POINTER(DfrBwdFrame), ctypes.c_int32,
                                                   ctypes.POINTER(DfrWcs), ctypes.c_int32,
                                                   ctypes.c_uint32, ctypes.c_void_p]
        L.dfr_num_params.argtypes = [ctypes.POINTER(DfrWcs)]
        L.dfr_last_launch_config.argtypes = [ctypes.POINTER(ctypes.c_int32)]
        L.dfr_measure_pipe_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
        L.dfr_device_status.argtypes = [ctypes.c_void_p]
        _LIB = L
    return _LIB


def _check(rc):
    if rc != 0:
        raise DfrError(rc, lib().dfr_last_error().decode())
    return rc


# ------------------------------------------------------------------------------ WCS records
def to_c(w) -> DfrWcs:
    if isinstance(w, DfrWcs):
        return w
    c = DfrWcs()
    c.naxis[0], c.naxis[1] = int(w["naxis"][0]), int(w["naxis"][1])
    c.crpix[0], c.crpix[1] = float(w["crpix"][0]), float(w["crpix"][1])
    c.crval[0], c.crval[1] = float(w["crval"][0]), float(w["crval"][1])
    for i in range(2):
        for j in range(2):
            c.cd[i][j] = float(w["cd"][i][j])
    for k in ("a", "b", "ap", "bp"):
        setattr(c, k + "_order", int(w.get(k + "_order", 0)))
        arr = np.zeros((10, 10)) if w.get(k) is None else np.asarray(w[k], dtype=np.float64)
        dst = getattr(c, k)
        for p in range(10):
            for q in range(10):
                dst[p][q] = float(arr[p, q])
    return c


def from_c(c: DfrWcs) -> dict:
    w = {"naxis": (c.naxis[0], c.naxis[1]), "crpix": (c.crpix[0], c.crpix[1]),
         "crval": (c.crval[0], c.crval[1]),
         "cd": [[c.cd[0][0], c.cd[0][1]], [c.cd[1][0], c.cd[1][1]]]}
    for k in ("a", "b", "ap", "bp"):
        w[k + "_order"] = getattr(c, k + "_order")
        src = getattr(c, k)
        w[k] = np.array([[src[p][q] for q in range(10)] for p in range(10)], dtype=np.float64)
    return w


def wcs_from_header(text) -> dict:
    """Parse FITS header cards (str or bytes) into a WCS record (dfr_wcs_from_header)."""
    b = text.encode() if isinstance(text, str) else bytes(text)
    c = DfrWcs()
    _check(lib().dfr_wcs_from_header(b, len(b), ctypes.byref(c)))
    return from_c(c)


def fit_inverse_sip(w, order):
    """Copy of ``w`` with AP/BP of ``order`` fitted (dfr_wcs_fit_inverse_sip); also returns the
    max and RMS round-trip residual in pixels."""
    c = to_c(w)
    mx, rms = ctypes.c_double(), ctypes.c_double()
    _check(lib().dfr_wcs_fit_inverse_sip(ctypes.byref(c), int(order), ctypes.byref(mx),
                                         ctypes.byref(rms)))
    return from_c(c), mx.value, rms.value


def target_bbox(src, tgt):
    """(x0, y0, w, h) of the target pixels the source frame can cover (dfr_target_bbox)."""
    bb = (ctypes.c_int32 * 4)()
    _check(lib().dfr_target_bbox(ctypes.byref(to_c(src)), ctypes.byref(to_c(tgt)), bb))
    return tuple(int(v) for v in bb)


def num_params(src) -> int:
    n = lib().dfr_num_params(ctypes.byref(to_c(src)))
    if n < 0:
        _check(n)
    return n


def last_launch_config():
    """The launch configurations the library last chose (dfr_last_launch_config): a dict with
    the single-frame tile height and the last batch's form, chains / CTAs per SM, TMA, tile
    height."""
    v = (ctypes.c_int32 * 5)()
    _check(lib().dfr_last_launch_config(v))
    return {"single_tile_h": int(v[0]),
            "batch": {"form": "graph" if v[1] == 1 else "table", "k": int(v[2]),
                      "tma": bool(v[3]), "tile_h": int(v[4])}}


def measure_pipe_peaks(stream=None):
    """Measured pipe throughput of the current device (dfr_measure_pipe_peaks), in operations per
    second: FP64 FMA flops, FP32 FMA flops (scalar, packed FP32x2), special-function results."""
    v = (ctypes.c_double * 4)()
    _check(lib().dfr_measure_pipe_peaks(v, _stream_ptr(stream)))
    return {"fp64_fma_flops": v[0], "fp32_fma_flops": v[1], "fp32x2_fma_flops": v[2],
            "mufu_per_s": v[3]}


def device_status(stream=None):
    """Raise if a kernel reported a timed-out wait or a failed check since the last call."""
    _check(lib().dfr_device_status(_stream_ptr(stream)))


# ------------------------------------------------------------------------------ tensors
def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_f32(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or t.dim() != 2:
        raise ValueError("%s must be a 2-D float32 CUDA tensor" % name)
    if t.stride(1) != 1:
        raise ValueError("%s must have unit stride along x" % name)
    return t


def _naxis(w):
    nax = w.naxis if isinstance(w, DfrWcs) else w["naxis"]
    return int(nax[0]), int(nax[1])


def _check_image(img, wcs, name):
    """The kernels read NAXIS2 rows of NAXIS1 pixels at the tensor's row stride: refuse a smaller
    tensor (it would be read past its end)."""
    nx, ny = _naxis(wcs)
    if img.shape[0] < ny or img.shape[1] < nx:
        raise ValueError("%s has shape %s, smaller than the WCS NAXIS (%d, %d)"
                         % (name, tuple(img.shape), ny, nx))


def _check_out(out, fp, w, h, name="out"):
    """Value and footprint planes of a (w, h) bounding box: at least h rows of w pixels, and the
    footprint the same shape and row stride (the library takes one pitch for both)."""
    if out.shape[0] < h or out.shape[1] < w:
        raise ValueError("%s has shape %s, smaller than the box (%d, %d)"
                         % (name, tuple(out.shape), h, w))
    if fp is not None and (tuple(fp.shape) != tuple(out.shape) or fp.stride(0) != out.stride(0)):
        raise ValueError("the footprint must have the shape and row stride of %s" % name)


def _flags(precision, exact_inverse, tma, nan_mask=False):
    f = SPLIT if precision == "split" else FP64
    if precision not in ("split", "fp64"):
        raise ValueError("precision must be 'split' or 'fp64'")
    if exact_inverse:
        f |= EXACT_INVERSE
    if not tma:
        f |= NO_TMA
    if nan_mask:
        f |= NAN_MASK
    return f


def _order(order):
    return ORDERS[order] if isinstance(order, str) else int(order)


def bspline_prefilter(img, out=None, stream=None):
    """Cubic B-spline coefficients of a device image (dfr_bspline_prefilter); ``out`` may be
    ``img`` itself (in place)."""
    torch = _torch()
    img = _dev_f32(img, "img")
    if out is None:
        out = torch.empty_like(img)
    out = _dev_f32(out, "out")
    h, w = img.shape
    _check(lib().dfr_bspline_prefilter(ctypes.c_void_p(img.data_ptr()), img.stride(0), w, h,
                                       ctypes.c_void_p(out.data_ptr()), out.stride(0),
                                       _stream_ptr(stream)))
    return out


def _source_for(img, order, prefiltered, stream=None):
    """The image a launch reads: for the B-spline order its coefficients (prefiltered here
    unless the caller passes them)."""
    if _order(order) == BSPLINE3 and not prefiltered:
        return bspline_prefilter(img, stream=stream)
    return img


def reproject(src_img, src_wcs, tgt_wcs, shape_out=None, bbox=None, order="bilinear",
              precision="split", exact_inverse=False, footprint=True, coords=False, tma=True,
              out=None, fp_out=None, stream=None, nan_mask=False, prefiltered=False):
    """Reproject a device image onto the target grid (dfr_reproject).

    shape_out (h, w) defaults to the target NAXIS; bbox = (x0, y0, w, h) selects part of the
    target grid; nan_mask: NaN source pixels are missing (no weight); order "bspline3"
    prefilters the image first unless ``prefiltered`` (then src_img holds the coefficients).
    Returns (value, footprint or None[, coords (h, w, 2) float64])."""
    torch = _torch()
    src_img = _dev_f32(src_img, "src_img")
    _check_image(src_img, src_wcs, "src_img")
    src_img = _source_for(src_img, order, prefiltered, stream)
    if bbox is None:
        if shape_out is None:
            nax = tgt_wcs.naxis if isinstance(tgt_wcs, DfrWcs) else tgt_wcs["naxis"]
            shape_out = (int(nax[1]), int(nax[0]))
        bbox = (0, 0, int(shape_out[1]), int(shape_out[0]))
    x0, y0, w, h = (int(v) for v in bbox)
    dev = src_img.device
    if out is None:
        out = torch.empty((h, w), dtype=torch.float32, device=dev)
    out = _dev_f32(out, "out")
    fp = None
    if footprint:
        fp = fp_out if fp_out is not None else torch.empty((h, w), dtype=torch.float32, device=dev)
        fp = _dev_f32(fp, "footprint")
    _check_out(out, fp, w, h)
    cr = torch.empty((h, w, 2), dtype=torch.float64, device=dev) if coords else None
    _check(lib().dfr_reproject(
        ctypes.byref(to_c(src_wcs)), ctypes.byref(to_c(tgt_wcs)), ctypes.c_void_p(src_img.data_ptr()),
        src_img.stride(0), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(fp.data_ptr() if fp is not None else 0), out.stride(0), x0, y0, w, h,
        _order(order), _flags(precision, exact_inverse, tma, nan_mask),
        ctypes.c_void_p(cr.data_ptr() if cr is not None else 0), _stream_ptr(stream)))
    return (out, fp, cr) if coords else (out, fp)


def reproject_batch(images, src_wcs_list, tgt_wcs, bboxes=None, order="bilinear",
                    precision="split", outs=None, fps=None, footprint=True, stream=None,
                    nan_mask=False, prefiltered=False, tma=True):
    """Reproject many exposures in one launch (dfr_reproject_batch: a graph of single-frame
    kernels or one kernel over the frame table, as the autotuner picks).

    bboxes default to dfr_target_bbox per frame. Returns (values, footprints) lists."""
    torch = _torch()
    n = len(images)
    frames = (DfrFrame * max(n, 1))()
    vals, fpl, keep = [], [], []
    for i in range(n):
        img = _dev_f32(images[i], "images[%d]" % i)
        _check_image(img, src_wcs_list[i], "images[%d]" % i)
        img = _source_for(img, order, prefiltered, stream)
        keep.append(img)
        bb = bboxes[i] if bboxes is not None else target_bbox(src_wcs_list[i], tgt_wcs)
        x0, y0, w, h = (int(v) for v in bb)
        o = outs[i] if outs is not None else torch.empty((max(h, 1), max(w, 1)),
                                                          dtype=torch.float32, device=img.device)
        o = _dev_f32(o, "outs[%d]" % i)
        f = None
        if footprint:
            f = fps[i] if fps is not None else torch.empty_like(o)
            f = _dev_f32(f, "fps[%d]" % i)
        _check_out(o, f, w, h, "outs[%d]" % i)
        fr = frames[i]
        fr.wcs = to_c(src_wcs_list[i])
        fr.img = img.data_ptr()
        fr.pitch = img.stride(0)
        fr.out = o.data_ptr()
        fr.footprint = f.data_ptr() if f is not None else 0
        fr.out_pitch = o.stride(0)
        fr.x0, fr.y0, fr.w, fr.h = x0, y0, w, h
        vals.append(o)
        fpl.append(f)
    _check(lib().dfr_reproject_batch(frames, n, ctypes.byref(to_c(tgt_wcs)), _order(order),
                                     _flags(precision, False, tma, nan_mask),
                                     _stream_ptr(stream)))
    return vals, fpl


def reproject_batch_noalloc(images, src_wcs_list, tgt_wcs, bboxes, outs, fps=None,
                            order="bilinear", precision="split", stream=None, prefiltered=False,
                            tma=True):
    """dfr_reproject_batch_noalloc: the batched reprojection for callers that cannot allocate
    device memory. The library keeps its frame table in a fixed device array (at most 64
    frames per call) instead of calling cudaMalloc; the caller passes every image and output
    buffer (``outs``, optional ``fps``). For order "bspline3" the images must already hold the
    B-spline coefficients (``prefiltered=True``: the prefilter needs scratch memory, so this
    entry point does not run it). Returns (outs, fps)."""
    if _order(order) == BSPLINE3 and not prefiltered:
        raise ValueError("reproject_batch_noalloc with order bspline3 takes prefiltered "
                         "coefficients (prefiltered=True); see bspline_prefilter")
    n = len(images)
    frames = (DfrFrame * max(n, 1))()
    for i in range(n):
        img = _dev_f32(images[i], "images[%d]" % i)
        _check_image(img, src_wcs_list[i], "images[%d]" % i)
        o = _dev_f32(outs[i], "outs[%d]" % i)
        f = _dev_f32(fps[i], "fps[%d]" % i) if fps is not None else None
        _check_out(o, f, int(bboxes[i][2]), int(bboxes[i][3]), "outs[%d]" % i)
        fr = frames[i]
        fr.wcs = to_c(src_wcs_list[i])
        fr.img = img.data_ptr()
        fr.pitch = img.stride(0)
        fr.out = o.data_ptr()
        fr.footprint = f.data_ptr() if f is not None else 0
        fr.out_pitch = o.stride(0)
        fr.x0, fr.y0, fr.w, fr.h = (int(v) for v in bboxes[i])
    _check(lib().dfr_reproject_batch_noalloc(frames, n, ctypes.byref(to_c(tgt_wcs)),
                                             _order(order), _flags(precision, False, tma),
                                             _stream_ptr(stream)))
    return outs, fps


def coadd(images, src_wcs_list, tgt_wcs, bboxes=None, order="bilinear", precision="split",
          sum_vf=None, sum_f=None, stream=None, tma=True, nan_mask=False, prefiltered=False):
    """Co-add exposures onto the target grid (dfr_coadd): sum_vf += value * footprint and
    sum_f += footprint per target pixel, frames in order. ``sum_vf`` / ``sum_f`` (device,
    target-sized) are created zeroed when not given. ``bboxes`` default to (0, 0, 0, 0), which
    lets the library size each frame's box. Returns (sum_vf, sum_f)."""
    torch = _torch()
    t = to_c(tgt_wcs)
    nx, ny = int(t.naxis[0]), int(t.naxis[1])
    n = len(images)
    dev = _dev_f32(images[0], "images[0]").device if n else torch.device("cuda")
    if sum_vf is None:
        sum_vf = torch.zeros((ny, nx), dtype=torch.float32, device=dev)
    if sum_f is None:
        sum_f = torch.zeros_like(sum_vf)
    sum_vf = _dev_f32(sum_vf, "sum_vf")
    sum_f = _dev_f32(sum_f, "sum_f")
    if sum_f.stride(0) != sum_vf.stride(0) or tuple(sum_f.shape) != tuple(sum_vf.shape):
        raise ValueError("sum_vf and sum_f must share shape and row stride")
    if tuple(sum_vf.shape) != (ny, nx):
        raise ValueError("co-add sums must have the target shape (NAXIS2, NAXIS1)")
    frames = (DfrFrame * max(n, 1))()
    keep = []
    for i in range(n):
        img = _dev_f32(images[i], "images[%d]" % i)
        _check_image(img, src_wcs_list[i], "images[%d]" % i)
        img = _source_for(img, order, prefiltered, stream)
        keep.append(img)
        fr = frames[i]
        fr.wcs = to_c(src_wcs_list[i])
        fr.img = img.data_ptr()
        fr.pitch = img.stride(0)
        fr.out = 0
        fr.footprint = 0
        fr.out_pitch = 0
        bb = bboxes[i] if bboxes is not None else (0, 0, 0, 0)
        fr.x0, fr.y0, fr.w, fr.h = (int(v) for v in bb)
    _check(lib().dfr_coadd(frames, n, ctypes.byref(t), _order(order),
                           _flags(precision, False, tma, nan_mask),
                           ctypes.c_void_p(sum_vf.data_ptr()),
                           ctypes.c_void_p(sum_f.data_ptr()), sum_vf.stride(0),
                           _stream_ptr(stream)))
    return sum_vf, sum_f


def coadd_normalize(sum_vf, sum_f, min_weight=0.0, out=None, stream=None):
    """Mean of a co-add (dfr_coadd_normalize): sum_vf / sum_f where sum_f > min_weight, else 0."""
    torch = _torch()
    sum_vf = _dev_f32(sum_vf, "sum_vf")
    sum_f = _dev_f32(sum_f, "sum_f")
    if out is None:
        out = torch.empty_like(sum_vf)
    out = _dev_f32(out, "out")
    h, w = sum_vf.shape
    _check(lib().dfr_coadd_normalize(ctypes.c_void_p(sum_vf.data_ptr()),
                                     ctypes.c_void_p(sum_f.data_ptr()), sum_vf.stride(0), w, h,
                                     float(min_weight), ctypes.c_void_p(out.data_ptr()),
                                     out.stride(0), _stream_ptr(stream)))
    return out


def reproject_backward(src_img, src_wcs, tgt_wcs, grad_out, bbox, order="bilinear",
                       precision="split", exact_inverse=False, grad_src=None, want_src=True,
                       want_params=True, stream=None, tma=True):
    """Adjoint of reproject (dfr_reproject_backward): returns (grad_src, grad_params).

    ``tma=False`` selects the per-pixel kernel (no staged source / gradient boxes)."""
    torch = _torch()
    src_img = _dev_f32(src_img, "src_img")
    _check_image(src_img, src_wcs, "src_img")
    grad_out = _dev_f32(grad_out, "grad_out")
    x0, y0, w, h = (int(v) for v in bbox)
    _check_out(grad_out, None, w, h, "grad_out")
    gs = None
    if want_src:
        gs = grad_src if grad_src is not None else torch.zeros_like(src_img)
        gs = _dev_f32(gs, "grad_src")
        _check_image(gs, src_wcs, "grad_src")
    gp = torch.zeros(num_params(src_wcs), dtype=torch.float64, device=src_img.device) \
        if want_params else None
    _check(lib().dfr_reproject_backward(
        ctypes.byref(to_c(src_wcs)), ctypes.byref(to_c(tgt_wcs)),
        ctypes.c_void_p(src_img.data_ptr()), src_img.stride(0),
        ctypes.c_void_p(grad_out.data_ptr()), grad_out.stride(0), x0, y0, w, h, _order(order),
        _flags(precision, exact_inverse, tma),
        ctypes.c_void_p(gs.data_ptr() if gs is not None else 0), gs.stride(0) if gs is not None else 0,
        ctypes.c_void_p(gp.data_ptr() if gp is not None else 0), _stream_ptr(stream)))
    return gs, gp


def reproject_backward_batch(src_imgs, src_wcss, tgt_wcs, grad_outs, bboxes, order="bilinear",
                             precision="split", exact_inverse=False, grad_srcs=None,
                             want_src=True, want_params=True, stream=None, tma=True):
    """Batched adjoint (dfr_reproject_backward_batch): the reproject_backward calls of every
    frame at once. Returns (list of grad_src or None, list of grad_params or None)."""
    torch = _torch()
    n = len(src_imgs)
    if not (len(src_wcss) == len(grad_outs) == len(bboxes) == n):
        raise ValueError("src_imgs, src_wcss, grad_outs and bboxes must have the same length")
    if grad_srcs is not None and len(grad_srcs) != n:
        raise ValueError("grad_srcs must have one entry per frame")
    arr = (DfrBwdFrame * max(n, 1))()
    keep, gss, gps = [], [], []
    for f in range(n):
        img = _dev_f32(src_imgs[f], "src_imgs[%d]" % f)
        _check_image(img, src_wcss[f], "src_imgs[%d]" % f)
        go = _dev_f32(grad_outs[f], "grad_outs[%d]" % f)
        x0, y0, w, h = (int(v) for v in bboxes[f])
        _check_out(go, None, w, h, "grad_outs[%d]" % f)
        gs = None
        if want_src:
            gs = grad_srcs[f] if grad_srcs is not None else torch.zeros_like(img)
            gs = _dev_f32(gs, "grad_srcs[%d]" % f)
            _check_image(gs, src_wcss[f], "grad_srcs[%d]" % f)
        gp = torch.zeros(num_params(src_wcss[f]), dtype=torch.float64, device=img.device) \
            if want_params else None
        fr = arr[f]
        fr.wcs = to_c(src_wcss[f])
        fr.img, fr.pitch = img.data_ptr(), img.stride(0)
        fr.grad_out, fr.go_pitch = go.data_ptr(), go.stride(0)
        fr.x0, fr.y0, fr.w, fr.h = x0, y0, w, h
        fr.grad_src = gs.data_ptr() if gs is not None else 0
        fr.gs_pitch = gs.stride(0) if gs is not None else 0
        fr.grad_params = gp.data_ptr() if gp is not None else 0
        keep += [img, go]
        gss.append(gs)
        gps.append(gp)
    _check(lib().dfr_reproject_backward_batch(arr, n, ctypes.byref(to_c(tgt_wcs)), _order(order),
                                              _flags(precision, exact_inverse, tma),
                                              _stream_ptr(stream)))
    return gss, gps


def _host_ptr(a, name, shape=None):
    """(pointer, row stride in elements) of a host float32 2-D array or CPU tensor."""
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float32 or a.dim() != 2 or a.stride(1) != 1:
            raise ValueError("%s must be a 2-D float32 host tensor with unit x stride" % name)
        t = a
        ptr, stride = t.data_ptr(), t.stride(0)
    else:
        if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.ndim == 2
                and a.strides[1] == 4 and a.strides[0] % 4 == 0):
            raise ValueError("%s must be a 2-D float32 array with unit x stride" % name)
        t = a
        ptr, stride = a.ctypes.data, a.strides[0] // 4
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return ptr, stride


def reproject_host(src_img, src_wcs, tgt_wcs, shape_out=None, bbox=None, order="bilinear",
                   precision="split", exact_inverse=False, out=None, fp_out=None,
                   footprint=True, nan_mask=False):
    """Host image in, host (value, footprint) out (dfr_reproject_host): bands of the output are
    copied in, computed and copied out on overlapping streams. Inputs and outputs are float32
    numpy arrays or CPU tensors; page-locked tensors (``pin_memory()``) let the copies overlap.
    Returns (value, footprint or None), the given ``out`` / ``fp_out`` when passed."""
    if bbox is None:
        if shape_out is None:
            nax = tgt_wcs.naxis if isinstance(tgt_wcs, DfrWcs) else tgt_wcs["naxis"]
            shape_out = (int(nax[1]), int(nax[0]))
        bbox = (0, 0, int(shape_out[1]), int(shape_out[0]))
    x0, y0, w, h = (int(v) for v in bbox)
    if not isinstance(src_img, np.ndarray) and not hasattr(src_img, "data_ptr"):
        src_img = np.ascontiguousarray(src_img, dtype=np.float32)
    ip, istride = _host_ptr(src_img, "src_img")
    nx, ny = _naxis(src_wcs)
    if src_img.shape[0] < ny or src_img.shape[1] < nx:
        raise ValueError("src_img has shape %s, smaller than the WCS NAXIS (%d, %d)"
                         % (tuple(src_img.shape), ny, nx))
    if out is None:
        out = np.empty((h, w), np.float32)
    op, ostride = _host_ptr(out, "out", (h, w))
    fp = None
    fpp = 0
    if footprint:
        fp = fp_out if fp_out is not None else np.empty((h, w), np.float32)
        fpp, fstride = _host_ptr(fp, "fp_out", (h, w))
        if fstride != ostride:
            raise ValueError("out and fp_out must share the row stride")
    _check(lib().dfr_reproject_host(
        ctypes.byref(to_c(src_wcs)), ctypes.byref(to_c(tgt_wcs)), ctypes.c_void_p(ip), istride,
        ctypes.c_void_p(op), ctypes.c_void_p(fpp), ostride, x0, y0, w, h, _order(order),
        _flags(precision, exact_inverse, True, nan_mask)))
    return out, fp


def calculate_reprojection(source_img, source_wcs, target_wcs, shape_out=None, order="bilinear",
                           precision="split"):
    """Paper-style call (Sec. 2): host image in, host (value, footprint) out.

    ``source_wcs`` / ``target_wcs`` may be WCS records or FITS header text; ``shape_out``
    defaults to the target NAXIS. The work runs on the current CUDA device through
    dfr_reproject_host (copies overlapped with the computation)."""
    if isinstance(source_wcs, (str, bytes)):
        source_wcs = wcs_from_header(source_wcs)
    if isinstance(target_wcs, (str, bytes)):
        target_wcs = wcs_from_header(target_wcs)
    img = np.ascontiguousarray(source_img, dtype=np.float32)
    return reproject_host(img, source_wcs, target_wcs, shape_out=shape_out, order=order,
                          precision=precision)


def _autograd():
    torch = _torch()

    class Reproject(torch.autograd.Function):
        """value = reproject(src_img; src WCS parameters theta). Differentiable with respect to
        the source image and the parameter vector theta (layout of dfr_reproject_backward)."""

        @staticmethod
        def forward(ctx, src_img, theta, src_wcs, tgt_wcs, bbox, order, precision, exact_inverse):
            w = set_params(src_wcs, theta.detach().cpu().numpy())
            val, _ = reproject(src_img, w, tgt_wcs, bbox=bbox, order=order, precision=precision,
                               exact_inverse=exact_inverse, footprint=False)
            ctx.save_for_backward(src_img)
            ctx.cfg = (w, tgt_wcs, bbox, order, precision, exact_inverse)
            return val

        @staticmethod
        def backward(ctx, grad_out):
            (src_img,) = ctx.saved_tensors
            w, tgt_wcs, bbox, order, precision, exact_inverse = ctx.cfg
            gs, gp = reproject_backward(src_img, w, tgt_wcs, grad_out.contiguous(), bbox, order,
                                        precision, exact_inverse,
                                        want_src=ctx.needs_input_grad[0],
                                        want_params=ctx.needs_input_grad[1])
            return gs, gp, None, None, None, None, None, None

    return Reproject


def param_vector(w):
    """Source parameter vector in the dfr_reproject_backward layout."""
    vals = [w["crval"][0], w["crval"][1], w["cd"][0][0], w["cd"][0][1], w["cd"][1][0],
            w["cd"][1][1]]
    for k in ("a", "b"):
        arr = np.asarray(w[k])
        for n in range(1, int(w[k + "_order"]) + 1):
            for p in range(n, -1, -1):
                vals.append(float(arr[p, n - p]))
    return np.array(vals, dtype=np.float64)


def set_params(w, theta):
    """Copy of w with the parameter vector ``theta`` written back."""
    out = dict(w)
    out["crval"] = (float(theta[0]), float(theta[1]))
    out["cd"] = [[float(theta[2]), float(theta[3])], [float(theta[4]), float(theta[5])]]
    idx = 6
    for k in ("a", "b"):
        arr = np.array(w[k], dtype=np.float64, copy=True)
        for n in range(1, int(w[k + "_order"]) + 1):
            for p in range(n, -1, -1):
                arr[p, n - p] = theta[idx]
                idx += 1
        out[k] = arr
    return out


class _LazyReproject:
    _cls = None

    def apply(self, *args):
        if _LazyReproject._cls is None:
            _LazyReproject._cls = _autograd()
        return _LazyReproject._cls.apply(*args)


Reproject = _LazyReproject()
