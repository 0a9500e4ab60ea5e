"""Oracle reprojection (TEST INFRASTRUCTURE): Sec. 3.1 steps 1-3 per target pixel, FP64, and the
co-add of several reprojected exposures (the combination the method serves, Sec. 1).

For each target pixel: pixel -> world with the target WCS (Sec. 3.2.1), world -> source pixel
with the source WCS (Sec. 3.2.2), then interpolation of the source and of the footprint
(Sec. 3.1 step 3). Target pixels are given either as a bounding box of the target grid or as
an explicit list; work is split into chunks of pixels only to bound memory (every pixel is
independent, so chunking does not change any result).
"""
from __future__ import annotations

import numpy as np

from . import interp as _interp
from . import wcs as _wcs

ORDERS = {"nearest": _interp.NEAREST, "bilinear": _interp.BILINEAR, "bicubic": _interp.BICUBIC,
          "lanczos3": _interp.LANCZOS3, "bspline3": _interp.BSPLINE3}
CHUNK = 1 << 20


def _order(order):
    return ORDERS[order] if isinstance(order, str) else int(order)


def coords(src, tgt, xt, yt, inverse="poly"):
    """Source pixel coordinates (x_s, y_s, valid) of target pixels (xt, yt)."""
    return _wcs.source_coords(src, tgt, np.asarray(xt, np.float64), np.asarray(yt, np.float64),
                              inverse=inverse)


def reproject_pixels(src, tgt, img, xt, yt, order, inverse="poly", use_snap=True,
                     nan_mask=False):
    """Value, footprint, x_s, y_s at an explicit list of target pixels (nan_mask: NaN source
    pixels are missing, see interp.interpolate)."""
    order = _order(order)
    xt = np.asarray(xt, np.float64).ravel()
    yt = np.asarray(yt, np.float64).ravel()
    val = np.empty(xt.shape)
    fp = np.empty(xt.shape)
    xs = np.empty(xt.shape)
    ys = np.empty(xt.shape)
    for s in range(0, xt.size, CHUNK):
        e = min(s + CHUNK, xt.size)
        x, y, ok = coords(src, tgt, xt[s:e], yt[s:e], inverse)
        x = np.where(ok, x, np.nan)
        y = np.where(ok, y, np.nan)
        val[s:e], fp[s:e] = _interp.interpolate(img, x, y, order, valid=ok, use_snap=use_snap,
                                                nan_mask=nan_mask)
        xs[s:e], ys[s:e] = x, y
    return val, fp, xs, ys


def reproject(src, tgt, img, order, bbox=None, inverse="poly", use_snap=True, nan_mask=False):
    """Reproject ``img`` (source WCS ``src``) onto the target grid ``tgt``.

    bbox = (x0, y0, w, h) in target pixels; default the whole target (NAXIS1 x NAXIS2).
    Returns (value, footprint, x_s, y_s), each h x w float64."""
    if bbox is None:
        bbox = (0, 0, tgt["naxis"][0], tgt["naxis"][1])
    x0, y0, w, h = bbox
    X, Y = np.meshgrid(np.arange(x0, x0 + w, dtype=np.float64),
                       np.arange(y0, y0 + h, dtype=np.float64))
    val, fp, xs, ys = reproject_pixels(src, tgt, img, X, Y, order, inverse, use_snap, nan_mask)
    return (val.reshape(h, w), fp.reshape(h, w), xs.reshape(h, w), ys.reshape(h, w))


def target_bbox(src, tgt, samples=64, margin=2):
    """Target-pixel bounding box (x0, y0, w, h) of the source frame: the source boundary,
    sampled ``samples`` points per edge, mapped pixel -> world (source) -> pixel (target),
    widened by ``margin`` px and clipped to the target grid."""
    W, H = src["naxis"]
    t = np.linspace(0.0, 1.0, samples)
    ex = np.concatenate([-0.5 + t * W, np.full(samples, W - 0.5), -0.5 + t * W,
                         np.full(samples, -0.5)])
    ey = np.concatenate([np.full(samples, -0.5), -0.5 + t * H, np.full(samples, H - 0.5),
                         -0.5 + t * H])
    ra, dec = _wcs.pix2world(src, ex, ey)
    x, y, ok = _wcs.world2pix(tgt, ra, dec, inverse="newton")
    x, y = x[ok], y[ok]
    TW, TH = tgt["naxis"]
    if x.size == 0:
        return (0, 0, 0, 0)
    x0 = max(int(np.floor(x.min())) - margin, 0)
    y0 = max(int(np.floor(y.min())) - margin, 0)
    x1 = min(int(np.ceil(x.max())) + margin, TW - 1)
    y1 = min(int(np.ceil(y.max())) + margin, TH - 1)
    if x1 < x0 or y1 < y0:
        return (0, 0, 0, 0)
    return (x0, y0, x1 - x0 + 1, y1 - y0 + 1)


def coadd(frames, tgt, order, pixels=None, inverse="poly", nan_mask=False):
    """Co-add of exposures on the target grid, FP64: for every target pixel the sums over the
    frames of value * footprint and of footprint, value and footprint as in ``reproject``
    (a frame contributes 0 where it does not cover the pixel). The mean image is
    sum_vf / sum_f where sum_f > 0.

    frames: list of (src_wcs, img). pixels: optional (xt, yt) arrays of target pixels; default
    the whole target grid (NAXIS2 x NAXIS1 arrays). Returns (sum_vf, sum_f)."""
    if pixels is None:
        TW, TH = tgt["naxis"]
        Y, X = np.mgrid[0:TH, 0:TW].astype(np.float64)
        shape = (TH, TW)
    else:
        X = np.asarray(pixels[0], np.float64)
        Y = np.asarray(pixels[1], np.float64)
        shape = X.shape
    sum_vf = np.zeros(X.size)
    sum_f = np.zeros(X.size)
    for src, img in frames:
        val, fp, _, _ = reproject_pixels(src, tgt, img, X.ravel(), Y.ravel(), order, inverse,
                                         nan_mask=nan_mask)
        sum_vf += val * fp
        sum_f += fp
    return sum_vf.reshape(shape), sum_f.reshape(shape)
