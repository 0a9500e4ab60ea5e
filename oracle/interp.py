"""Oracle interpolation with footprint normalisation, in FP64 (TEST INFRASTRUCTURE).

Sec. 3.1 step 3 interpolates the source at the computed positions and, alongside it, an
all-ones "identity tensor" (the footprint); the result is divided by the footprint. The paper
names three schemes (nearest, bilinear, bicubic, Sec. 4.2) without defining them further.
Readings taken here:

  * Pixel centres are at integer 0-based coordinates (Sec. 3.2 shifts by one pixel).
  * Taps outside [0, W-1] x [0, H-1] contribute zero (the ones-image is zero-padded too), so
    footprint = sum of in-bounds weights and value = sum(w * S) / footprint over in-bounds taps.
  * A position is covered iff -0.5 <= x <= W - 0.5 and -0.5 <= y <= H - 0.5 (and the sky
    position projects onto the source); uncovered pixels get value 0 and footprint 0, and so
    does any pixel whose footprint is 0.
  * nearest: index floor(x + 0.5) (round half up).
  * bilinear: tent weights (1 - t, t) at floor(x), floor(x) + 1.
  * bicubic: Keys (1981) cubic convolution with parameter a (default -0.5), taps floor(x) - 1
    .. floor(x) + 2, written from its piecewise kernel definition.
  * lanczos3 (an extension beyond the paper's three schemes): the Lanczos kernel
    L(d) = sinc(d) sinc(d / 3) for |d| < 3, taps floor(x) - 2 .. floor(x) + 3, weights divided
    by their sum along each axis (so they sum to 1 and a constant is reproduced).
  * FP64 snapping: a coordinate within 1e-9 px of an integer is taken as that integer (so that
    an identity map returns its input bit for bit despite round-off in the transform).
"""
from __future__ import annotations

import numpy as np

NEAREST, BILINEAR, BICUBIC, LANCZOS3 = 0, 1, 2, 3
SNAP_PX = 1e-9


def keys_kernel(s, a=-0.5):
    """Keys cubic convolution kernel W(s)."""
    s = np.abs(s)
    out = np.zeros_like(s, dtype=np.float64)
    m1 = s <= 1.0
    m2 = (s > 1.0) & (s < 2.0)
    out[m1] = (a + 2.0) * s[m1] ** 3 - (a + 3.0) * s[m1] ** 2 + 1.0
    out[m2] = a * s[m2] ** 3 - 5.0 * a * s[m2] ** 2 + 8.0 * a * s[m2] - 4.0 * a
    return out


def lanczos3_kernel(d):
    """L(d) = sinc(d) sinc(d / 3) for |d| < 3, else 0 (numpy's sinc is sin(pi x) / (pi x))."""
    d = np.asarray(d, dtype=np.float64)
    return np.where(np.abs(d) < 3.0, np.sinc(d) * np.sinc(d / 3.0), 0.0)


def taps_1d(coord, order, a=-0.5):
    """(first tap index, weights[k, n]) along one axis for the given scheme."""
    if order == NEAREST:
        i0 = np.floor(coord + 0.5)
        return i0.astype(np.int64), np.ones((1,) + coord.shape)
    i0 = np.floor(coord)
    t = coord - i0
    if order == BILINEAR:
        return i0.astype(np.int64), np.stack([1.0 - t, t])
    if order == BICUBIC:
        w = np.stack([keys_kernel(t + 1.0, a), keys_kernel(t, a),
                      keys_kernel(1.0 - t, a), keys_kernel(2.0 - t, a)])
        return (i0 - 1).astype(np.int64), w
    if order == LANCZOS3:
        w = np.stack([lanczos3_kernel(t + 2.0 - k) for k in range(6)])
        return (i0 - 2).astype(np.int64), w / w.sum(axis=0)
    raise ValueError("order")


def snap(c):
    r = np.rint(c)
    return np.where(np.abs(c - r) < SNAP_PX, r, c)


def covered(img_shape, x, y, valid=None):
    H, W = img_shape
    ok = np.isfinite(x) & np.isfinite(y)
    ok &= (x >= -0.5) & (x <= W - 0.5) & (y >= -0.5) & (y <= H - 0.5)
    if valid is not None:
        ok &= valid
    return ok


def interpolate(img, x, y, order, valid=None, a=-0.5, use_snap=True, nan_mask=False):
    """Value and footprint of ``img`` (H x W) at positions (x, y). Returns float64 arrays.

    nan_mask: NaN source pixels count as missing, like pixels outside the image: they take no
    weight in the value or the footprint. A pixel is then covered only where the remaining
    weight is positive (bicubic weights can be negative, so masking may leave a sum <= 0)."""
    img = np.asarray(img)
    H, W = img.shape
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if use_snap:
        x, y = snap(x), snap(y)
    ok = covered(img.shape, x, y, valid)
    xs = np.where(ok, x, 0.0)
    ys = np.where(ok, y, 0.0)
    ix, wx = taps_1d(xs, order, a)
    iy, wy = taps_1d(ys, order, a)
    num = np.zeros(x.shape)
    fp = np.zeros(x.shape)
    for j in range(wy.shape[0]):
        yy = iy + j
        iny = (yy >= 0) & (yy < H)
        for i in range(wx.shape[0]):
            xx = ix + i
            inside = iny & (xx >= 0) & (xx < W) & ok
            w = wx[i] * wy[j]
            s = img[np.clip(yy, 0, H - 1), np.clip(xx, 0, W - 1)].astype(np.float64)
            if nan_mask:
                inside = inside & ~np.isnan(s)
            num += np.where(inside, w * s, 0.0)
            fp += np.where(inside, w, 0.0)
    live = ok & ((fp > 0.0) if nan_mask else (fp != 0.0))
    val = np.where(live, num / np.where(live, fp, 1.0), 0.0)
    fp = np.where(live, fp, 0.0)
    return val, fp


def interpolate_adjoint(img_shape, x, y, order, grad_val, valid=None, a=-0.5, use_snap=True):
    """Transpose of ``interpolate`` with respect to the source pixels: returns dL/dS given
    dL/dval, i.e. dL/dS[j] = sum over (pixel, tap hitting j) of grad * w / footprint."""
    H, W = img_shape
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if use_snap:
        x, y = snap(x), snap(y)
    ok = covered(img_shape, x, y, valid)
    xs = np.where(ok, x, 0.0)
    ys = np.where(ok, y, 0.0)
    ix, wx = taps_1d(xs, order, a)
    iy, wy = taps_1d(ys, order, a)
    fp = np.zeros(x.shape)
    for j in range(wy.shape[0]):
        for i in range(wx.shape[0]):
            yy, xx = iy + j, ix + i
            inside = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W) & ok
            fp += np.where(inside, wx[i] * wy[j], 0.0)
    live = ok & (fp != 0.0)
    g = np.where(live, np.asarray(grad_val, dtype=np.float64) / np.where(live, fp, 1.0), 0.0)
    out = np.zeros((H, W))
    for j in range(wy.shape[0]):
        for i in range(wx.shape[0]):
            yy, xx = iy + j, ix + i
            inside = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W) & live
            np.add.at(out, (yy[inside], xx[inside]), (wx[i] * wy[j] * g)[inside])
    return out
