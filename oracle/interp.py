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
  * bspline3 (an extension beyond the paper's three schemes): the cubic B-spline through the
    image. The source is first turned into B-spline coefficients by the recursive prefilter
    (``bspline3_prefilter``); evaluation uses the B-spline weights on taps floor(x) - 1 ..
    floor(x) + 2, with the coefficients continued by mirroring (whole-sample symmetric) outside
    the image, so a covered pixel has footprint 1.
  * FP64 snapping: a coordinate within 1e-9 px of an integer is taken as that integer (so that
    an identity map returns its input bit for bit despite round-off in the transform).
"""
from __future__ import annotations

import numpy as np

NEAREST, BILINEAR, BICUBIC, LANCZOS3, BSPLINE3 = 0, 1, 2, 3, 4
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


def bspline3_kernel(d):
    """Cubic B-spline: 2/3 - |d|^2 + |d|^3 / 2 for |d| <= 1, (2 - |d|)^3 / 6 for 1 < |d| < 2."""
    d = np.abs(np.asarray(d, dtype=np.float64))
    return np.where(d <= 1.0, 2.0 / 3.0 - d * d + 0.5 * d ** 3,
                    np.where(d < 2.0, (2.0 - d) ** 3 / 6.0, 0.0))


def mirror_index(i, n):
    """Whole-sample symmetric extension of integer indices over [0, n)."""
    i = np.asarray(i)
    if n == 1:
        return np.zeros_like(i)
    p = 2 * (n - 1)
    i = np.mod(i, p)
    return np.where(i < n, i, p - i)


def bspline3_prefilter_1d(s, axis):
    """Cubic B-spline coefficients along one axis (mirror boundaries): the recursive filter of
    Unser, Aldroubi & Eden (1991) with pole z = sqrt(3) - 2 and gain 6 = (1 - z)(1 - 1/z):
    causal c+[k] = 6 s[k] + z c+[k-1] from c+[0] = sum_j z^j 6 s[mirror(j)], anticausal
    c[k] = z (c[k+1] - c+[k]) from c[n-1] = z / (z^2 - 1) (c+[n-1] + z c+[n-2])."""
    s = np.moveaxis(np.asarray(s, dtype=np.float64), axis, 0)
    n = s.shape[0]
    if n == 1:
        return np.moveaxis(s.copy(), 0, axis)
    z = np.sqrt(3.0) - 2.0
    horizon = int(np.ceil(np.log(1e-17) / np.log(abs(z))))
    j = np.arange(horizon)
    cp = np.empty_like(s)
    cp[0] = np.tensordot(z ** j, 6.0 * s[mirror_index(j, n)], axes=(0, 0))
    for k in range(1, n):
        cp[k] = 6.0 * s[k] + z * cp[k - 1]
    c = np.empty_like(s)
    c[n - 1] = z / (z * z - 1.0) * (cp[n - 1] + z * cp[n - 2])
    for k in range(n - 2, -1, -1):
        c[k] = z * (c[k + 1] - cp[k])
    return np.moveaxis(c, 0, axis)


def bspline3_prefilter(img):
    """2-D cubic B-spline coefficients of an image: rows, then columns."""
    return bspline3_prefilter_1d(bspline3_prefilter_1d(img, 1), 0)


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
    if order == BSPLINE3:
        w = np.stack([bspline3_kernel(t + 1.0 - k) for k in range(4)])
        return (i0 - 1).astype(np.int64), w
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
    if order == BSPLINE3:
        # img holds B-spline coefficients (bspline3_prefilter); mirrored outside the image
        val = np.zeros(x.shape)
        for j in range(4):
            yy = mirror_index(iy + j, H)
            for i in range(4):
                xx = mirror_index(ix + i, W)
                val += wx[i] * wy[j] * img[yy, xx].astype(np.float64)
        return np.where(ok, val, 0.0), np.where(ok, 1.0, 0.0)
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


def bspline3_prefilter_matrix(n):
    """The 1-D prefilter as an n x n matrix: column j is the prefilter applied to unit vector
    e_j (the map is linear, so this is the map itself)."""
    return bspline3_prefilter_1d(np.eye(n), 0)


def bspline3_prefilter_adjoint(g):
    """Transpose of ``bspline3_prefilter``: the prefilter is C = My S Mx^T (rows by Mx, then
    columns by My), so dL/dS = My^T (dL/dC) Mx."""
    g = np.asarray(g, dtype=np.float64)
    H, W = g.shape
    return bspline3_prefilter_matrix(H).T @ g @ bspline3_prefilter_matrix(W)


def interpolate_adjoint(img_shape, x, y, order, grad_val, valid=None, a=-0.5, use_snap=True):
    """Transpose of ``interpolate`` with respect to the source pixels: returns dL/dS given
    dL/dval, i.e. dL/dS[j] = sum over (pixel, tap hitting j) of grad * w / footprint. For
    bspline3 the source pixels are the B-spline coefficients (mirrored taps, footprint 1);
    compose with ``bspline3_prefilter_adjoint`` for the image itself."""
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
    if order == BSPLINE3:
        g = np.where(ok, np.asarray(grad_val, dtype=np.float64), 0.0)
        out = np.zeros((H, W))
        for j in range(4):
            yy = mirror_index(iy + j, H)
            for i in range(4):
                xx = mirror_index(ix + i, W)
                np.add.at(out, (yy[ok], xx[ok]), (wx[i] * wy[j] * g)[ok])
        return out
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
