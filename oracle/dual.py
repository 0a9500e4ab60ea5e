"""Forward-mode dual numbers and reprojection-loss gradients (TEST INFRASTRUCTURE).

A ``Dual`` carries a value array ``v`` and a derivative array ``d`` of shape (k,) + v.shape,
one row per differentiated parameter. The oracle's WCS code (oracle.wcs) is written over a math
namespace; passing this module as that namespace runs the very same Sec. 3.2.2 formulas on
duals, so gradients come from the definition itself rather than from hand-derived adjoints.

Parameters (source WCS, in this order): CRVAL1, CRVAL2 (degrees), CD1_1, CD1_2, CD2_1, CD2_2,
then A_pq for 1 <= p+q <= A_ORDER ordered by p+q then p descending, then B_pq likewise.
"""
from __future__ import annotations

import numpy as np

from . import interp as _interp
from . import wcs as _wcs


class Dual:
    __slots__ = ("v", "d")
    __array_priority__ = 1000
    __array_ufunc__ = None

    def __init__(self, v, d):
        self.v = np.asarray(v, dtype=np.float64)
        self.d = np.asarray(d, dtype=np.float64)

    # -- helpers
    @staticmethod
    def _lift(d, nd):
        extra = nd - (d.ndim - 1)
        if extra > 0:
            d = d.reshape((d.shape[0],) + (1,) * extra + d.shape[1:])
        return d

    def _bin(self, other, fv, fd):
        if isinstance(other, Dual):
            v = fv(self.v, other.v)
            nd = v.ndim
            return Dual(v, fd(self.v, self._lift(self.d, nd), other.v, self._lift(other.d, nd)))
        o = np.asarray(other, dtype=np.float64)
        v = fv(self.v, o)
        return Dual(v, fd(self.v, self._lift(self.d, v.ndim), o, None))

    # -- arithmetic
    def __add__(self, o):
        return self._bin(o, np.add, lambda a, da, b, db: da + db if db is not None else da + 0 * b)

    __radd__ = __add__

    def __sub__(self, o):
        return self._bin(o, np.subtract,
                         lambda a, da, b, db: da - db if db is not None else da + 0 * b)

    def __rsub__(self, o):
        return (-self) + o

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __mul__(self, o):
        return self._bin(o, np.multiply,
                         lambda a, da, b, db: da * b + a * db if db is not None else da * b)

    __rmul__ = __mul__

    def __truediv__(self, o):
        def fd(a, da, b, db):
            if db is None:
                return da / b
            return (da * b - a * db) / (b * b)
        return self._bin(o, np.divide, fd)

    def __rtruediv__(self, o):
        o = np.asarray(o, dtype=np.float64)
        v = o / self.v
        return Dual(v, -self._lift(self.d, v.ndim) * o / (self.v * self.v))

    def __pow__(self, n):
        n = int(n)
        if n == 0:
            return Dual(np.ones_like(self.v), np.zeros_like(self.d))
        return Dual(self.v ** n, n * self.v ** (n - 1) * self.d)


def _v(a):
    return a.v if isinstance(a, Dual) else np.asarray(a, dtype=np.float64)


def _dd(a, shape):
    """Derivative rows of ``a`` broadcast to ``shape`` (zeros for a plain number)."""
    if isinstance(a, Dual):
        d = Dual._lift(a.d, len(shape))
        return np.broadcast_to(d, (a.d.shape[0],) + shape)
    return None


def _unary(a, f, fprime):
    if not isinstance(a, Dual):
        return f(np.asarray(a, dtype=np.float64))
    return Dual(f(a.v), fprime(a.v) * a.d)


def sin(a):
    return _unary(a, np.sin, np.cos)


def cos(a):
    return _unary(a, np.cos, lambda x: -np.sin(x))


def sqrt(a):
    return _unary(a, np.sqrt, lambda x: 0.5 / np.sqrt(x))


def sinc(a):
    """numpy's normalised sinc, sin(pi x) / (pi x), with derivative (cos(pi x) - sinc(x)) / x;
    below |x| = 1e-3 the derivative's Taylor series -pi^2 x / 3 + pi^4 x^3 / 30 (the closed
    form cancels there)."""
    def fprime(x):
        small = np.abs(x) < 1e-3
        xs = np.where(small, 1.0, x)
        series = -np.pi ** 2 * x / 3.0 + np.pi ** 4 * x ** 3 / 30.0
        return np.where(small, series, (np.cos(np.pi * xs) - np.sinc(xs)) / xs)
    return _unary(a, np.sinc, fprime)


def arcsin(a):
    return _unary(a, np.arcsin, lambda x: 1.0 / np.sqrt(1.0 - x * x))


def arctan2(y, x):
    yv, xv = _v(y), _v(x)
    v = np.arctan2(yv, xv)
    if not isinstance(y, Dual) and not isinstance(x, Dual):
        return v
    r2 = xv * xv + yv * yv
    k = y.d.shape[0] if isinstance(y, Dual) else x.d.shape[0]
    d = np.zeros((k,) + v.shape)
    if isinstance(y, Dual):
        d = d + Dual._lift(y.d, v.ndim) * (xv / r2)
    if isinstance(x, Dual):
        d = d - Dual._lift(x.d, v.ndim) * (yv / r2)
    return Dual(v, d)


# ----------------------------------------------------------------------------- parameters
def param_names(w):
    names = ["CRVAL1", "CRVAL2", "CD1_1", "CD1_2", "CD2_1", "CD2_2"]
    for nm, order in (("A", w["a_order"]), ("B", w["b_order"])):
        for n in range(1, order + 1):
            for p in range(n, -1, -1):
                names.append("%s_%d_%d" % (nm, p, n - p))
    return names


def dual_wcs(w):
    """Copy of the WCS record whose differentiated parameters are Dual scalars."""
    names = param_names(w)
    k = len(names)

    def seed(val, idx):
        d = np.zeros(k)
        d[idx] = 1.0
        return Dual(val, d)

    out = dict(w)
    out["crval"] = (seed(w["crval"][0], 0), seed(w["crval"][1], 1))
    out["cd"] = [[seed(w["cd"][0][0], 2), seed(w["cd"][0][1], 3)],
                 [seed(w["cd"][1][0], 4), seed(w["cd"][1][1], 5)]]
    idx = 6
    for nm in ("a", "b"):
        arr = np.asarray(w[nm], dtype=np.float64)
        lst = [[float(arr[p, q]) for q in range(arr.shape[1])] for p in range(arr.shape[0])]
        order = w[nm + "_order"]
        for n in range(1, order + 1):
            for p in range(n, -1, -1):
                lst[p][n - p] = seed(float(arr[p, n - p]), idx)
                idx += 1
        out[nm] = lst
    return out, names


def flat_params(w):
    """Parameter vector in param_names order."""
    vals = [w["crval"][0], w["crval"][1], w["cd"][0][0], w["cd"][0][1], w["cd"][1][0],
            w["cd"][1][1]]
    for nm in ("a", "b"):
        arr = np.asarray(w[nm])
        for n in range(1, w[nm + "_order"] + 1):
            for p in range(n, -1, -1):
                vals.append(float(arr[p, n - p]))
    return np.array(vals, dtype=np.float64)


def set_params(w, theta):
    """Copy of w with the parameter vector ``theta`` written back."""
    out = dict(w)
    out["crval"] = (float(theta[0]), float(theta[1]))
    out["cd"] = [[float(theta[2]), float(theta[3])], [float(theta[4]), float(theta[5])]]
    idx = 6
    for nm in ("a", "b"):
        arr = np.array(w[nm], dtype=np.float64, copy=True)
        for n in range(1, w[nm + "_order"] + 1):
            for p in range(n, -1, -1):
                arr[p, n - p] = theta[idx]
                idx += 1
        out[nm] = arr
    return out


# ----------------------------------------------------------------------------- gradients
def _interp_dual(img, x, y, order, valid, a=-0.5):
    """Value of the footprint-normalised interpolation with dual coordinates (x, y)."""
    H, W = img.shape
    xv, yv = _v(x), _v(y)
    ok = _interp.covered(img.shape, xv, yv, valid)
    xs = np.where(ok, xv, 0.0)
    ys = np.where(ok, yv, 0.0)
    k = x.d.shape[0]
    n = xv.shape

    def weights(c, cv):
        if order == _interp.NEAREST:
            i0 = np.floor(cv + 0.5).astype(np.int64)
            return i0, [Dual(np.ones(n), np.zeros((k,) + n))]
        i0 = np.floor(cv)
        t = c - i0  # Dual
        if order == _interp.BILINEAR:
            return i0.astype(np.int64), [1.0 - t, t]
        if order == _interp.BSPLINE3:
            # cubic B-spline at d = t + 1 - k, k = 0..3, as polynomials in t (s = 1 - t)
            s = 1.0 - t
            w0 = s * s * s * (1.0 / 6.0)
            w1 = t * t * (0.5 * t - 1.0) + 2.0 / 3.0
            w2 = s * s * (0.5 * s - 1.0) + 2.0 / 3.0
            w3 = t * t * t * (1.0 / 6.0)
            return (i0 - 1).astype(np.int64), [w0, w1, w2, w3]
        if order == _interp.LANCZOS3:
            # L(d) = sinc(d) sinc(d / 3) at d = t + 2 - k, k = 0..5, divided by their sum
            L = [sinc(t + float(2 - k)) * sinc((t + float(2 - k)) * (1.0 / 3.0))
                 for k in range(6)]
            tot = L[0] + L[1] + L[2] + L[3] + L[4] + L[5]
            return (i0 - 2).astype(np.int64), [Lk / tot for Lk in L]
        aa = a
        # Keys kernel for the four taps at distances t+1, t, 1-t, 2-t, as polynomials in t
        w0 = aa * t * (t - 1.0) * (t - 1.0)
        w1 = (aa + 2.0) * t * t * t - (aa + 3.0) * t * t + 1.0
        s = 1.0 - t
        w2 = (aa + 2.0) * s * s * s - (aa + 3.0) * s * s + 1.0
        w3 = aa * s * t * t
        return (i0 - 1).astype(np.int64), [w0, w1, w2, w3]

    xd = Dual(xs, np.where(ok, x.d, 0.0))
    yd = Dual(ys, np.where(ok, y.d, 0.0))
    ix, wx = weights(xd, xs)
    iy, wy = weights(yd, ys)
    if order == _interp.BSPLINE3:
        # img holds B-spline coefficients, continued by mirroring; footprint 1 where covered
        num = Dual(np.zeros(n), np.zeros((k,) + n))
        for j, wyj in enumerate(wy):
            yy = _interp.mirror_index(iy + j, H)
            for i, wxi in enumerate(wx):
                xx = _interp.mirror_index(ix + i, W)
                num = num + wxi * wyj * img[yy, xx].astype(np.float64)
        return Dual(np.where(ok, num.v, 0.0), np.where(ok, num.d, 0.0))
    num = Dual(np.zeros(n), np.zeros((k,) + n))
    fp = Dual(np.zeros(n), np.zeros((k,) + n))
    for j, wyj in enumerate(wy):
        yy = iy + j
        for i, wxi in enumerate(wx):
            xx = ix + i
            inside = ((yy >= 0) & (yy < H) & (xx >= 0) & (xx < W) & ok).astype(np.float64)
            wgt = wxi * wyj * inside
            s = img[np.clip(yy, 0, H - 1), np.clip(xx, 0, W - 1)].astype(np.float64)
            num = num + wgt * s
            fp = fp + wgt
    live = ok & (fp.v != 0.0)
    safe = Dual(np.where(live, fp.v, 1.0), fp.d)
    val = num / safe
    return Dual(np.where(live, val.v, 0.0), np.where(live, val.d, 0.0))


def reproject_dual(src, tgt, img, xt, yt, order, inverse="newton"):
    """Dual-valued output of the reprojection at target pixels (xt, yt), with derivatives
    with respect to the source WCS parameters (param_names order)."""
    order = {"nearest": 0, "bilinear": 1, "bicubic": 2, "lanczos3": 3,
             "bspline3": 4}.get(order, order)
    ra, dec = _wcs.pix2world(tgt, np.asarray(xt, np.float64), np.asarray(yt, np.float64))
    dsrc, names = dual_wcs(src)
    import oracle.dual as m
    x, y, ok = _wcs.world2pix(dsrc, ra, dec, inverse=inverse, m=m)
    return _interp_dual(img, x, y, order, ok), names


def loss_grad(src, tgt, img, reference, order, inverse="newton", chunk=1 << 16, bbox=None):
    """L = sum over target pixels of (O - reference)^2 and dL/dtheta (source WCS parameters)
    by forward-mode duals; also dL/dS (source pixels) via the interpolation adjoint."""
    if bbox is None:
        bbox = (0, 0, tgt["naxis"][0], tgt["naxis"][1])
    x0, y0, w, h = bbox
    X, Y = np.meshgrid(np.arange(x0, x0 + w, dtype=np.float64),
                       np.arange(y0, y0 + h, dtype=np.float64))
    X, Y = X.ravel(), Y.ravel()
    ref = np.asarray(reference, dtype=np.float64).ravel()
    loss_parts, grad = [], None
    for s in range(0, X.size, chunk):
        e = min(s + chunk, X.size)
        o, names = reproject_dual(src, tgt, img, X[s:e], Y[s:e], order, inverse)
        r = o.v - ref[s:e]
        loss_parts.append(r * r)
        g = (2.0 * r * o.d).sum(axis=1)
        grad = g if grad is None else grad + g
    loss = float(np.sum(np.concatenate(loss_parts)))
    return loss, grad, names
