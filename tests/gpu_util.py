"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and compare it with the
oracle element by element. Test-only code."""
import numpy as np

import synth
from oracle import interp as OI
from oracle import reproject as OR
from oracle import wcs as OW

VALUE_RTOL = 1e-5        # |gpu - oracle| <= 1e-5 * max(|oracle|, 1)  (1 = sky-noise sigma)
SPLIT_PX = 1e-3          # split-precision source coordinates vs the FP64 oracle
FP64_PX = 1e-8           # all-FP64 path vs the FP64 oracle (libm differences only)


def dfr():
    import paper_2505_03932_gb300 as d
    return d


def torch():
    import torch as t
    return t


def with_inverse(cfg, k=0):
    """Source WCS of frame k with AP/BP fitted by the oracle (when it has SIP)."""
    src = cfg["src"][k]
    if src["a_order"] > 0 and cfg.get("inverse_order", 0) > 0:
        src, _ = OW.with_inverse_sip(src, cfg["inverse_order"])
    return src


def to_dev(img):
    return torch().from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()


def gpu(src, tgt, img_d, order, precision, bbox=None, exact=False, tma=True, nan_mask=False):
    """GPU value, footprint and emitted source coordinates (numpy)."""
    val, fp, cr = dfr().reproject(img_d, src, tgt, bbox=bbox, order=order, precision=precision,
                                  exact_inverse=exact, coords=True, tma=tma, nan_mask=nan_mask)
    torch().cuda.synchronize()
    dfr().device_status()
    return val.cpu().numpy(), fp.cpu().numpy(), cr.cpu().numpy()


def value_check(img, order, val, fp, cr, precision, nan_mask=False):
    """Oracle interpolation at the GPU's own coordinates; returns max normalised error.

    With nan_mask the remaining weight F can fall below the 0.25 floor of the unmasked case
    (signed bicubic weights), and FP32 rounding of the weighted sum is divided by F: the error
    is normalised by max(1, 0.25 / F) as well."""
    x = cr[..., 0].ravel()
    y = cr[..., 1].ravel()
    ok = np.isfinite(x) & np.isfinite(y)
    ov, ofp = OI.interpolate(img, np.where(ok, x, np.nan), np.where(ok, y, np.nan),
                             OR.ORDERS[order] if isinstance(order, str) else order, valid=ok,
                             use_snap=(precision == "fp64"), nan_mask=nan_mask)
    g = val.ravel().astype(np.float64)
    gf = fp.ravel().astype(np.float64)
    # coverage decisions are taken in the same precision on both sides: they must agree
    assert np.array_equal(gf != 0, ofp != 0), "coverage differs at %d pixels" % int(
        np.sum((gf != 0) != (ofp != 0)))
    err = np.abs(g - ov) / np.maximum(np.abs(ov), 1.0)
    if nan_mask:
        err = err / np.maximum(1.0, 0.25 / np.where(ofp > 0, ofp, 1.0))
    ferr = np.abs(gf - ofp)
    return float(err.max(initial=0.0)), float(ferr.max(initial=0.0))


def coord_check(src, tgt, cr, bbox, inverse="poly", sample=None, rng=None):
    """Max distance (px) between GPU coordinates and the oracle's FP64 source coordinates."""
    x0, y0, w, h = bbox
    if sample is None:
        Y, X = np.mgrid[0:h, 0:w]
        X, Y = X.ravel(), Y.ravel()
    else:
        X = rng.integers(0, w, sample)
        Y = rng.integers(0, h, sample)
    ox, oy, ok = OR.coords(src, tgt, X + x0, Y + y0, inverse=inverse)
    gx = cr[Y, X, 0]
    gy = cr[Y, X, 1]
    both = ok & np.isfinite(gx)
    assert np.array_equal(ok, np.isfinite(gx)), "projection validity differs"
    d = np.hypot(gx - ox, gy - oy)[both]
    return float(d.max(initial=0.0)), float(np.sqrt(np.mean(d ** 2))) if d.size else 0.0
