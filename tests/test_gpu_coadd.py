"""GPU parity of the co-add (dfr_coadd, dfr_coadd_normalize) through the C ABI.

  * sums vs the oracle: the oracle interpolates every frame at the GPU's own source coordinates
    (FP64) and adds value * footprint and footprint in FP64; |sum_vf - ref| <= 1e-5 *
    max(sum |value| footprint, 1) and |sum_f - ref| <= 1e-5 per pixel; the FP64 path is also
    compared with the oracle co-add end to end;
  * the co-add equals the FP32 sum, in frame order, of the single-frame outputs: sum_f bit for
    bit, sum_vf bit for bit wherever every footprint is 0 or 1 (one rounding either way);
  * the mean is sum_vf / sum_f in IEEE FP32 (bit for bit), 0 where the weight is <= min_weight;
  * splitting the frame list over two calls gives the same bits as one call;
  * the stack configuration (32 x 6000x4000 -> 12000x8000, bicubic) at full size, sampled.
"""
import numpy as np
import pytest

import synth
from oracle import interp as OI
from oracle import reproject as OR
from oracle import wcs as OW

from gpu_util import dfr, gpu, to_dev, torch

pytestmark = pytest.mark.gpu


def _stack(seed=31, n=6, w=300, h=220):
    rng = synth.rng_for(seed)
    srcs, imgs = [], []
    for k in range(n):
        s = synth.tan_wcs(w, h, rho_deg=float(rng.uniform(-3, 3)),
                          crpix=((w + 1) / 2 + rng.uniform(-90, 90), (h + 1) / 2 + rng.uniform(-70, 70)))
        s = synth.add_sip(s, 3, 1e-6, rng)
        s["a"] *= 50.0
        s["b"] *= 50.0
        s, _ = OW.with_inverse_sip(s, 4)
        srcs.append(s)
        imgs.append(synth.sky_image(w, h, 25, rng))
    tgt = synth.tan_wcs(420, 330, rho_deg=0.8)
    return srcs, imgs, tgt


def _reference_at_gpu_coords(srcs, imgs, tgt, order, precision):
    """FP64 sums of the oracle's interpolation at each frame's GPU coordinates, the GPU's single
    frame outputs, and sum |value| footprint (for the tolerance)."""
    NX, NY = tgt["naxis"]
    rv, rf, mag = (np.zeros((NY, NX)) for _ in range(3))
    singles = []
    for s, img in zip(srcs, imgs):
        bb = dfr().target_bbox(s, tgt)
        x0, y0, w, h = bb
        if w == 0 or h == 0:
            singles.append((bb, None, None))
            continue
        v, f, cr = gpu(s, tgt, to_dev(img), order, precision, bb)
        x, y = cr[..., 0].ravel(), cr[..., 1].ravel()
        ok = np.isfinite(x) & np.isfinite(y)
        src_img = OI.bspline3_prefilter(img) if order == "bspline3" else img
        ov, of = OI.interpolate(src_img, np.where(ok, x, np.nan), np.where(ok, y, np.nan),
                                OR.ORDERS[order], valid=ok, use_snap=(precision == "fp64"))
        assert np.array_equal(of != 0, f.ravel() != 0)
        rv[y0:y0 + h, x0:x0 + w] += (ov * of).reshape(h, w)
        rf[y0:y0 + h, x0:x0 + w] += of.reshape(h, w)
        mag[y0:y0 + h, x0:x0 + w] += (np.abs(ov) * of).reshape(h, w)
        singles.append((bb, v, f))
    return rv, rf, mag, singles


@pytest.mark.parametrize("order", ["nearest", "bilinear", "bicubic", "lanczos3", "bspline3"])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_coadd_matches_oracle_and_single_frames(order, precision):
    srcs, imgs, tgt = _stack()
    sv, sf = dfr().coadd([to_dev(i) for i in imgs], srcs, tgt, order=order, precision=precision)
    torch().cuda.synchronize()
    dfr().device_status()
    sv, sf = sv.cpu().numpy(), sf.cpu().numpy()
    rv, rf, mag, singles = _reference_at_gpu_coords(srcs, imgs, tgt, order, precision)
    assert (rf > 0).mean() > 0.5 and rf.max() >= 3
    assert np.abs(sf - rf).max() <= 1e-5
    assert np.all(np.abs(sv - rv) <= 1e-5 * np.maximum(mag, 1.0))
    # FP32 sequential accumulation of the single-frame outputs, frame order
    av = np.zeros_like(sv)
    af = np.zeros_like(sf)
    unit = np.ones(sv.shape, bool)
    for bb, v, f in singles:
        if v is None:
            continue
        x0, y0, w, h = bb
        av[y0:y0 + h, x0:x0 + w] += v * f
        af[y0:y0 + h, x0:x0 + w] += f
        unit[y0:y0 + h, x0:x0 + w] &= (f == 0) | (f == 1)
    assert np.array_equal(sf, af)
    assert np.array_equal(sv[unit], av[unit])
    assert np.all(np.abs(sv - av) <= 1e-6 * np.maximum(np.abs(av), 1.0))
    if precision == "fp64":
        src_imgs = [OI.bspline3_prefilter(i) if order == "bspline3" else i for i in imgs]
        ov, of = OR.coadd(list(zip(srcs, src_imgs)), tgt, order)
        assert np.abs(sf - of).max() <= 1e-5
        assert np.all(np.abs(sv - ov) <= 1e-5 * np.maximum(mag, 1.0))


def test_coadd_normalize_and_incremental_calls():
    srcs, imgs, tgt = _stack(seed=32)
    d = [to_dev(i) for i in imgs]
    sv, sf = dfr().coadd(d, srcs, tgt, order="bicubic")
    sv2, sf2 = dfr().coadd(d[:2], srcs[:2], tgt, order="bicubic")
    dfr().coadd(d[2:], srcs[2:], tgt, order="bicubic", sum_vf=sv2, sum_f=sf2)
    assert torch().equal(sv, sv2) and torch().equal(sf, sf2)
    m = dfr().coadd_normalize(sv, sf).cpu().numpy()
    a, b = sv.cpu().numpy(), sf.cpu().numpy()
    cov = b > 0
    assert np.array_equal(m[cov], (a[cov] / b[cov]).astype(np.float32))
    assert np.all(m[~cov] == 0)
    m2 = dfr().coadd_normalize(sv, sf, min_weight=1.5).cpu().numpy()
    assert np.all(m2[b <= 1.5] == 0) and np.array_equal(m2[b > 1.5], m[b > 1.5])
    # unaligned views take the scalar kernel: same bits
    m3 = dfr().coadd_normalize(sv[:, 1:], sf[:, 1:]).cpu().numpy()
    assert np.array_equal(m3, m[:, 1:])
    # in place: the mean overwrites sum_vf
    dfr().coadd_normalize(sv, sf, out=sv)
    assert np.array_equal(sv.cpu().numpy(), m)
    torch().cuda.synchronize()
    dfr().device_status()


def test_coadd_explicit_boxes_and_no_tma():
    srcs, imgs, tgt = _stack(seed=33, n=4)
    d = [to_dev(i) for i in imgs]
    bbs = [dfr().target_bbox(s, tgt) for s in srcs]
    a = dfr().coadd(d, srcs, tgt, bboxes=bbs, order="bilinear")
    b = dfr().coadd(d, srcs, tgt, order="bilinear")
    c = dfr().coadd(d, srcs, tgt, order="bilinear", tma=False)
    for x, y in ((a, b), (a, c)):
        assert torch().equal(x[0], y[0]) and torch().equal(x[1], y[1])


def test_config4_coadd_full_size_sampled():
    T = torch()
    c = synth.config4()
    tgt = c["tgt"]
    srcs = [OW.with_inverse_sip(s, 6)[0] for s in c["src"]]
    imgs_d = [to_dev(i) for i in c["images"]]
    sv, sf = dfr().coadd(imgs_d, srcs, tgt, order="bicubic")
    T.cuda.synchronize()
    dfr().device_status()
    # sampled target pixels inside the first frame's box (the dithered frames overlap there),
    # with the oracle at each frame's GPU coordinates
    rng = synth.rng_for(405)
    bx0, by0, bw, bh = dfr().target_bbox(srcs[0], tgt)
    px = bx0 + rng.integers(0, bw, 3000)
    py = by0 + rng.integers(0, bh, 3000)
    rv, rf, mag = np.zeros(3000), np.zeros(3000), np.zeros(3000)
    for k in range(32):
        bb = dfr().target_bbox(srcs[k], tgt)
        x0, y0, w, h = bb
        inside = (px >= x0) & (px < x0 + w) & (py >= y0) & (py < y0 + h)
        if not inside.any():
            continue
        v, f, cr = dfr().reproject(imgs_d[k], srcs[k], tgt, bbox=bb, order="bicubic", coords=True)
        iy = T.from_numpy(py[inside] - y0).cuda()
        ix = T.from_numpy(px[inside] - x0).cuda()
        crs = cr[iy, ix].cpu().numpy()
        ok = np.isfinite(crs[:, 0])
        ov, of = OI.interpolate(c["images"][k], np.where(ok, crs[:, 0], np.nan),
                                np.where(ok, crs[:, 1], np.nan), OR.ORDERS["bicubic"], valid=ok,
                                use_snap=False)
        rv[inside] += ov * of
        rf[inside] += of
        mag[inside] += np.abs(ov) * of
        del v, f, cr
    g_v = sv[T.from_numpy(py).cuda(), T.from_numpy(px).cuda()].cpu().numpy()
    g_f = sf[T.from_numpy(py).cuda(), T.from_numpy(px).cuda()].cpu().numpy()
    assert (rf > 0).mean() > 0.9 and rf.max() >= 20
    assert np.abs(g_f - rf).max() <= 1e-5 * 32
    assert np.all(np.abs(g_v - rv) <= 1e-5 * np.maximum(mag, 1.0))
