"""GPU parity of dfr_reproject with the FP64 oracle (element by element), through the C ABI.

Criteria (derived from the 1e-3 px / 1e-5 relative targets):
  * source coordinates: all-FP64 path within 1e-8 px of the oracle, split path within 1e-3 px;
  * values: the oracle interpolates at the GPU's own emitted coordinates (same coverage
    decisions, taken on the same numbers) and |gpu - oracle| <= 1e-5 * max(|oracle|, 1);
  * end to end (oracle coordinates) the FP64 path meets the same 1e-5 bound.
"""
import numpy as np
import pytest

import synth
from oracle import interp as OI
from oracle import reproject as OR
from oracle import wcs as OW

from gpu_util import (FP64_PX, SPLIT_PX, VALUE_RTOL, coord_check, dfr, gpu, to_dev, torch,
                      value_check, with_inverse)

pytestmark = pytest.mark.gpu


def _small_sip(order="bicubic", w=700, h=450, seed=7, tgt_rot=1.2, scale=1.01,
               shift=(41.3, -17.9), sip_order=3, inv_order=4):
    rng = synth.rng_for(seed)
    src = synth.add_sip(synth.tan_wcs(w, h), sip_order, 1e-6, rng)
    src, _ = OW.with_inverse_sip(src, inv_order)
    tgt = synth.tan_wcs(w + 37, h - 21, scale_arcsec=2.5 * scale, rho_deg=tgt_rot,
                        crpix=(src["crpix"][0] + shift[0], src["crpix"][1] + shift[1]))
    img = synth.sky_image(w, h, synth.sources_for_area(w, h, 6000), rng)
    return src, tgt, img


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_config0_full(precision):
    c = synth.config0()
    src, tgt, img = c["src"][0], c["tgt"], c["images"][0]
    bbox = (0, 0, 512, 512)
    val, fp, cr = gpu(src, tgt, to_dev(img), "bilinear", precision, bbox)
    dmax, _ = coord_check(src, tgt, cr, bbox)
    assert dmax < (FP64_PX if precision == "fp64" else SPLIT_PX)
    e, fe = value_check(img, "bilinear", val, fp, cr, precision)
    assert e <= VALUE_RTOL and fe <= 1e-6
    if precision == "fp64":
        ov, ofp, _, _ = OR.reproject(src, tgt, img, "bilinear")
        err = np.abs(val - ov) / np.maximum(np.abs(ov), 1.0)
        assert err.max() <= VALUE_RTOL
        assert np.abs(fp - ofp).max() <= 1e-6


@pytest.mark.parametrize("order", ["nearest", "bilinear", "bicubic", "lanczos3"])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_sip_ragged_tiles(order, precision):
    src, tgt, img = _small_sip()
    bbox = (0, 0, tgt["naxis"][0], tgt["naxis"][1])
    val, fp, cr = gpu(src, tgt, to_dev(img), order, precision, bbox)
    dmax, _ = coord_check(src, tgt, cr, bbox)
    assert dmax < (FP64_PX if precision == "fp64" else SPLIT_PX)
    e, fe = value_check(img, order, val, fp, cr, precision)
    assert e <= VALUE_RTOL and fe <= 1e-6
    assert (fp == 0).any() and (fp > 0).mean() > 0.8  # partial coverage exercised


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_bbox_offset_pitch_and_degenerate_shapes(precision):
    src, tgt, img = _small_sip(order="bilinear", w=300, h=200)
    big = np.zeros((200, 320), np.float32)
    big[:, :300] = img
    img_d = to_dev(big)[:, :300]  # source pitch 320 > NAXIS1
    T = torch()
    for bbox in [(13, 7, 150, 77), (0, 0, 1, 1), (5, 9, 1, 120), (2, 3, 200, 1), (250, 150, 90, 70)]:
        x0, y0, w, h = bbox
        out = T.full((h, w + 5), -7.0, device="cuda")[:, :w]
        fp = T.full((h, w + 5), -7.0, device="cuda")[:, :w]
        val, fpv = dfr().reproject(img_d, src, tgt, bbox=bbox, order="bilinear",
                                   precision=precision, out=out, fp_out=fp)
        v2, f2, cr = gpu(src, tgt, to_dev(img), "bilinear", precision, bbox)
        T.cuda.synchronize()
        assert np.array_equal(val.cpu().numpy(), v2) and np.array_equal(fpv.cpu().numpy(), f2)
        e, fe = value_check(img, "bilinear", v2, f2, cr, precision)
        assert e <= VALUE_RTOL and fe <= 1e-6


@pytest.mark.parametrize("order", ["nearest", "bilinear", "bicubic"])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_identity_is_bit_exact(order, precision):
    c = synth.config0()
    src, img = c["src"][0], c["images"][0]
    val, fp, _ = gpu(src, src, to_dev(img), order, precision, (0, 0, 512, 512))
    assert np.array_equal(val, img) and np.all(fp == 1.0)


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_integer_shift_nearest_bit_exact(precision):
    c = synth.config0()
    src, img = c["src"][0], c["images"][0]
    tgt = synth.copy_wcs(src)
    tgt["crpix"] = (src["crpix"][0] + 5.0, src["crpix"][1] - 3.0)
    val, fp, _ = gpu(src, tgt, to_dev(img), "nearest", precision, (0, 0, 512, 512))
    exp = np.zeros_like(img)
    exp[:509, 5:] = img[3:, :507]
    assert np.array_equal(val, exp)
    assert set(np.unique(fp)) <= {0.0, 1.0}


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_half_pixel_shift_nearest_ties_round_up(precision):
    """A CRPIX shift of (-0.5, +1.5) px with the same sky projection: every source position is
    exactly halfway between two pixel centres, and nearest takes the upper one (floor(x + 0.5)),
    as the oracle does on the same positions."""
    c = synth.config0()
    src, img = c["src"][0], c["images"][0]
    tgt = synth.copy_wcs(src)
    tgt["crpix"] = (src["crpix"][0] - 0.5, src["crpix"][1] + 1.5)
    val, fp, cr = gpu(src, tgt, to_dev(img), "nearest", precision, (0, 0, 512, 512))
    Y, X = np.mgrid[0:512, 0:512].astype(np.float64)
    assert np.array_equal(cr[..., 0], X + 0.5) and np.array_equal(cr[..., 1], Y - 1.5)
    exp = np.zeros_like(img)
    exp[1:, :511] = img[:511, 1:]
    assert np.array_equal(val, exp)
    ov, ofp = OI.interpolate(img, X + 0.5, Y - 1.5, OI.NEAREST)
    assert np.array_equal(val, ov.astype(np.float32)) and np.array_equal(fp, ofp.astype(np.float32))


def test_linear_ramp_bilinear_and_quadratic_bicubic():
    c = synth.config0()
    src, tgt = c["src"][0], c["tgt"]
    Y, X = np.mgrid[0:512, 0:512].astype(np.float64)
    ramp = (0.01 * X - 0.02 * Y + 3.0).astype(np.float32)
    quad = (1e-4 * X * X - 2e-4 * X * Y + 5e-5 * Y * Y + 0.01 * X + 1.0).astype(np.float32)
    for img, order in ((ramp, "bilinear"), (quad, "bicubic")):
        for precision in ("fp64", "split"):
            val, fp, cr = gpu(src, tgt, to_dev(img), order, precision, (0, 0, 512, 512))
            x, y = cr[..., 0], cr[..., 1]
            inner = (x > 2) & (x < 509) & (y > 2) & (y < 509)
            if order == "bilinear":
                exact = 0.01 * x - 0.02 * y + 3.0
            else:
                exact = 1e-4 * x * x - 2e-4 * x * y + 5e-5 * y * y + 0.01 * x + 1.0
            # float32 source rounding bounds the reproduction, ~1e-6 of the image range
            assert np.abs(val - exact)[inner].max() <= 1e-6 * np.abs(img).max() + 4e-7 * 8


def _far_pair(target_sip):
    """Different tangent points (a projective map with a live denominator), rotation and scale
    change, optionally a SIP target grid."""
    rng = synth.rng_for(99)
    src = synth.add_sip(synth.tan_wcs(500, 400, crval=(150.0, 30.0)), 3, 1e-6, rng)
    src, _ = OW.with_inverse_sip(src, 4)
    tgt = synth.tan_wcs(520, 380, crval=(150.05, 30.04), rho_deg=-2.0, scale_arcsec=2.7)
    if target_sip:
        tgt = synth.add_sip(tgt, 2, 1e-6, rng)
    return src, tgt, synth.sky_image(500, 400, 40, rng)


@pytest.mark.parametrize("case", ["small_sip", "far_tangent", "far_tangent_target_sip"])
def test_tma_and_direct_gather_agree_bitwise(case):
    """The TMA-staged rows (interior fast path included) and the direct global-memory gather run
    the same arithmetic: values, footprints and emitted coordinates are equal bit for bit."""
    if case == "small_sip":
        src, tgt, img = _small_sip()
    else:
        src, tgt, img = _far_pair(case.endswith("target_sip"))
    bbox = (0, 0, tgt["naxis"][0], tgt["naxis"][1])
    for order in ("nearest", "bilinear", "bicubic", "lanczos3", "bspline3"):
        a = gpu(src, tgt, to_dev(img), order, "split", bbox, tma=True)
        b = gpu(src, tgt, to_dev(img), order, "split", bbox, tma=False)
        for u, v in zip(a, b):
            assert np.array_equal(u, v, equal_nan=True)


def test_split_vs_fp64_coordinates():
    src, tgt, img = _small_sip()
    bbox = (0, 0, tgt["naxis"][0], tgt["naxis"][1])
    _, _, c64 = gpu(src, tgt, to_dev(img), "bicubic", "fp64", bbox)
    _, _, c32 = gpu(src, tgt, to_dev(img), "bicubic", "split", bbox)
    d = np.hypot(c64[..., 0] - c32[..., 0], c64[..., 1] - c32[..., 1])
    assert np.nanmax(d) < SPLIT_PX


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_exact_inverse_newton(precision):
    src, tgt, img = _small_sip(order="bilinear", w=400, h=300)
    bbox = (0, 0, tgt["naxis"][0], tgt["naxis"][1])
    val, fp, cr = gpu(src, tgt, to_dev(img), "bilinear", precision, bbox, exact=True)
    dmax, _ = coord_check(src, tgt, cr, bbox, inverse="newton")
    assert dmax < (FP64_PX if precision == "fp64" else SPLIT_PX)
    e, fe = value_check(img, "bilinear", val, fp, cr, precision)
    assert e <= VALUE_RTOL and fe <= 1e-6


def test_far_tangent_points_and_target_sip():
    """Different CRVAL (projective map), a SIP target grid, and a target partly off the source."""
    rng = synth.rng_for(99)
    src = synth.add_sip(synth.tan_wcs(500, 400, crval=(150.0, 30.0)), 3, 1e-6, rng)
    src, _ = OW.with_inverse_sip(src, 4)
    tgt = synth.add_sip(synth.tan_wcs(520, 380, crval=(150.05, 30.04), rho_deg=-2.0,
                                      scale_arcsec=2.7), 2, 1e-6, rng)
    img = synth.sky_image(500, 400, 40, rng)
    bbox = (0, 0, 520, 380)
    for precision in ("fp64", "split"):
        val, fp, cr = gpu(src, tgt, to_dev(img), "bicubic", precision, bbox)
        dmax, _ = coord_check(src, tgt, cr, bbox)
        assert dmax < (FP64_PX if precision == "fp64" else SPLIT_PX)
        e, fe = value_check(img, "bicubic", val, fp, cr, precision)
        assert e <= VALUE_RTOL and fe <= 1e-6


def test_source_far_hemisphere_is_uncovered():
    """A wide target grid whose tangent point is 80 deg from the source's: pixels whose sky
    position lies on the far hemisphere of the source projection are uncovered. The FP64 path
    decides per pixel exactly like the oracle; the split path (one wide-precision anchor per cell) never
    covers such a pixel."""
    src = synth.tan_wcs(64, 64, crval=(0.0, 0.0))
    tgt = synth.tan_wcs(64, 64, crval=(80.0, 0.0), scale_arcsec=3600.0 * 3)  # 3 deg/px
    img = np.ones((64, 64), np.float32)
    X, Y = np.meshgrid(np.arange(64.0), np.arange(64.0))
    _, _, ok = OR.coords(src, tgt, X, Y)
    assert (~ok).any() and ok.any()
    val, fp, cr = gpu(src, tgt, to_dev(img), "bilinear", "fp64", (0, 0, 64, 64))
    assert np.array_equal(np.isfinite(cr[..., 0]), ok)
    val, fp, cr = gpu(src, tgt, to_dev(img), "bilinear", "split", (0, 0, 64, 64))
    assert np.all(fp[~ok] == 0) and np.all(val[~ok] == 0)
    far = synth.tan_wcs(64, 64, crval=(120.0, 0.0))
    with pytest.raises(dfr().DfrError):
        dfr().reproject(to_dev(img), src, far, order="bilinear", precision="split")
    dfr().reproject(to_dev(img), src, far, order="bilinear", precision="fp64")


def test_config1_full_size_sampled():
    """The bench workload (4096^2 TAN-SIP 3, bicubic, split) in its bench launch form, checked
    on 20000 sampled pixels: coordinates vs the oracle and values at the GPU coordinates."""
    c = synth.config1()
    src = with_inverse(c)
    tgt, img = c["tgt"], c["images"][0]
    img_d = to_dev(img)
    bbox = (0, 0, 4096, 4096)
    val, fp, cr = gpu(src, tgt, img_d, "bicubic", "split", bbox)
    rng = synth.rng_for(2024)
    dmax, drms = coord_check(src, tgt, cr, bbox, sample=20000, rng=rng)
    assert dmax < SPLIT_PX
    idx = rng.integers(0, 4096 * 4096, 20000)
    sel = (idx // 4096, idx % 4096)
    e, fe = value_check(img, "bicubic", val[sel][None], fp[sel][None], cr[sel][None], "split")
    assert e <= VALUE_RTOL and fe <= 1e-6
    # the bench call (no coordinate output) writes the same values
    v2, f2 = dfr().reproject(img_d, src, tgt, bbox=bbox, order="bicubic", precision="split")
    assert np.array_equal(v2.cpu().numpy(), val) and np.array_equal(f2.cpu().numpy(), fp)


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_legacy_header_keywords_lonpole_crota2(precision):
    """Headers with CDELT + CROTA2 (no CD) and LONPOLE != 180 on both sides: parsed by the
    library (LONPOLE folded into CD), reprojected on the GPU, against the oracle on its own
    parse of the same text (LONPOLE kept, rotation on the sphere)."""
    src, tgt, img = _small_sip(w=400, h=300, seed=12)
    s = 2.5 / 3600

    def legacy(w, rho, scale, lonpole):
        lines = [ln for ln in synth.header_cards(w, "\n").split("\n") if not ln.startswith("CD")]
        return "\n".join(lines[:-1] + ["CDELT1  = %.17g" % (-s * scale),
                                       "CDELT2  = %.17g" % (s * scale),
                                       "CROTA2  = %.17g" % rho, "LONPOLE = %.17g" % lonpole,
                                       "END"])

    ts, tt = legacy(src, 0.0, 1.0, 215.0), legacy(tgt, 1.2, 1.01, 150.0)
    c_src, c_tgt = dfr().wcs_from_header(ts), dfr().wcs_from_header(tt)
    o_src, o_tgt = OW.parse_header(ts), OW.parse_header(tt)
    bbox = (0, 0, tgt["naxis"][0], tgt["naxis"][1])
    val, fp, cr = gpu(c_src, c_tgt, to_dev(img), "bicubic", precision, bbox)
    dmax, _ = coord_check(o_src, o_tgt, cr, bbox)
    assert dmax < (FP64_PX if precision == "fp64" else SPLIT_PX)
    e, fe = value_check(img, "bicubic", val, fp, cr, precision)
    assert e <= VALUE_RTOL and fe <= 1e-6
    assert (fp > 0).mean() > 0.5


@pytest.mark.parametrize("order", ["nearest", "bilinear", "bicubic"])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_nan_masked_source(order, precision):
    """DFR_NAN_MASK: NaN source pixels (scattered, plus a 9x6 block) take no weight; the oracle's
    masked interpolation at the GPU's coordinates matches value and footprint (coverage too).
    Without the flag the NaN reach the output; the batch path equals the single call."""
    src, tgt, img = _small_sip(w=400, h=300, seed=13)
    rng = synth.rng_for(14)
    holed = img.copy()
    holed[rng.integers(0, 300, 600), rng.integers(0, 400, 600)] = np.nan
    holed[120:126, 200:209] = np.nan
    d = to_dev(holed)
    bbox = (0, 0, tgt["naxis"][0], tgt["naxis"][1])
    val, fp, cr = gpu(src, tgt, d, order, precision, bbox, nan_mask=True)
    assert np.isfinite(val).all() and np.isfinite(fp).all()
    e, fe = value_check(holed, order, val, fp, cr, precision, nan_mask=True)
    assert e <= VALUE_RTOL and fe <= 1e-6
    v1, f1, _ = gpu(src, tgt, to_dev(img), order, precision, bbox)
    if order == "nearest":
        assert ((f1 > 0) & (fp == 0)).sum() > 100  # pixels on holes become uncovered
    else:
        assert ((fp > 0) & (fp < f1)).sum() > 100  # pixels next to holes keep a partial weight
    v0, _ = dfr().reproject(d, src, tgt, bbox=bbox, order=order, precision=precision)
    assert torch().isnan(v0).any()
    vb, fb = dfr().reproject_batch([d], [src], tgt, [bbox], order=order, precision=precision,
                                   nan_mask=True)
    assert np.array_equal(vb[0].cpu().numpy(), val) and np.array_equal(fb[0].cpu().numpy(), fp)



def test_lanczos3_identity_and_constant():
    """Lanczos-3 on the GPU: the identity map returns the image bit for bit (weights 1 at the
    node), and a constant image is reproduced to FP32 rounding on every covered pixel."""
    src = synth.tan_wcs(300, 200)
    img = synth.sky_image(300, 200, 20, synth.rng_for(30))
    for precision in ("fp64", "split"):
        v, f = dfr().reproject(to_dev(img), src, src, order="lanczos3", precision=precision)
        assert np.array_equal(v.cpu().numpy(), img) and bool((f == 1).all())
    tgt = synth.tan_wcs(320, 210, rho_deg=1.7, crpix=(152.3, 98.9))
    const = np.full((200, 300), 2.5, np.float32)
    for precision in ("fp64", "split"):
        v, f = dfr().reproject(to_dev(const), src, tgt, order="lanczos3", precision=precision)
        v, f = v.cpu().numpy(), f.cpu().numpy()
        assert (f > 0).mean() > 0.5
        assert np.abs(v[f > 0] - 2.5).max() < 1e-5



@pytest.mark.parametrize("shape", [(300, 200), (37, 53), (1, 17), (17, 1), (2, 9)])
def test_bspline_prefilter_matches_oracle(shape):
    """GPU prefilter (FP32 recursion, rows then columns) against the oracle's FP64 coefficients,
    element by element (1e-5 of the largest coefficient), out of place and in place."""
    h, w = shape
    img = synth.rng_for(40).standard_normal((h, w)).astype(np.float32) * 10
    ref = OI.bspline3_prefilter(img.astype(np.float64))
    d = to_dev(img)
    c = dfr().bspline_prefilter(d).cpu().numpy()
    tol = 1e-5 * np.abs(ref).max()
    assert np.abs(c - ref).max() <= tol
    dfr().bspline_prefilter(d, out=d)
    assert np.array_equal(d.cpu().numpy(), c)


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_bspline3_reprojection(precision):
    """B-spline reprojection against the oracle's evaluation on its own FP64 coefficients at the
    GPU's coordinates (values 1e-5; footprint 1 exactly where covered); the identity map returns
    the image to FP32 rounding of the coefficients."""
    src, tgt, img = _small_sip(w=400, h=300, seed=41)
    bbox = (0, 0, tgt["naxis"][0], tgt["naxis"][1])
    val, fp, cr = gpu(src, tgt, to_dev(img), "bspline3", precision, bbox)
    coef = OI.bspline3_prefilter(img.astype(np.float64))
    e, fe = value_check(coef, "bspline3", val, fp, cr, precision)
    assert e <= VALUE_RTOL and fe == 0.0
    assert set(np.unique(fp)) <= {0.0, 1.0} and (fp == 1).mean() > 0.5
    plain = synth.tan_wcs(300, 200)
    im2 = synth.sky_image(300, 200, 20, synth.rng_for(42))
    v, f = dfr().reproject(to_dev(im2), plain, plain, order="bspline3", precision=precision)
    assert np.abs(v.cpu().numpy() - im2).max() <= 1e-5 * max(np.abs(im2).max(), 1.0)
    assert bool((f == 1).all())


def _host_case(case):
    if case == "rot90":
        src, _, img = _small_sip(w=500, h=300, seed=51)
        tgt = synth.tan_wcs(320, 520, rho_deg=90.0, crpix=(160.5, 250.5))
        return src, tgt, img, (0, 0, 320, 520)
    src, tgt, img = _small_sip(seed=52)
    if case == "odd_bbox":
        return src, tgt, img, (13, 7, 611, 397)
    return src, tgt, img, (0, 0, tgt["naxis"][0], tgt["naxis"][1])


@pytest.mark.parametrize("case", ["full", "rot90", "odd_bbox"])
def test_host_pipeline_equals_device_call(case):
    """dfr_reproject_host (bands copied in, computed and copied out on overlapping streams)
    gives the device call's bits: split path (banded, including a 90 deg rotation where every
    band reads every source row), FP64 path and the B-spline order (one band), from page-locked
    tensors and from pageable numpy arrays."""
    T = torch()
    src, tgt, img, bbox = _host_case(case)
    x0, y0, w, h = bbox
    d = to_dev(img)
    for order, precision in (("bicubic", "split"), ("lanczos3", "split"), ("bilinear", "fp64"),
                             ("bspline3", "split")):
        v, f = dfr().reproject(d, src, tgt, bbox=bbox, order=order, precision=precision)
        v, f = v.cpu().numpy(), f.cpu().numpy()
        hv, hf = dfr().reproject_host(img, src, tgt, bbox=bbox, order=order, precision=precision)
        assert np.array_equal(hv, v) and np.array_equal(hf, f), (order, precision)
        pin = T.from_numpy(img).pin_memory()
        po = T.empty((h, w)).pin_memory()
        pf = T.empty((h, w)).pin_memory()
        dfr().reproject_host(pin, src, tgt, bbox=bbox, order=order, precision=precision, out=po,
                             fp_out=pf)
        assert np.array_equal(po.numpy(), v) and np.array_equal(pf.numpy(), f), (order, precision)
    dfr().device_status()


def test_calculate_reprojection_from_headers():
    """The paper-style host call on FITS header text (the 50x50 demo pair of Sec. 4.1, as read
    here): host numpy in, host numpy out, against the oracle end to end (FP64 path)."""
    c = synth.demo50()
    src, tgt, img = c["src"][0], c["tgt"], c["images"][0]
    v, f = dfr().calculate_reprojection(img, synth.header_cards(src), synth.header_cards(tgt),
                                        order="bilinear", precision="fp64")
    ov, of, _, _ = OR.reproject(src, tgt, img, "bilinear")
    assert v.shape == (50, 50)
    assert np.abs(v - ov).max() <= VALUE_RTOL * max(np.abs(ov).max(), 1.0)
    assert np.abs(f - of).max() <= 1e-6


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (2, 2), (3, 5), (301, 203)])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_tiny_and_odd_sources(shape, precision):
    """Degenerate and odd-sized sources (w x h): single pixels, single rows and columns, and an
    odd width whose rows are not 16-byte multiples (no TMA: the global-memory gather), for every
    order, against the oracle at the GPU's coordinates (coverage decisions must agree)."""
    w, h = shape
    rng = synth.rng_for(60 + w * 7 + h)
    src = synth.tan_wcs(w, h, crval=(150.0, 2.0))
    img = synth.sky_image(w, h, 1, rng) if w * h > 4 else rng.standard_normal((h, w))
    img = img.astype(np.float32)
    tgt = synth.tan_wcs(w + 6, h + 6, rho_deg=0.9, scale_arcsec=2.3,
                        crpix=((w + 7) / 2.0 + 0.37, (h + 7) / 2.0 - 0.21))
    bbox = (0, 0, w + 6, h + 6)
    for order in ("nearest", "bilinear", "bicubic", "lanczos3", "bspline3"):
        val, fp, cr = gpu(src, tgt, to_dev(img), order, precision, bbox)
        ref_img = OI.bspline3_prefilter(img.astype(np.float64)) if order == "bspline3" else img
        e, fe = value_check(ref_img, order, val, fp, cr, precision)
        assert e <= VALUE_RTOL and fe <= 1e-6, (order, e, fe)
        assert (fp > 0).any(), order


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_large_frame_sampled(precision):
    """A 20000x16000 source (SIP-3) onto a 24000x20000 bounding box (480 Mpix, about 5 GB on the
    device: 64-bit output offsets, 469k anchor cells / 1.9M FP64 tiles in one launch), checked
    on a seeded sample of 4000 pixels: coordinates against the FP64 oracle, values at the GPU's
    coordinates, coverage decisions on the same numbers."""
    T = torch()
    rng = synth.rng_for(70)
    W, H = 20000, 16000
    src = synth.add_sip(synth.tan_wcs(W, H, scale_arcsec=1.0), 3, 1e-6, rng)
    src, _ = OW.with_inverse_sip(src, 4)
    tgt = synth.tan_wcs(24000, 20000, scale_arcsec=0.95, rho_deg=0.6,
                        crpix=(12000.5 + 310.0, 10000.5 - 170.0))
    img = (rng.standard_normal((H, W)) * 0.1).astype(np.float32)
    img[:: 37, :: 41] += 50.0  # sparse bright points
    bbox = (0, 0, 24000, 20000)
    d = to_dev(img)
    val, fp, cr = dfr().reproject(d, src, tgt, bbox=bbox, order="bicubic", precision=precision,
                                  coords=True)
    T.cuda.synchronize()
    dfr().device_status()
    px = T.from_numpy(rng.integers(0, 24000, 4000)).cuda()
    py = T.from_numpy(rng.integers(0, 20000, 4000)).cuda()
    v = val[py, px].cpu().numpy()
    f = fp[py, px].cpu().numpy()
    c = cr[py, px].cpu().numpy()
    del val, fp, cr
    ox, oy, ok = OR.coords(src, tgt, px.cpu().numpy(), py.cpu().numpy())
    dd = np.hypot(c[:, 0] - ox, c[:, 1] - oy)[ok]
    assert dd.max() < (FP64_PX if precision == "fp64" else SPLIT_PX)
    e, fe = value_check(img, "bicubic", v[None], f[None], c[None], precision)
    assert e <= VALUE_RTOL and fe <= 1e-6
    assert (f > 0).mean() > 0.5 and (f == 0).any()
