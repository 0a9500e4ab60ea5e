"""C-ABI checks that need no GPU: the library loads, exports every symbol the header declares,
and its host-side calls (header parsing, inverse-SIP fit, bounding boxes, argument errors)
agree with the oracle or fail with the documented codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import reproject as OR
from oracle import wcs as OW

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dfr():
    import paper_2505_03932_gb300 as d
    if not os.path.exists(d._LIBPATH):
        from paper_2505_03932_gb300 import build
        build.build()
    d.lib()
    return d


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\s*\*)\s+(dfr_\w+)\s*\(", text, re.M))
    return names


def test_library_exports_every_declared_symbol(dfr):
    syms = _declared_symbols()
    assert {"dfr_wcs_from_header", "dfr_reproject", "dfr_reproject_batch",
            "dfr_reproject_backward"} <= syms
    L = dfr.lib()
    for s in sorted(syms):
        assert hasattr(L, s), s
    assert L.dfr_abi_version() == 1


@pytest.mark.parametrize("sep", ["", "\n"])
def test_header_parse_matches_oracle_bitwise(dfr, sep):
    c = synth.config1()
    src, _ = OW.with_inverse_sip(c["src"][0], 4)
    text = synth.header_cards(src, sep)
    w = dfr.wcs_from_header(text)
    o = OW.parse_header(text)
    assert tuple(w["naxis"]) == tuple(o["naxis"])
    assert w["crpix"] == o["crpix"] and w["crval"] == o["crval"] and w["cd"] == o["cd"]
    for k in ("a", "b", "ap", "bp"):
        assert w[k + "_order"] == o[k + "_order"]
        assert np.array_equal(w[k], o[k])


def test_header_pc_cdelt(dfr):
    lines = [ln for ln in synth.header_cards(synth.tan_wcs(100, 80), "\n").split("\n")
             if not ln.startswith("CD")]
    pc = lines[:-1] + ["CDELT1  = -0.001", "CDELT2  = 0.002", "PC1_1   = 0.5",
                       "PC1_2   = 0.25", "PC2_1   = -0.25", "PC2_2   = 0.5", "END"]
    text = "\n".join(pc)
    assert dfr.wcs_from_header(text)["cd"] == OW.parse_header(text)["cd"]


@pytest.mark.parametrize("edit,code", [
    (lambda t: t.replace("RA---TAN", "RA---SIN"), -3),
    (lambda t: t.replace("END", "LONPOLE = 'abc'\nEND"), -2),
    (lambda t: "\n".join(l for l in t.split("\n") if not l.startswith("CRPIX1")), -2),
    (lambda t: "\n".join(l for l in t.split("\n") if not l.startswith("CD")), -2),
    (lambda t: re.sub(r"CD2_2   =\s*\S+", "CD2_2   = 0.0", re.sub(r"CD1_1   =\s*\S+",
                                                                 "CD1_1   = 0.0", t)), -4),
    (lambda t: t.replace("CRVAL1  = ", "CRVAL1  = 'x'  /"), -2),
])
def test_header_errors(dfr, edit, code):
    w = synth.tan_wcs(100, 80, rho_deg=0.0)
    text = edit(synth.header_cards(w, "\n"))
    with pytest.raises(dfr.DfrError) as ei:
        dfr.wcs_from_header(text)
    assert ei.value.code == code
    assert dfr.lib().dfr_last_error().decode() != ""


def test_inverse_sip_fit_matches_oracle(dfr):
    c = synth.config1()
    src = c["src"][0]
    lw, lmax, lrms = dfr.fit_inverse_sip(src, 4)
    ow, st = OW.with_inverse_sip(src, 4)
    # both fits minimise the same least-squares problem: coefficients agree to round-off
    # relative to the term scale, and the residuals agree
    for k in ("ap", "bp"):
        R = 2048.0
        for n in range(1, 5):
            for p in range(n, -1, -1):
                q = n - p
                assert abs(lw[k][p, q] - ow[k][p, q]) * R ** (p + q) < 1e-9
    assert abs(lmax - st["max_px"]) < 1e-9 and abs(lrms - st["rms_px"]) < 1e-9


def test_target_bbox_contains_oracle_coverage(dfr):
    c = synth.config0()
    src = synth.add_sip(c["src"][0], 3, 2e-5, synth.rng_for(3))
    src, _ = OW.with_inverse_sip(src, 4)
    tgt = synth.copy_wcs(c["tgt"])
    tgt["naxis"] = (700, 640)
    tgt["crpix"] = (tgt["crpix"][0] + 60, tgt["crpix"][1] + 40)
    x0, y0, w, h = dfr.target_bbox(src, tgt)
    _, fp, _, _ = OR.reproject(src, tgt, c["images"][0], "bilinear")
    ys, xs = np.nonzero(fp)
    assert xs.min() >= x0 and xs.max() < x0 + w and ys.min() >= y0 and ys.max() < y0 + h
    assert w * h < 1.1 * (np.ptp(xs) + 5) * (np.ptp(ys) + 5)


def test_target_bbox_disjoint_frame_is_empty(dfr):
    src = synth.tan_wcs(100, 100)
    tgt = synth.tan_wcs(100, 100, crval=(151.0, 2.0))
    assert dfr.target_bbox(src, tgt) == (0, 0, 0, 0)


def test_argument_errors_before_any_launch(dfr):
    L = dfr.lib()
    s = dfr.to_c(synth.tan_wcs(64, 64))
    t = dfr.to_c(synth.tan_wcs(64, 64))
    dummy = ctypes.c_void_p(16)
    call = lambda **kw: L.dfr_reproject(
        ctypes.byref(kw.get("s", s)), ctypes.byref(t), kw.get("img", dummy), kw.get("pitch", 64),
        kw.get("out", dummy), None, kw.get("opitch", 64), 0, 0, kw.get("w", 64), kw.get("h", 64),
        kw.get("order", 1), kw.get("flags", 1), None, None)
    assert call(order=5) == -1
    assert call(order=4, flags=1 | 8) == -1  # B-spline coefficients with the NaN mask
    assert call(flags=64) == -1
    assert call(pitch=10) == -1
    assert call(opitch=10) == -1
    assert call(img=None) == -1
    assert call(w=-1) == -1
    bad = dfr.to_c(synth.tan_wcs(64, 64))
    bad.cd[0][0] = bad.cd[1][1] = 0.0
    assert call(s=bad) == -4
    sip = synth.add_sip(synth.tan_wcs(64, 64), 3, 1e-6, synth.rng_for(1))
    assert call(s=dfr.to_c(sip)) == -5  # A/B without AP/BP and no exact inverse
    nan = dfr.to_c(synth.tan_wcs(64, 64))
    nan.crval[0] = float("nan")
    assert call(s=nan) == -1
    # empty output: nothing to do, no launch
    assert call(w=0, h=0, img=None, out=None) == 0
    assert L.dfr_reproject_batch(None, 0, ctypes.byref(t), 1, 1, None) == 0
    assert L.dfr_reproject_batch(None, 3, ctypes.byref(t), 1, 1, None) == -1


def test_coadd_argument_errors_before_any_launch(dfr):
    L = dfr.lib()
    t = dfr.to_c(synth.tan_wcs(64, 48))
    dummy = ctypes.c_void_p(16)
    frames = (dfr.DfrFrame * 2)()
    for fr in frames:
        fr.wcs = dfr.to_c(synth.tan_wcs(40, 30))
        fr.img = 16
        fr.pitch = 40
        fr.x0, fr.y0, fr.w, fr.h = 0, 0, 20, 20
    co = lambda n=2, vf=dummy, f=dummy, pitch=64, fr=frames: L.dfr_coadd(
        fr, n, ctypes.byref(t), 1, 1, vf, f, pitch, None)
    assert co(n=0) == 0
    assert co(n=-1) == -1
    assert co(vf=None) == -1
    assert co(f=None) == -1
    assert co(pitch=63) == -1
    frames[1].x0 = 50  # 50 + 20 > NAXIS1 = 64
    assert co() == -1
    assert "outside the target grid" in L.dfr_last_error().decode()
    frames[1].x0, frames[1].y0 = 0, -1
    assert co() == -1
    nz = lambda **kw: L.dfr_coadd_normalize(
        kw.get("vf", dummy), kw.get("f", dummy), kw.get("pitch", 64), kw.get("w", 64),
        kw.get("h", 48), kw.get("mw", 0.0), kw.get("mean", dummy), kw.get("mp", 64), None)
    assert nz(w=0) == 0
    assert nz(w=-1) == -1
    assert nz(mean=None) == -1
    assert nz(pitch=10) == -1
    assert nz(mp=10) == -1
    assert nz(mw=-1.0) == -1
    assert nz(mw=float("nan")) == -1


def _cards_without_cd(w):
    return [ln for ln in synth.header_cards(w, "\n").split("\n") if not ln.startswith("CD")]


def test_header_crota2_matches_the_cdelt_rotation_convention(dfr):
    """CDELT + CROTA2 (no CD, no PC) -> CD of the CROTA2 convention, which is how the synthetic
    WCS records build their CD from (scale, rotation)."""
    s = 2.5 / 3600
    for rho in (0.0, 1.2, -37.5, 90.0):
        w = synth.tan_wcs(100, 80, rho_deg=rho)
        text = "\n".join(_cards_without_cd(w)[:-1] + ["CDELT1  = %.17g" % -s,
                                                      "CDELT2  = %.17g" % s,
                                                      "CROTA2  = %.17g" % rho, "END"])
        for got in (dfr.wcs_from_header(text)["cd"], OW.parse_header(text)["cd"]):
            assert np.allclose(got, w["cd"], rtol=0, atol=1e-18)
    # PC wins over CROTA2
    text = "\n".join(_cards_without_cd(synth.tan_wcs(100, 80))[:-1] + [
        "CDELT1  = -0.001", "CDELT2  = 0.002", "CROTA2  = 30.0", "PC1_1   = 1.0", "END"])
    assert dfr.wcs_from_header(text)["cd"] == [[-0.001, 0.0], [0.0, 0.002]]


def test_header_lonpole_folded_into_cd_maps_like_the_oracle(dfr):
    """LONPOLE != 180: the library folds the native-longitude rotation into CD; the oracle keeps
    LONPOLE and rotates on the sphere. Both records give the same sky positions (1e-12 deg) and
    the same source pixels."""
    rng = synth.rng_for(17)
    base = synth.add_sip(synth.tan_wcs(300, 200, crval=(210.0, 47.0), rho_deg=3.0), 3, 1e-6, rng)
    text0 = synth.header_cards(base, "\n")
    X = rng.uniform(-50, 350, 400)
    Y = rng.uniform(-50, 250, 400)
    for lon in (170.0, 0.0, 245.5, -90.0):
        text = text0.replace("END", "LONPOLE = %.17g\nEND" % lon)
        c = dfr.wcs_from_header(text)
        o = OW.parse_header(text)
        assert o["lonpole"] == lon and "lonpole" not in c
        ra_c, dec_c = OW.pix2world(c, X, Y)
        ra_o, dec_o = OW.pix2world(o, X, Y)
        dra = (ra_c - ra_o + 180.0) % 360.0 - 180.0
        assert np.abs(dra * np.cos(np.radians(dec_o))).max() < 1e-12
        assert np.abs(dec_c - dec_o).max() < 1e-12
        u_c, v_c, ok_c = OW.world_to_intermediate(c, ra_o, dec_o)
        u_o, v_o, ok_o = OW.world_to_intermediate(o, ra_o, dec_o)
        assert np.array_equal(ok_c, ok_o)
        assert np.abs(u_c - u_o).max() < 1e-9 and np.abs(v_c - v_o).max() < 1e-9


def test_adjoint_refuses_the_nan_mask_flag(dfr):
    L = dfr.lib()
    rc = L.dfr_reproject_backward(None, None, None, 0, None, 0, 0, 0, 0, 0, 1,
                                  dfr.SPLIT | dfr.NAN_MASK, None, 0, None, None)
    assert rc == -1 and "NAN_MASK" in L.dfr_last_error().decode()


def test_adjoint_refuses_bspline3(dfr):
    L = dfr.lib()
    s = dfr.to_c(synth.tan_wcs(64, 64))
    rc = L.dfr_reproject_backward(ctypes.byref(s), ctypes.byref(s), ctypes.c_void_p(16), 64,
                                  ctypes.c_void_p(16), 64, 0, 0, 64, 64, dfr.BSPLINE3, dfr.SPLIT,
                                  None, 0, None, None)
    assert rc == -1 and "BSPLINE3" in L.dfr_last_error().decode()


def test_bspline_prefilter_argument_errors(dfr):
    L = dfr.lib()
    d = ctypes.c_void_p(16)
    e = ctypes.c_void_p(32)
    assert L.dfr_bspline_prefilter(d, 64, 0, 10, d, 64, None) == 0
    assert L.dfr_bspline_prefilter(d, 64, -1, 10, d, 64, None) == -1
    assert L.dfr_bspline_prefilter(None, 64, 8, 10, d, 64, None) == -1
    assert L.dfr_bspline_prefilter(d, 4, 8, 10, e, 64, None) == -1
    assert L.dfr_bspline_prefilter(d, 64, 8, 10, d, 72, None) == -1  # in place, other stride


def test_host_entry_argument_errors(dfr):
    L = dfr.lib()
    s = dfr.to_c(synth.tan_wcs(64, 48))
    d = ctypes.c_void_p(16)
    call = lambda **kw: L.dfr_reproject_host(
        ctypes.byref(s), ctypes.byref(s), kw.get("img", d), kw.get("pitch", 64), kw.get("out", d),
        None, kw.get("opitch", 64), 0, 0, kw.get("w", 64), kw.get("h", 48), kw.get("order", 1), 1)
    assert call(w=0) == 0
    assert call(w=-1) == -1
    assert call(img=None) == -1
    assert call(out=None) == -1
    assert call(pitch=63) == -1
    assert call(opitch=10) == -1
