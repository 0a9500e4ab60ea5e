"""Pins for the oracle's coordinate transforms (Sec. 3.2.1, Sec. 3.2.2) — CPU only.

Each check compares the oracle with something other than itself: a textbook closed form of
the gnomonic projection ("standard coordinates"), an invariant (CRPIX -> CRVAL, round trips),
a special case with an exact affine or projective answer computed by independent vector
algebra, or a hand-worked case of the SIP convention.
"""
import math

import numpy as np
import pytest

import synth
from oracle import wcs as W

DEC0S = [0.0, 2.0, 60.0, 89.9]


def _wcs(dec0=2.0, ra0=150.0, rho=0.7, scale=2.5, crpix=(101.3, 57.8), n=(512, 384)):
    return synth.tan_wcs(n[0], n[1], crval=(ra0, dec0), scale_arcsec=scale, rho_deg=rho,
                         crpix=crpix)


@pytest.mark.parametrize("dec0", DEC0S)
def test_crpix_maps_to_crval(dec0):
    w = synth.add_sip(_wcs(dec0=dec0), 3, 1e-6, synth.rng_for(5))
    ra, dec = W.pix2world(w, np.array([w["crpix"][0] - 1.0]), np.array([w["crpix"][1] - 1.0]))
    assert abs(ra[0] - w["crval"][0]) < 1e-12
    assert abs(dec[0] - w["crval"][1]) < 1e-12


def _std_to_sky(xi, eta, ra0, dec0):
    """Textbook inverse gnomonic projection (standard coordinates xi, eta in radians)."""
    a0, d0 = math.radians(ra0), math.radians(dec0)
    den = math.cos(d0) - eta * math.sin(d0)
    dra = math.atan2(xi, den)
    dec = math.atan((eta * math.cos(d0) + math.sin(d0)) * math.cos(dra) / den)
    return a0 + dra, dec


def _sky_to_std(ra, dec, ra0, dec0):
    """Textbook gnomonic projection: xi = cos d sin da / D, eta = (...)/D."""
    a, d = math.radians(ra), math.radians(dec)
    a0, d0 = math.radians(ra0), math.radians(dec0)
    D = math.sin(d) * math.sin(d0) + math.cos(d) * math.cos(d0) * math.cos(a - a0)
    xi = math.cos(d) * math.sin(a - a0) / D
    eta = (math.sin(d) * math.cos(d0) - math.cos(d) * math.sin(d0) * math.cos(a - a0)) / D
    return xi, eta


@pytest.mark.parametrize("dec0", DEC0S)
def test_pix2world_matches_textbook_gnomonic(dec0):
    # CD = identity (1 deg / px) so (u', v') in degrees equals the pixel offset; a 1000-point
    # grid of offsets up to 10 deg from the tangent point.
    w = synth.tan_wcs(10, 10, crval=(150.0, dec0), crpix=(1.0, 1.0))
    w["cd"] = [[1.0, 0.0], [0.0, 1.0]]
    rng = synth.rng_for(11)
    up = rng.uniform(-10, 10, 1000)
    vp = rng.uniform(-10, 10, 1000)
    ra, dec = W.pix2world(w, up, vp)
    for k in range(1000):
        ra_t, dec_t = _std_to_sky(math.radians(up[k]), math.radians(vp[k]), 150.0, dec0)
        dra = (math.radians(ra[k]) - ra_t + math.pi) % (2 * math.pi) - math.pi
        assert abs(dra * math.cos(dec_t)) < 1e-12
        assert abs(math.radians(dec[k]) - dec_t) < 1e-12


def test_equator_and_meridian_closed_forms():
    w = synth.tan_wcs(10, 10, crval=(0.0, 0.0), crpix=(1.0, 1.0))
    w["cd"] = [[1.0, 0.0], [0.0, 1.0]]
    t = np.linspace(-20.0, 20.0, 81)
    ra, dec = W.pix2world(w, t, np.zeros_like(t))
    np.testing.assert_allclose(np.radians(ra), np.arctan(np.radians(t)), rtol=0, atol=1e-14)
    np.testing.assert_allclose(dec, 0.0, atol=1e-14)
    ra, dec = W.pix2world(w, np.zeros_like(t), t)
    np.testing.assert_allclose(np.radians(dec), np.arctan(np.radians(t)), rtol=0, atol=1e-14)


@pytest.mark.parametrize("dec0", DEC0S)
def test_world_to_intermediate_matches_textbook(dec0):
    w = synth.tan_wcs(10, 10, crval=(150.0, dec0), crpix=(1.0, 1.0))
    w["cd"] = [[1.0, 0.0], [0.0, 1.0]]
    rng = synth.rng_for(12)
    for _ in range(300):
        ra = 150.0 + rng.uniform(-5, 5) / max(math.cos(math.radians(dec0)), 0.05)
        dec = min(dec0 + rng.uniform(-5, 5), 89.99)
        u, v, ok = W.world_to_intermediate(w, np.array([ra]), np.array([dec]))
        xi, eta = _sky_to_std(ra, dec, 150.0, dec0)
        assert ok[0]
        assert abs(math.radians(u[0]) - xi) < 1e-12 * max(1.0, abs(xi))
        assert abs(math.radians(v[0]) - eta) < 1e-12 * max(1.0, abs(eta))


@pytest.mark.parametrize("dec0", DEC0S)
def test_round_trip_tan(dec0):
    w = _wcs(dec0=dec0, n=(4096, 4096), crpix=(2048.5, 2048.5))
    rng = synth.rng_for(13)
    x = np.concatenate([rng.uniform(-0.5, 4095.5, 4000), 2047.5 + rng.uniform(-2, 2, 200)])
    y = np.concatenate([rng.uniform(-0.5, 4095.5, 4000), 2047.5 + rng.uniform(-2, 2, 200)])
    ra, dec = W.pix2world(w, x, y)
    x2, y2, ok = W.world2pix(w, ra, dec)
    assert ok.all()
    assert np.max(np.hypot(x2 - x, y2 - y)) < 1e-9


def test_round_trip_literal_asin_conditioning():
    """The printed theta = asin(D) agrees with the oracle's atan2 form within its conditioning
    bound |d theta| <= 4 eps / cos(theta), and meets 1e-9 px away from the tangent point."""
    w = _wcs(dec0=2.0, n=(8192, 8192), crpix=(4096.5, 4096.5))
    rng = synth.rng_for(14)
    x = rng.uniform(-0.5, 8191.5, 3000)
    y = rng.uniform(-0.5, 8191.5, 3000)
    ra, dec = W.pix2world(w, x, y, theta_mode="asin")
    xa, ya, _ = W.world2pix(w, ra, dec, theta_mode="asin")
    xt, yt, _ = W.world2pix(w, ra, dec)
    d = np.hypot(x - (w["crpix"][0] - 1), y - (w["crpix"][1] - 1))
    scale = math.radians(2.5 / 3600.0)
    bound = 8 * np.finfo(float).eps / np.maximum(d * scale, 1e-300) / scale  # px
    err = np.hypot(xa - xt, ya - yt)
    assert np.all(err <= bound + 1e-11)
    far = d > 3000
    assert np.max(np.hypot(xa - x, ya - y)[far]) < 1e-9


@pytest.mark.parametrize("dec0", [2.0, 60.0])
def test_round_trip_sip_newton(dec0):
    w = synth.add_sip(_wcs(dec0=dec0, n=(4096, 4096), crpix=(2048.5, 2048.5)), 3, 1e-6,
                      synth.rng_for(15))
    rng = synth.rng_for(16)
    x = rng.uniform(-0.5, 4095.5, 3000)
    y = rng.uniform(-0.5, 4095.5, 3000)
    ra, dec = W.pix2world(w, x, y)
    x2, y2, ok = W.world2pix(w, ra, dec, inverse="newton")
    assert ok.all()
    assert np.max(np.hypot(x2 - x, y2 - y)) < 1e-9


def test_affine_special_case_same_crval():
    """Same tangent point, no SIP: the TAN planes coincide, so the map is exactly affine:
    x_s - (crpix_s - 1) = CD_s^-1 CD_t (x_t - (crpix_t - 1))."""
    c = synth.config0()
    src, tgt = c["src"][0], c["tgt"]
    rng = synth.rng_for(17)
    xt = rng.uniform(-0.5, 511.5, 5000)
    yt = rng.uniform(-0.5, 511.5, 5000)
    xs, ys, ok = W.source_coords(src, tgt, xt, yt)
    A = np.linalg.solve(np.array(src["cd"]), np.array(tgt["cd"]))
    d = np.stack([xt - (tgt["crpix"][0] - 1), yt - (tgt["crpix"][1] - 1)])
    e = A @ d
    assert ok.all()
    assert np.max(np.abs(xs - (e[0] + src["crpix"][0] - 1))) < 1e-9
    assert np.max(np.abs(ys - (e[1] + src["crpix"][1] - 1))) < 1e-9


def _frame(ra0, dec0):
    """Columns = unit vectors (east, north, tangent point) of the tangent plane at (ra0, dec0)."""
    a, d = math.radians(ra0), math.radians(dec0)
    e0 = np.array([math.cos(d) * math.cos(a), math.cos(d) * math.sin(a), math.sin(d)])
    ex = np.array([-math.sin(a), math.cos(a), 0.0])
    ey = np.array([-math.sin(d) * math.cos(a), -math.sin(d) * math.sin(a), math.cos(d)])
    return np.stack([ex, ey, e0], axis=1)


@pytest.mark.parametrize("offset", [(0.05, 0.03), (1.0, -0.7), (-3.0, 5.0)])
def test_tan_to_tan_is_projective(offset):
    """Different tangent points, no SIP: the map between the two tangent planes is the
    homography proj(F_s^T F_t (xi, eta, 1)), built here from plain vector algebra."""
    src = _wcs(dec0=30.0, rho=0.3, n=(2048, 2048), crpix=(1024.5, 1024.5))
    tgt = _wcs(dec0=30.0 + offset[1], ra0=150.0 + offset[0], rho=-1.1, scale=2.6,
               n=(2048, 2048), crpix=(1000.2, 1050.9))
    rng = synth.rng_for(18)
    xt = rng.uniform(-0.5, 2047.5, 3000)
    yt = rng.uniform(-0.5, 2047.5, 3000)
    xs, ys, ok = W.source_coords(src, tgt, xt, yt)
    H = _frame(*src["crval"]).T @ _frame(*tgt["crval"])
    ct, cs = np.array(tgt["cd"]), np.array(src["cd"])
    d = np.stack([xt - (tgt["crpix"][0] - 1), yt - (tgt["crpix"][1] - 1)])
    st = np.radians(ct @ d)
    vec = H @ np.vstack([st, np.ones(xt.size)])
    ss = np.degrees(vec[:2] / vec[2])
    e = np.linalg.solve(cs, ss)
    good = ok & (vec[2] > 0)
    assert good.sum() > 100
    assert np.max(np.abs(xs - (e[0] + src["crpix"][0] - 1))[good]) < 1e-9
    assert np.max(np.abs(ys - (e[1] + src["crpix"][1] - 1))[good]) < 1e-9


def test_sip_sign_golden():
    """Hand-worked case of the SIP convention (Shupe et al. 2005): A_2_0 = 1e-5 moves u = 100,
    v = 0 to u = 100 + 1e-5 * 100^2 = 100.1. With CRVAL = (0, 0) and CD = diag(-1, 1)/3600 the
    point is on the equator at ra = atan(xi) with xi = -100.1 arcsec (in radians)."""
    text = open(__file__.replace("test_oracle_wcs.py", "golden/sip_sign_header.txt")).read()
    w = W.parse_header(text)
    expect = {}
    for line in open(__file__.replace("test_oracle_wcs.py", "golden/sip_sign_expect.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split("=")
            expect[k.strip()] = float(v)
    x = np.array([expect["x"]])
    y = np.array([expect["y"]])
    ra, dec = W.pix2world(w, x, y)
    assert abs(((ra[0] + 180.0) % 360.0 - 180.0) - expect["ra_deg"]) < 1e-13
    assert abs(dec[0] - expect["dec_deg"]) < 1e-13


def test_zero_sip_equals_plain_tan_bitwise():
    c = synth.config0()
    src, tgt = c["src"][0], c["tgt"]
    src_sip = synth.copy_wcs(src)
    src_sip["a_order"] = src_sip["b_order"] = 3
    src_sip["ap_order"] = src_sip["bp_order"] = 4
    rng = synth.rng_for(19)
    xt = rng.uniform(-0.5, 511.5, 2000)
    yt = rng.uniform(-0.5, 511.5, 2000)
    a = W.source_coords(src, tgt, xt, yt)
    b = W.source_coords(src_sip, tgt, xt, yt)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_inverse_sip_fit_residual_small_vs_newton():
    c = synth.config1()
    src = c["src"][0]
    src4, stats = W.with_inverse_sip(src, 4)
    assert stats["max_px"] < 0.05
    rng = synth.rng_for(20)
    x = rng.uniform(-0.5, 4095.5, 2000)
    y = rng.uniform(-0.5, 4095.5, 2000)
    ra, dec = W.pix2world(src4, x, y)
    xp, yp, _ = W.world2pix(src4, ra, dec, inverse="poly")
    xn, yn, _ = W.world2pix(src4, ra, dec, inverse="newton")
    assert np.max(np.hypot(xn - x, yn - y)) < 1e-9
    assert np.max(np.hypot(xp - xn, yp - yn)) <= stats["max_px"] * 1.5 + 1e-9


def test_sip_jacobian_stays_invertible():
    """The synthetic SIP draws keep det(I + J_SIP) well above 0.5 over each frame."""
    for cfg in (synth.config1(), synth.config3()):
        w = cfg["src"][0]
        Wd, Hd = w["naxis"]
        X, Y = np.meshgrid(np.linspace(-0.5, Wd - 0.5, 64), np.linspace(-0.5, Hd - 0.5, 64))
        u = X.ravel() - (w["crpix"][0] - 1)
        v = Y.ravel() - (w["crpix"][1] - 1)
        a = [[float(t) for t in r] for r in w["a"]]
        b = [[float(t) for t in r] for r in w["b"]]
        au, av = W.sip_partials(a, w["a_order"], u, v)
        bu, bv = W.sip_partials(b, w["b_order"], u, v)
        det = (1 + au) * (1 + bv) - av * bu
        assert det.min() > 0.5


def test_sip_partials_match_finite_differences():
    w = synth.add_sip(_wcs(n=(2048, 2048)), 5, 1e-7, synth.rng_for(21))
    a = [[float(t) for t in r] for r in w["a"]]
    u = np.array([-900.0, 13.0, 1000.0])
    v = np.array([700.0, -5.0, -1000.0])
    du, dv = W.sip_partials(a, 5, u, v)
    h = 1e-3
    fdu = (W.sip_value(a, 5, u + h, v) - W.sip_value(a, 5, u - h, v)) / (2 * h)
    fdv = (W.sip_value(a, 5, u, v + h) - W.sip_value(a, 5, u, v - h)) / (2 * h)
    np.testing.assert_allclose(du, fdu, rtol=1e-7, atol=1e-12)
    np.testing.assert_allclose(dv, fdv, rtol=1e-7, atol=1e-12)


def test_header_round_trip_is_exact():
    c = synth.config1()
    src, _ = W.with_inverse_sip(c["src"][0], 4)
    for sep in ("", "\n"):
        w = W.parse_header(synth.header_cards(src, sep))
        assert w["naxis"] == src["naxis"]
        assert w["crpix"] == src["crpix"] and w["crval"] == src["crval"]
        assert w["cd"] == src["cd"]
        for k in ("a", "b", "ap", "bp"):
            assert w[k + "_order"] == src[k + "_order"]
            assert np.array_equal(w[k], src[k])


def test_header_pc_cdelt_and_errors():
    base = synth.header_cards(_wcs(), "\n")
    lines = [ln for ln in base.split("\n") if not ln.startswith("CD")]
    pc = lines[:-1] + ["CDELT1  = -0.001", "CDELT2  = 0.002", "PC1_1   = 0.5",
                       "PC1_2   = 0.25", "PC2_1   = -0.25", "PC2_2   = 0.5", "END"]
    w = W.parse_header("\n".join(pc))
    assert w["cd"] == [[-0.0005, -0.00025], [-0.0005, 0.001]]
    with pytest.raises(W.HeaderError):
        W.parse_header(base.replace("RA---TAN", "RA---SIN"))
    assert W.parse_header(base.replace("END", "LONPOLE =                 170.\nEND"))[
        "lonpole"] == 170.0
    with pytest.raises(W.HeaderError):
        W.parse_header("\n".join(lines))


def test_lonpole_is_a_rotation_of_the_intermediate_plane():
    """General phi_p (LONPOLE) on the sphere equals phi_p = 180 deg with the intermediate plane
    rotated: the paper's native longitude is phi = atan2(-u', v'), so phi - d is the longitude of
    (u' cos d + v' sin d, -u' sin d + v' cos d). Both directions, 1e-12 deg / 1e-9 px, and the
    pixel -> world -> pixel round trip of the LONPOLE record."""
    rng = np.random.default_rng(5)
    w = _wcs()
    X = rng.uniform(-100, 600, 500)
    Y = rng.uniform(-100, 500, 500)
    for lon in (0.0, 100.0, 181.5, 300.0):
        d = np.radians(lon - 180.0)
        wl = dict(w, lonpole=lon)
        cd = np.array(w["cd"])
        rot = np.array([[np.cos(d), np.sin(d)], [-np.sin(d), np.cos(d)]]) @ cd
        wr = dict(w, cd=rot.tolist())
        ra_l, dec_l = W.pix2world(wl, X, Y)
        ra_r, dec_r = W.pix2world(wr, X, Y)
        dra = (ra_l - ra_r + 180.0) % 360.0 - 180.0
        assert np.abs(dra * np.cos(np.radians(dec_r))).max() < 1e-12
        assert np.abs(dec_l - dec_r).max() < 1e-12
        x, y, ok = W.world2pix(wl, ra_l, dec_l)
        assert ok.all() and np.abs(x - X).max() < 1e-9 and np.abs(y - Y).max() < 1e-9
        u_l, v_l, _ = W.world_to_intermediate(wl, ra_r, dec_r)
        u_r, v_r, _ = W.world_to_intermediate(wr, ra_r, dec_r)
        assert np.abs(u_l - u_r).max() < 1e-9 and np.abs(v_l - v_r).max() < 1e-9
