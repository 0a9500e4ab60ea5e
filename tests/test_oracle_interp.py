"""Pins for the oracle's interpolation, footprint and adjoint (Sec. 3.1 step 3) — CPU only."""
import numpy as np
import pytest
import scipy.ndimage

import synth
from oracle import interp as I
from oracle import reproject as R


def _golden_keys():
    rows = {}
    path = __file__.replace("test_oracle_interp.py", "golden/keys_weights.txt")
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            t, *w = line.split()
            rows[float(t)] = [float(eval(x)) for x in w]
    return rows


def test_keys_weights_golden():
    """Textbook Keys (a = -0.5) weights at t = 0, 0.25, 0.5 (tests/golden/keys_weights.txt)."""
    for t, w in _golden_keys().items():
        i0, wx = I.taps_1d(np.array([10.0 + t]), I.BICUBIC)
        assert i0[0] == 9
        np.testing.assert_allclose(wx[:, 0], w, rtol=0, atol=1e-15)


@pytest.mark.parametrize("a", [-0.5, -0.75])
def test_keys_partition_of_unity(a):
    t = np.linspace(0, 1, 101)[:-1]
    _, wx = I.taps_1d(5.0 + t, I.BICUBIC, a)
    np.testing.assert_allclose(wx.sum(axis=0), 1.0, atol=1e-15)


def test_nearest_integer_shift_bit_exact():
    rng = synth.rng_for(30)
    img = rng.standard_normal((40, 50)).astype(np.float32)
    Y, X = np.mgrid[0:40, 0:50].astype(np.float64)
    val, fp = I.interpolate(img, X + 3.0, Y - 2.0, I.NEAREST)
    exp = np.zeros((40, 50))
    exp[2:, :47] = img[:38, 3:]
    assert np.array_equal(val, exp)
    assert set(np.unique(fp)) <= {0.0, 1.0}
    assert np.array_equal(fp != 0, exp != 0)


def test_nearest_half_pixel_ties_round_up():
    """Positions exactly halfway between pixel centres go to the upper pixel (index
    floor(x + 0.5)); round-half-even or round-half-down would pick the lower one at every other
    (or every) column. At x = W - 0.5 the position is covered but its pixel lies outside the
    image: value and footprint 0."""
    rng = synth.rng_for(31)
    img = rng.standard_normal((40, 50)).astype(np.float32)
    Y, X = np.mgrid[0:40, 0:50].astype(np.float64)
    val, fp = I.interpolate(img, X + 0.5, Y - 1.5, I.NEAREST)
    exp = np.zeros((40, 50))
    exp[1:, :49] = img[:39, 1:]
    assert np.array_equal(val, exp)
    efp = np.zeros((40, 50))
    efp[1:, :49] = 1.0
    assert np.array_equal(fp, efp)
    # negative half: -0.5 is covered and rounds up to pixel 0
    v, f = I.interpolate(img, np.array([-0.5, 0.5, 1.5, 2.5]), np.array([0.0, 0.0, 0.0, 0.0]),
                         I.NEAREST)
    assert np.array_equal(v, img[0, [0, 1, 2, 3]].astype(np.float64))
    assert np.array_equal(f, np.ones(4))


@pytest.mark.parametrize("order", [I.NEAREST, I.BILINEAR, I.BICUBIC])
def test_identity_bit_exact(order):
    rng = synth.rng_for(31)
    img = rng.standard_normal((33, 47)).astype(np.float32)
    Y, X = np.mgrid[0:33, 0:47].astype(np.float64)
    eps = 1e-11 * rng.standard_normal(X.shape)  # transform round-off below the snap radius
    val, fp = I.interpolate(img, X + eps, Y - eps, order)
    assert np.array_equal(val.astype(np.float32), img)
    assert np.all(fp == 1.0)


def test_bilinear_reproduces_linear_ramp():
    Y, X = np.mgrid[0:64, 0:80].astype(np.float64)
    img = 0.37 * X - 1.3 * Y + 12.0
    rng = synth.rng_for(32)
    x = rng.uniform(0, 79, 5000)
    y = rng.uniform(0, 63, 5000)
    val, fp = I.interpolate(img, x, y, I.BILINEAR)
    np.testing.assert_allclose(val, 0.37 * x - 1.3 * y + 12.0, rtol=0,
                               atol=1e-6 * np.abs(img).max())
    np.testing.assert_allclose(fp, 1.0, atol=1e-15)


def test_bicubic_reproduces_quadratic():
    Y, X = np.mgrid[0:64, 0:80].astype(np.float64)
    f = lambda x, y: 0.01 * x * x - 0.02 * x * y + 0.005 * y * y + 0.3 * x - 0.1 * y + 2.0
    img = f(X, Y)
    rng = synth.rng_for(33)
    x = rng.uniform(1, 77, 5000)
    y = rng.uniform(1, 61, 5000)
    val, _ = I.interpolate(img, x, y, I.BICUBIC)
    np.testing.assert_allclose(val, f(x, y), rtol=0, atol=1e-6 * np.abs(img).max())


@pytest.mark.parametrize("order", [I.NEAREST, I.BILINEAR, I.BICUBIC])
def test_constant_image_and_footprint(order):
    img = np.full((20, 30), 7.25)
    rng = synth.rng_for(34)
    x = rng.uniform(-2, 31, 20000)
    y = rng.uniform(-2, 21, 20000)
    val, fp = I.interpolate(img, x, y, order)
    cov = (x >= -0.5) & (x <= 29.5) & (y >= -0.5) & (y <= 19.5) & (fp > 0)
    assert np.all(np.abs(val[cov] - 7.25) <= 8 * np.spacing(7.25))
    assert np.all(val[~cov] == 0) and np.all(fp[~cov] == 0)
    inner = (x >= 2) & (x <= 27) & (y >= 2) & (y <= 17)
    np.testing.assert_allclose(fp[inner], 1.0, atol=1e-15)


def test_footprint_at_edges_is_in_bounds_weight_sum():
    img = np.ones((10, 10))
    # x = -0.5: bilinear taps -1 (out), 0 (in, w = 0.5); bicubic taps -2..1 with
    # weights (-1/16, 9/16, 9/16, -1/16), in-bounds 0, 1 -> 0.5.
    for order, exp in ((I.BILINEAR, 0.5), (I.BICUBIC, 0.5), (I.NEAREST, 1.0)):
        _, fp = I.interpolate(img, np.array([-0.5]), np.array([5.0]), order)
        assert abs(fp[0] - exp) < 1e-15
        _, fp = I.interpolate(img, np.array([-0.5]), np.array([-0.5]), order)
        assert abs(fp[0] - exp * exp) < 1e-15
    _, fp = I.interpolate(img, np.array([-0.51]), np.array([5.0]), I.BILINEAR)
    assert fp[0] == 0.0


@pytest.mark.parametrize("order", [0, 1])
def test_matches_scipy_map_coordinates(order):
    """Unnormalised sums equal scipy's spline interpolation of order 0/1 with zero padding."""
    rng = synth.rng_for(35)
    img = rng.standard_normal((30, 40))
    x = rng.uniform(-0.5, 39.5, 4000)
    y = rng.uniform(-0.5, 29.5, 4000)
    if order == 0:  # keep away from rounding ties, where the two conventions differ
        x = np.floor(x) + np.clip(x - np.floor(x), 0.01, 0.49)
    val, fp = I.interpolate(img, x, y, order)
    ref = scipy.ndimage.map_coordinates(img, [y, x], order=order, mode="constant", cval=0.0)
    # scipy's constant mode returns cval for any position outside [0, n-1], so compare there
    inner = (x >= 0) & (x <= 39) & (y >= 0) & (y <= 29)
    assert inner.sum() > 3000
    np.testing.assert_allclose(val[inner], ref[inner], rtol=0, atol=1e-12 if order else 0)
    np.testing.assert_allclose(fp[inner], 1.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [I.NEAREST, I.BILINEAR, I.BICUBIC, I.LANCZOS3, I.BSPLINE3])
def test_adjoint_dot_product_and_dense(order):
    """<W s, g> = <s, W^T g> to 1e-12, and W built column by column from unit images equals the
    transpose built by the adjoint from unit gradients (brute force, 16x16)."""
    rng = synth.rng_for(36)
    H = Wd = 16
    x = rng.uniform(-1, 16, 200)
    y = rng.uniform(-1, 16, 200)
    s = rng.standard_normal((H, Wd))
    g = rng.standard_normal(200)
    val, _ = I.interpolate(s, x, y, order)
    adj = I.interpolate_adjoint((H, Wd), x, y, order, g)
    assert abs(np.dot(val, g) - np.sum(s * adj)) < 1e-12 * max(1.0, abs(np.dot(val, g)))
    Wm = np.zeros((200, H * Wd))
    for j in range(H * Wd):
        e = np.zeros(H * Wd)
        e[j] = 1.0
        Wm[:, j] = I.interpolate(e.reshape(H, Wd), x, y, order)[0]
    Wt = np.zeros((H * Wd, 200))
    for p in range(200):
        e = np.zeros(200)
        e[p] = 1.0
        Wt[:, p] = I.interpolate_adjoint((H, Wd), x, y, order, e).ravel()
    np.testing.assert_allclose(Wm.T, Wt, rtol=0, atol=1e-14)


def test_bspline3_image_adjoint_dense():
    """The B-spline path from the image: value = evaluate(prefilter(S)). Its matrix, built
    column by column from unit images, equals the transpose of prefilter_adjoint o
    interpolate_adjoint built from unit gradients (brute force, 10x13 image, 150 positions)."""
    rng = synth.rng_for(37)
    H, Wd = 10, 13
    x = rng.uniform(-0.5, Wd - 0.5, 150)
    y = rng.uniform(-0.5, H - 0.5, 150)
    Wm = np.zeros((150, H * Wd))
    for j in range(H * Wd):
        e = np.zeros(H * Wd)
        e[j] = 1.0
        Wm[:, j] = I.interpolate(I.bspline3_prefilter(e.reshape(H, Wd)), x, y, I.BSPLINE3)[0]
    Wt = np.zeros((H * Wd, 150))
    for p in range(150):
        e = np.zeros(150)
        e[p] = 1.0
        Wt[:, p] = I.bspline3_prefilter_adjoint(
            I.interpolate_adjoint((H, Wd), x, y, I.BSPLINE3, e)).ravel()
    np.testing.assert_allclose(Wm.T, Wt, rtol=0, atol=1e-13)
    # the prefilter matrix is the filter itself: its product with a vector is the filter
    v = rng.standard_normal(H)
    np.testing.assert_allclose(I.bspline3_prefilter_matrix(H) @ v,
                               I.bspline3_prefilter_1d(v, 0), rtol=0, atol=1e-14)


def test_reprojection_identity_wcs_bit_exact():
    c = synth.config0()
    src = c["src"][0]
    img = c["images"][0]
    for order in ("nearest", "bilinear", "bicubic"):
        val, fp, _, _ = R.reproject(src, src, img, order)
        assert np.array_equal(val.astype(np.float32), img)
        assert np.all(fp == 1.0)


def test_reprojection_integer_crpix_shift_nearest_bit_exact():
    c = synth.config0()
    src = c["src"][0]
    tgt = synth.copy_wcs(src)
    tgt["crpix"] = (src["crpix"][0] + 5.0, src["crpix"][1] - 3.0)
    img = c["images"][0]
    val, fp, _, _ = R.reproject(src, tgt, img, "nearest")
    exp = np.zeros_like(val)
    exp[:509, 5:] = img[3:, :507]
    assert np.array_equal(val, exp)
    assert np.array_equal(fp, (exp != 0).astype(float)) or set(np.unique(fp)) <= {0.0, 1.0}


def test_target_bbox_contains_covered_pixels():
    c = synth.config0()
    src, tgt = c["src"][0], synth.copy_wcs(c["tgt"])
    tgt["naxis"] = (700, 640)
    tgt["crpix"] = (tgt["crpix"][0] + 60, tgt["crpix"][1] + 40)
    x0, y0, w, h = R.target_bbox(src, tgt)
    _, fp, _, _ = R.reproject(src, tgt, c["images"][0], "bilinear")
    ys, xs = np.nonzero(fp)
    assert xs.min() >= x0 and xs.max() < x0 + w and ys.min() >= y0 and ys.max() < y0 + h
    assert w <= 512 + 20 and h <= 512 + 20


def test_nan_mask_pins():
    """NaN-masked interpolation: (1) an image without NaN gives the unmasked result bit for bit;
    (2) bilinear next to one NaN tap equals the renormalised average of the other three taps,
    worked by hand; (3) a constant image with NaN holes interpolates to the constant wherever
    anything is left, and nearest on a NaN pixel is uncovered; (4) the footprint at an interior
    point is one minus the weight of the NaN taps."""
    rng = np.random.default_rng(3)
    img = rng.standard_normal((20, 24))
    x = rng.uniform(-0.5, 23.5, 300)
    y = rng.uniform(-0.5, 19.5, 300)
    for order in (I.NEAREST, I.BILINEAR, I.BICUBIC):
        a = I.interpolate(img, x, y, order)
        b = I.interpolate(img, x, y, order, nan_mask=True)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    holed = img.copy()
    holed[5, 7] = np.nan
    # bilinear at (7.25, 4.5): taps (7,4) (8,4) (7,5) (8,5) with weights .375 .125 .375 .125
    v, f = I.interpolate(holed, np.array([7.25]), np.array([4.5]), I.BILINEAR, nan_mask=True)
    w = {(4, 7): 0.375, (4, 8): 0.125, (5, 8): 0.125}
    expect = sum(wt * holed[r, c] for (r, c), wt in w.items()) / 0.625
    assert abs(f[0] - 0.625) < 1e-15 and abs(v[0] - expect) < 1e-14
    const = np.full((20, 24), 2.5)
    const[rng.integers(0, 20, 40), rng.integers(0, 24, 40)] = np.nan
    for order in (I.BILINEAR, I.BICUBIC):
        v, f = I.interpolate(const, x, y, order, nan_mask=True)
        assert np.all(np.abs(v[f > 0] - 2.5) < 1e-12)
    v, f = I.interpolate(holed, np.array([7.2]), np.array([5.1]), I.NEAREST, nan_mask=True)
    assert f[0] == 0.0 and v[0] == 0.0
    v, f = I.interpolate(holed, np.array([6.6]), np.array([5.0]), I.BICUBIC, nan_mask=True)
    ix, wx = I.taps_1d(np.array([6.6]), I.BICUBIC, -0.5)
    wnan = wx[7 - ix[0], 0] * 1.0  # y = 5 exactly: the row weight of row 5 is 1
    assert abs(f[0] - (1.0 - wnan)) < 1e-14


def test_nan_mask_nonpositive_remaining_weight_is_uncovered():
    """Bicubic at t = 1/2 in x: weights (-1/16, 9/16, 9/16, -1/16). With both central columns
    missing the remaining weight is -1/8 < 0: the pixel is uncovered (value and footprint 0)."""
    img = np.arange(8 * 8, dtype=np.float64).reshape(8, 8)
    img[:, 3:5] = np.nan
    v, f = I.interpolate(img, np.array([3.5]), np.array([3.0]), I.BICUBIC, nan_mask=True)
    assert v[0] == 0.0 and f[0] == 0.0
    v, f = I.interpolate(img, np.array([3.5]), np.array([3.0]), I.BILINEAR, nan_mask=True)
    assert v[0] == 0.0 and f[0] == 0.0  # both bilinear taps missing


def test_lanczos3_pins():
    """Lanczos-3: closed-form weights at t = 1/2 (sinc(1/2) = 2/pi, sinc(1/6) = 3/pi,
    sinc(3/2) = -2/(3 pi), sinc(5/2) = 2/(5 pi), sinc(5/6) = 3/(5 pi)), interpolation at the
    nodes (weights 1 at the node), symmetry w_k(t) = w_{5-k}(1 - t), partition of unity, and a
    constant image reproduced on every covered pixel."""
    pi = np.pi
    L05 = (2 / pi) * (3 / pi)
    L15 = (-2 / (3 * pi)) * (2 / pi)
    L25 = (2 / (5 * pi)) * (3 / (5 * pi))
    raw = np.array([L25, L15, L05, L05, L15, L25])
    i0, w = I.taps_1d(np.array([4.5]), I.LANCZOS3)
    assert i0[0] == 2
    assert np.allclose(w[:, 0], raw / raw.sum(), rtol=0, atol=1e-15)
    for x in (0.0, 3.0, 7.0):
        _, w = I.taps_1d(np.array([x]), I.LANCZOS3)
        assert np.allclose(w[:, 0], [0, 0, 1, 0, 0, 0], rtol=0, atol=1e-15)
    t = np.linspace(0.01, 0.99, 57)
    _, w = I.taps_1d(t, I.LANCZOS3)
    _, wr = I.taps_1d(1.0 - t, I.LANCZOS3)
    assert np.allclose(w, wr[::-1], rtol=0, atol=1e-14)
    assert np.allclose(w.sum(axis=0), 1.0, rtol=0, atol=1e-14)
    rng = np.random.default_rng(11)
    img = rng.standard_normal((20, 30))
    xs, ys = np.meshgrid(np.arange(30.0), np.arange(20.0))
    v, f = I.interpolate(img, xs.ravel(), ys.ravel(), I.LANCZOS3)
    assert np.allclose(v, img.ravel(), rtol=0, atol=1e-12)
    v, f = I.interpolate(np.full((20, 30), 1.75), rng.uniform(-0.5, 29.5, 400),
                         rng.uniform(-0.5, 19.5, 400), I.LANCZOS3)
    assert np.all(f > 0) and np.abs(v - 1.75).max() < 1e-12


def test_bspline3_prefilter_and_interpolation_pins():
    """Cubic B-spline: (1) the prefilter matches scipy's spline_filter (mirror mode) to 1e-12;
    (2) the spline through the coefficients passes through every pixel (B3 weights 1/6, 2/3, 1/6
    at the nodes), independently of scipy; (3) evaluation off the nodes, inside and out to the
    coverage edge, matches scipy's map_coordinates(order=3, mode='mirror'); (4) the weights are
    the closed form at t = 1/2 (1/48, 23/48, 23/48, 1/48) and sum to 1."""
    rng = np.random.default_rng(21)
    for shape in ((23, 31), (5, 7), (2, 9), (1, 6)):
        img = rng.standard_normal(shape)
        c = I.bspline3_prefilter(img)
        ref = scipy.ndimage.spline_filter(img, order=3, mode="mirror")
        assert np.abs(c - ref).max() < 1e-12
        H, W = shape
        ys, xs = np.meshgrid(np.arange(H, dtype=float), np.arange(W, dtype=float), indexing="ij")
        v, f = I.interpolate(c, xs.ravel(), ys.ravel(), I.BSPLINE3)
        assert np.abs(v - img.ravel()).max() < 1e-12 and np.all(f == 1.0)
    img = rng.standard_normal((23, 31))
    c = I.bspline3_prefilter(img)
    x = rng.uniform(-0.5, 30.5, 500)
    y = rng.uniform(-0.5, 22.5, 500)
    v, f = I.interpolate(c, x, y, I.BSPLINE3)
    ref = scipy.ndimage.map_coordinates(img, [y, x], order=3, mode="mirror")
    assert np.abs(v - ref).max() < 1e-10 and np.all(f == 1.0)
    _, w = I.taps_1d(np.array([3.5]), I.BSPLINE3)
    assert np.allclose(w[:, 0], [1 / 48, 23 / 48, 23 / 48, 1 / 48], rtol=0, atol=1e-15)
    _, w = I.taps_1d(rng.uniform(0, 20, 100), I.BSPLINE3)
    assert np.allclose(w.sum(axis=0), 1.0, rtol=0, atol=1e-14)
