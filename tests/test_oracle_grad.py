"""Pins for the oracle's forward-mode gradients — CPU only.

The dual-number gradient of L = sum (O(theta) - O_ref)^2 is checked against FP64 central
finite differences of the plain oracle, with per-parameter steps that move no source
coordinate by more than 1e-6 px (so a bilinear kink is crossed by almost no pixel).
"""
import numpy as np
import pytest

import synth
from oracle import dual as D
from oracle import reproject as R
from oracle import wcs as W


def _small_case(order="bilinear", n=96, seed=40):
    rng = synth.rng_for(seed)
    src = synth.add_sip(synth.tan_wcs(n, n), 3, 1e-6, rng)
    # stronger distortion than the 1e-6 draw so every SIP term matters at this size
    src["a"] *= 200.0
    src["b"] *= 200.0
    src, _ = W.with_inverse_sip(src, 4)
    tgt = synth.tan_wcs(n, n)
    img = synth.sky_image(n, n, 12, rng)
    pert = synth.copy_wcs(src)
    pert["crval"] = (src["crval"][0] + 0.3 / 3600, src["crval"][1] + 0.3 / 3600)
    pert["cd"] = [[c * (1 + 1e-4) for c in row] for row in src["cd"]]
    pert["a"] = src["a"] * 1.1
    pert["b"] = src["b"] * 1.1
    ref, _, _, _ = R.reproject(pert, tgt, img, order, inverse="newton")
    return src, tgt, img, ref


def test_dual_values_match_plain_oracle():
    src, tgt, img, _ = _small_case("bicubic")
    Y, X = np.mgrid[0:96, 0:96].astype(np.float64)
    o, _ = D.reproject_dual(src, tgt, img, X.ravel(), Y.ravel(), "bicubic")
    val, _, _, _ = R.reproject(src, tgt, img, "bicubic", inverse="newton", use_snap=False)
    np.testing.assert_allclose(o.v, val.ravel(), rtol=0, atol=1e-12)


def test_dual_coordinate_derivatives_match_fd():
    src, tgt, _, _ = _small_case()
    rng = synth.rng_for(41)
    xt = rng.uniform(0, 95, 50)
    yt = rng.uniform(0, 95, 50)
    ra, dec = W.pix2world(tgt, xt, yt)
    dsrc, names = D.dual_wcs(src)
    x, y, _ = W.world2pix(dsrc, ra, dec, inverse="newton", m=D)
    theta = D.flat_params(src)
    steps = fd_steps(src, tgt, px=1e-3)
    for i in range(len(names)):
        h = steps[i]
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        xp, yp, _ = W.world2pix(D.set_params(src, tp), ra, dec, inverse="newton")
        xm, ym, _ = W.world2pix(D.set_params(src, tm), ra, dec, inverse="newton")
        fdx = (xp - xm) / (2 * h)
        fdy = (yp - ym) / (2 * h)
        scale = max(np.abs(x.d[i]).max(), np.abs(y.d[i]).max(), 1e-30)
        assert np.max(np.abs(fdx - x.d[i])) < 1e-5 * scale, names[i]
        assert np.max(np.abs(fdy - y.d[i])) < 1e-5 * scale, names[i]


def fd_steps(src, tgt, px=1e-6):
    """Per-parameter step that moves no source coordinate by more than ``px`` pixels."""
    n = tgt["naxis"][0]
    Y, X = np.mgrid[0:n:4, 0:n:4].astype(np.float64)
    ra, dec = W.pix2world(tgt, X.ravel(), Y.ravel())
    dsrc, _ = D.dual_wcs(src)
    x, y, ok = W.world2pix(dsrc, ra, dec, inverse="newton", m=D)
    mx = np.maximum(np.abs(x.d[:, ok]).max(axis=1), np.abs(y.d[:, ok]).max(axis=1))
    return px / np.maximum(mx, 1e-300)


def test_dual_sinc_derivative_matches_fd():
    """The dual sinc's derivative (closed form, and its series below |x| = 1e-3) against FP64
    central differences of numpy's sinc, across the series boundary and at the nodes."""
    for x0 in (0.0, 1e-7, -4e-4, 9.99e-4, 1.001e-3, -0.3, 1.0, 2.7, -3.0):
        d = D.sinc(D.Dual(np.array([x0]), np.array([[1.0]])))
        h = 1e-5
        fd = (np.sinc(x0 + h) - np.sinc(x0 - h)) / (2 * h)
        assert abs(d.v[0] - np.sinc(x0)) == 0.0
        assert abs(d.d[0, 0] - fd) < 1e-9, (x0, d.d[0, 0], fd)


def test_dual_lanczos3_values_match_plain_oracle():
    src, tgt, img, _ = _small_case("lanczos3")
    Y, X = np.mgrid[0:96, 0:96].astype(np.float64)
    o, _ = D.reproject_dual(src, tgt, img, X.ravel(), Y.ravel(), "lanczos3")
    val, _, _, _ = R.reproject(src, tgt, img, "lanczos3", inverse="newton", use_snap=False)
    np.testing.assert_allclose(o.v, val.ravel(), rtol=0, atol=1e-12)


def test_dual_bspline3_values_match_plain_oracle():
    """B-spline duals (the image is taken as the coefficient array) against the plain oracle."""
    src, tgt, img, _ = _small_case("bspline3")
    Y, X = np.mgrid[0:96, 0:96].astype(np.float64)
    o, _ = D.reproject_dual(src, tgt, img, X.ravel(), Y.ravel(), "bspline3")
    val, _, _, _ = R.reproject(src, tgt, img, "bspline3", inverse="newton", use_snap=False)
    np.testing.assert_allclose(o.v, val.ravel(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("order", ["bilinear", "bicubic", "lanczos3", "bspline3"])
def test_loss_gradient_matches_central_fd(order):
    src, tgt, img, ref = _small_case(order)
    loss, grad, names = D.loss_grad(src, tgt, img, ref, order)
    theta = D.flat_params(src)
    steps = fd_steps(src, tgt)

    def L(th):
        o, _, _, _ = R.reproject(D.set_params(src, th), tgt, img, order, inverse="newton",
                                 use_snap=False)
        return float(np.sum((o - ref) ** 2))

    groups = {"crval": range(0, 2), "cd": range(2, 6), "sip": range(6, len(names))}
    fd = np.zeros_like(grad)
    for i in range(len(names)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += steps[i]
        tm[i] -= steps[i]
        fd[i] = (L(tp) - L(tm)) / (2 * steps[i])
    for g, idx in groups.items():
        idx = list(idx)
        gmax = np.abs(grad[idx]).max()
        for i in idx:
            tol = 1e-4 * max(abs(grad[i]), 1e-3 * gmax)
            assert abs(fd[i] - grad[i]) <= tol, (names[i], fd[i], grad[i])
