"""Pins of the oracle co-add (oracle.reproject.coadd), independent of its own formula:

  * constant exposures: the co-add mean is that constant on every covered pixel (the footprint
    normalisation of Sec. 3.1 makes each exposure's value the constant exactly, up to rounding);
  * a partition: an exposure cut into two halves (the halves' WCS are the whole frame's with
    CRPIX moved by the cut) co-adds to the reprojection of the whole exposure, nearest
    neighbour, on every pixel not at the seam;
  * disjoint exposures add without interaction, and a repeated exposure doubles the sums.
"""
import numpy as np

import synth
from oracle import reproject as OR
from oracle import wcs as OW


def _frames(seed, n, w=60, h=44):
    rng = synth.rng_for(seed)
    out = []
    for k in range(n):
        s = synth.tan_wcs(w, h, rho_deg=float(rng.uniform(-2, 2)),
                          crpix=((w + 1) / 2 + rng.uniform(-6, 6), (h + 1) / 2 + rng.uniform(-6, 6)))
        s = synth.add_sip(s, 3, 1e-6, rng)
        s, _ = OW.with_inverse_sip(s, 4)
        out.append((s, synth.sky_image(w, h, 5, rng)))
    return out


def test_constant_exposures_give_constant_mean():
    tgt = synth.tan_wcs(72, 56, rho_deg=0.7)
    frames = [(s, np.full_like(img, 3.25)) for s, img in _frames(3, 4)]
    for order in ("bilinear", "bicubic"):
        sv, sf = OR.coadd(frames, tgt, order)
        cov = sf > 0
        assert cov.sum() > 0.5 * cov.size
        assert np.abs(sv[cov] / sf[cov] - 3.25).max() < 1e-12
        assert np.all(sv[~cov] == 0)


def test_partition_of_an_exposure_coadds_to_the_whole():
    rng = synth.rng_for(8)
    W, H = 64, 48
    src = synth.tan_wcs(W, H, rho_deg=1.3)
    img = synth.sky_image(W, H, 8, rng)
    tgt = synth.tan_wcs(70, 54, rho_deg=-0.4, crpix=(36.2, 27.9))
    cut = 29
    left = synth.copy_wcs(src)
    left["naxis"] = (cut, H)
    right = synth.copy_wcs(src)
    right["naxis"] = (W - cut, H)
    right["crpix"] = (src["crpix"][0] - cut, src["crpix"][1])
    frames = [(left, img[:, :cut].copy()), (right, img[:, cut:].copy())]
    sv, sf = OR.coadd(frames, tgt, "nearest")
    val, fp, xs, ys = OR.reproject(src, tgt, img, "nearest")
    seam = np.abs(xs - (cut - 0.5)) < 1e-6
    ok = ~seam & np.isfinite(xs)
    assert np.array_equal(sf[ok], fp[ok])
    assert np.array_equal(sv[ok], (val * fp)[ok])


def test_disjoint_and_repeated_exposures():
    tgt = synth.tan_wcs(200, 60)
    rng = synth.rng_for(9)
    a = synth.tan_wcs(50, 40, crpix=(25.5 + 60, 20.5))   # left part of the target
    b = synth.tan_wcs(50, 40, crpix=(25.5 - 60, 20.5))   # right part
    ia, ib = synth.sky_image(50, 40, 4, rng), synth.sky_image(50, 40, 4, rng)
    sva, sfa = OR.coadd([(a, ia)], tgt, "bicubic")
    svb, sfb = OR.coadd([(b, ib)], tgt, "bicubic")
    assert not np.any((sfa > 0) & (sfb > 0))
    sv, sf = OR.coadd([(a, ia), (b, ib)], tgt, "bicubic")
    assert np.array_equal(sv, sva + svb) and np.array_equal(sf, sfa + sfb)
    sv2, sf2 = OR.coadd([(a, ia), (a, ia)], tgt, "bicubic")
    assert np.array_equal(sv2, 2 * sva) and np.array_equal(sf2, 2 * sfa)
    # an explicit pixel list gives the grid values at those pixels
    xt, yt = np.array([3.0, 70.0, 150.0]), np.array([5.0, 30.0, 59.0])
    pv, pf = OR.coadd([(a, ia), (b, ib)], tgt, "bicubic", pixels=(xt, yt))
    assert np.array_equal(pv, sv[yt.astype(int), xt.astype(int)])
    assert np.array_equal(pf, sf[yt.astype(int), xt.astype(int)])
