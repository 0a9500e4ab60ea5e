"""Argument checks of the Python binding that keep every launch inside the caller's tensors
(host side, no GPU): images at least NAXIS2 x NAXIS1, value planes at least the box, the
footprint plane the value plane's shape and row stride."""
import pytest

torch = pytest.importorskip("torch")

import synth
import paper_2505_03932_gb300 as dfr


def _wcs(w, h):
    return synth.tan_wcs(w, h)


def test_image_smaller_than_naxis_is_refused():
    w = _wcs(64, 48)
    dfr._check_image(torch.empty((48, 64)), w, "img")
    dfr._check_image(torch.empty((50, 70)), w, "img")  # larger is fine (a view of it is read)
    for shape in [(47, 64), (48, 63), (10, 10)]:
        with pytest.raises(ValueError):
            dfr._check_image(torch.empty(shape), w, "img")


def test_output_smaller_than_box_is_refused():
    out = torch.empty((32, 40))
    dfr._check_out(out, None, 40, 32)
    dfr._check_out(out, torch.empty((32, 40)), 40, 32)
    with pytest.raises(ValueError):
        dfr._check_out(out, None, 41, 32)
    with pytest.raises(ValueError):
        dfr._check_out(out, None, 40, 33)


def test_footprint_must_match_value_plane():
    out = torch.empty((32, 40))
    with pytest.raises(ValueError):
        dfr._check_out(out, torch.empty((32, 41)), 40, 32)
    # same shape but another row stride (a column slice of a wider buffer)
    wide = torch.empty((32, 48))[:, :40]
    with pytest.raises(ValueError):
        dfr._check_out(out, wide, 40, 32)


def test_noalloc_bspline_needs_prefiltered_coefficients():
    with pytest.raises(ValueError, match="prefiltered"):
        dfr.reproject_batch_noalloc([], [], _wcs(8, 8), [], [], order="bspline3")


def test_backward_batch_lists_must_agree():
    w = _wcs(8, 8)
    with pytest.raises(ValueError, match="same length"):
        dfr.reproject_backward_batch([None, None], [w], w, [None, None], [(0, 0, 8, 8)] * 2)
    with pytest.raises(ValueError, match="one entry per frame"):
        dfr.reproject_backward_batch([None], [w], w, [None], [(0, 0, 8, 8)], grad_srcs=[])
