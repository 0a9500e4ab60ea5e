"""GPU parity of the adjoint (dfr_reproject_backward) with the oracle, through the C ABI.

  * grad_src: equals the oracle's interpolation adjoint applied at the GPU's own coordinates,
    element by element (|d| <= 1e-5 |g_i| + 1e-6 max|g|); the GPU pair (forward, backward) passes
    the dot-product test <W s, g> = <s, W^T g> to 1e-5.
  * grad_params: given the same output gradient, equals the oracle's forward-mode dual-number
    gradient to 1e-4 * max(|g_ref|, 1e-3 * max |g_group|) (CRVAL, CD, SIP groups).
"""
import numpy as np
import pytest

import synth
from oracle import dual as OD
from oracle import interp as OI
from oracle import reproject as OR
from oracle import wcs as OW

from gpu_util import dfr, gpu, to_dev, torch

pytestmark = pytest.mark.gpu


def _case(n=256, order="bilinear", seed=5, boost=200.0):
    rng = synth.rng_for(seed)
    src = synth.add_sip(synth.tan_wcs(n, n), 3, 1e-6, rng)
    src["a"] *= boost
    src["b"] *= boost
    src, _ = OW.with_inverse_sip(src, 4)
    tgt = synth.tan_wcs(n, n)
    img = synth.sky_image(n, n, max(4, n * n // 4000), rng)
    pert = synth.copy_wcs(src)
    pert["crval"] = (src["crval"][0] + 0.3 / 3600, src["crval"][1] + 0.3 / 3600)
    pert["cd"] = [[c * (1 + 1e-4) for c in row] for row in src["cd"]]
    pert["a"] = src["a"] * 1.1
    pert["b"] = src["b"] * 1.1
    ref, _, _, _ = OR.reproject(pert, tgt, img, order, inverse="newton")
    return src, tgt, img, ref


def _group_check(grad, ref, names):
    groups = {"crval": [0, 1], "cd": [2, 3, 4, 5], "sip": list(range(6, len(names)))}
    worst = 0.0
    for idx in groups.values():
        if not idx:
            continue
        gmax = np.abs(ref[idx]).max()
        for i in idx:
            tol = 1e-4 * max(abs(ref[i]), 1e-3 * gmax)
            worst = max(worst, abs(grad[i] - ref[i]) / tol)
            assert abs(grad[i] - ref[i]) <= tol, (names[i], grad[i], ref[i])
    return worst


@pytest.mark.parametrize("order", ["nearest", "bilinear", "bicubic", "lanczos3"])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_grad_src_matches_oracle_adjoint(order, precision):
    src, tgt, img, _ = _case(order=order)
    n = 256
    bbox = (0, 0, n, n)
    img_d = to_dev(img)
    val, fp, cr = gpu(src, tgt, img_d, order, precision, bbox)
    g = synth.rng_for(9).standard_normal((n, n)).astype(np.float32)
    gs, _ = dfr().reproject_backward(img_d, src, tgt, to_dev(g), bbox, order, precision,
                                     want_params=False)
    gs = gs.cpu().numpy()
    x, y = cr[..., 0].ravel(), cr[..., 1].ravel()
    ok = np.isfinite(x)
    ref = OI.interpolate_adjoint(img.shape, np.where(ok, x, np.nan), np.where(ok, y, np.nan),
                                 OR.ORDERS[order], g.ravel(), valid=ok,
                                 use_snap=(precision == "fp64"))
    assert np.abs(gs - ref).max() <= 1e-5 * np.abs(ref).max()
    # per element: FP32 rounding of each sum (relative) plus a floor for sums that cancel
    assert np.all(np.abs(gs - ref) <= 1e-5 * np.abs(ref) + 1e-6 * np.abs(ref).max())
    # dot-product test of the GPU pair
    s = synth.rng_for(10).standard_normal((n, n)).astype(np.float32)
    ws, _ = dfr().reproject(to_dev(s), src, tgt, bbox=bbox, order=order, precision=precision)
    lhs = float(np.dot(ws.cpu().numpy().ravel().astype(np.float64), g.ravel()))
    rhs = float(np.dot(s.ravel().astype(np.float64), gs.ravel()))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1.0) * 10


@pytest.mark.parametrize("order", ["bilinear", "bicubic", "lanczos3"])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_param_gradients_match_dual_numbers(order, precision):
    src, tgt, img, ref = _case(order=order)
    n = 256
    bbox = (0, 0, n, n)
    # oracle: O(theta) in FP64 and its forward-mode derivative; grad_out = 2 (O - ref)
    Y, X = np.mgrid[0:n, 0:n].astype(np.float64)
    o, names = OD.reproject_dual(src, tgt, img, X.ravel(), Y.ravel(), order)
    r = o.v - ref.ravel()
    g_ref = (2.0 * r * o.d).sum(axis=1)
    go = (2.0 * r).reshape(n, n).astype(np.float32)
    _, gp = dfr().reproject_backward(to_dev(img), src, tgt, to_dev(go), bbox, order, precision,
                                     exact_inverse=True, want_src=False)
    torch().cuda.synchronize()
    dfr().device_status()
    gp = gp.cpu().numpy()
    assert gp.shape == g_ref.shape
    _group_check(gp, g_ref, names)


def test_param_gradients_poly_inverse_has_zero_sip_terms():
    src, tgt, img, _ = _case()
    go = np.ones((256, 256), np.float32)
    _, gp = dfr().reproject_backward(to_dev(img), src, tgt, to_dev(go), (0, 0, 256, 256),
                                     "bilinear", "split", exact_inverse=False, want_src=False)
    gp = gp.cpu().numpy()
    assert np.all(gp[6:] == 0.0) and np.any(gp[:6] != 0.0)


def test_grad_deterministic_and_empty():
    src, tgt, img, ref = _case()
    g = synth.rng_for(3).standard_normal((256, 256)).astype(np.float32)
    a = dfr().reproject_backward(to_dev(img), src, tgt, to_dev(g), (0, 0, 256, 256),
                                 "bicubic", "split", exact_inverse=True)[1].cpu().numpy()
    b = dfr().reproject_backward(to_dev(img), src, tgt, to_dev(g), (0, 0, 256, 256),
                                 "bicubic", "split", exact_inverse=True)[1].cpu().numpy()
    assert np.array_equal(a, b)
    gs, gp = dfr().reproject_backward(to_dev(img), src, tgt, to_dev(g[:1, :1]), (0, 0, 0, 0),
                                      "bilinear", "split")
    assert float(gs.abs().sum()) == 0.0 and float(gp.abs().sum()) == 0.0


def test_config3_window_gradients():
    """2048^2 TAN-SIP 3 differentiation case: gradients of L over a 384x384 window of the target
    (full-size source and WCS), Newton inverse, bilinear, against the oracle's dual numbers."""
    c = synth.config3()
    src = c["src"][0]
    src, _ = OW.with_inverse_sip(src, 4)
    pert = synth.copy_wcs(c["perturbed"])
    pert["ap"], pert["bp"], pert["ap_order"], pert["bp_order"] = src["ap"], src["bp"], 4, 4
    tgt, img = c["tgt"], c["images"][0]
    bbox = (1400, 300, 384, 384)
    ref, _, _, _ = OR.reproject(pert, tgt, img, "bilinear", bbox=bbox, inverse="newton")
    loss, g_ref, names = OD.loss_grad(src, tgt, img, ref, "bilinear", bbox=bbox)
    x0, y0, w, h = bbox
    Y, X = np.mgrid[y0:y0 + h, x0:x0 + w].astype(np.float64)
    o, _ = OD.reproject_dual(src, tgt, img, X.ravel(), Y.ravel(), "bilinear")
    go = (2.0 * (o.v - ref.ravel())).reshape(h, w).astype(np.float32)
    for precision in ("fp64", "split"):
        _, gp = dfr().reproject_backward(to_dev(img), src, tgt, to_dev(go), bbox, "bilinear",
                                         precision, exact_inverse=True, want_src=False)
        _group_check(gp.cpu().numpy(), g_ref, names)


@pytest.mark.parametrize("order,precision,exact", [("bilinear", "split", False),
                                                   ("bicubic", "split", True),
                                                   ("bicubic", "fp64", False),
                                                   ("lanczos3", "split", False)])
def test_backward_batch_equals_single_calls(order, precision, exact):
    """dfr_reproject_backward_batch over frames of uneven sizes, rotations and boxes (one of them
    empty, one sharing another's grad_src) against one dfr_reproject_backward call per frame:
    grad_params bit for bit, grad_src to float-atomic ordering (1e-6 of its scale)."""
    rng = synth.rng_for(31)
    tgt = synth.tan_wcs(600, 520, rho_deg=1.5, crpix=(300.5, 260.5))
    specs = [(300, 220, 0.0, (7, 3, 291, 237)), (420, 380, 2.0, None), (128, 96, -1.0, None),
             (256, 256, 0.5, (0, 0, 0, 0)), (300, 220, 0.0, (40, 60, 200, 180))]
    srcs, imgs, boxes, gos = [], [], [], []
    for k, (w, h, rho, bb) in enumerate(specs):
        s = synth.add_sip(synth.tan_wcs(w, h, rho_deg=rho), 3, 1e-6, rng)
        s["a"] *= 50.0
        s["b"] *= 50.0
        s, _ = OW.with_inverse_sip(s, 4)
        if k == 4:  # frame 4 reprojects frame 0's image with frame 0's WCS over another box
            s = srcs[0]
        srcs.append(s)
        imgs.append(imgs[0] if k == 4 else to_dev(synth.sky_image(w, h, 20, rng)))
        box = bb if bb is not None else dfr().target_bbox(s, tgt)
        boxes.append(box)
        gos.append(to_dev(synth.rng_for(40 + k).standard_normal((max(box[3], 1),
                                                                   max(box[2], 1)))
                          .astype(np.float32)))
    T = torch()
    gs_b = [T.zeros_like(i) for i in imgs]
    gs_b[4] = gs_b[0]  # shared: frames 0 and 4 add into one buffer
    gs_b, gp_b = dfr().reproject_backward_batch(imgs, srcs, tgt, gos, boxes, order, precision,
                                                exact_inverse=exact, grad_srcs=gs_b)
    T.cuda.synchronize()
    dfr().device_status()
    gs_s = [T.zeros_like(i) for i in imgs]
    gs_s[4] = gs_s[0]
    gp_s = []
    for k in range(len(imgs)):
        _, gp = dfr().reproject_backward(imgs[k], srcs[k], tgt, gos[k], boxes[k], order,
                                         precision, exact_inverse=exact, grad_src=gs_s[k])
        gp_s.append(gp)
    T.cuda.synchronize()
    for k in range(len(imgs)):
        assert T.equal(gp_b[k], gp_s[k]), k
        a, b = gs_b[k].cpu().numpy(), gs_s[k].cpu().numpy()
        scale = np.abs(b).max()
        if k == 3:  # the empty box: nothing scattered, parameters zero
            assert scale == 0.0 and float(gp_b[k].abs().sum()) == 0.0
            continue
        assert scale > 0
        assert np.abs(a - b).max() <= 1e-6 * scale, k


def test_config3_whole_frame_sampled_gradients():
    """The 2048^2 differentiation case over the whole frame: the loss gradient of a seeded 1 %
    sample of the target pixels (grad_out = 2 (O - ref) there, zero elsewhere, so the launch
    covers every cell of the frame), against the oracle's dual numbers summed over the same
    pixels (CRVAL, CD and the 18 SIP terms, Newton inverse)."""
    c = synth.config3()
    src = c["src"][0]
    src, _ = OW.with_inverse_sip(src, 4)
    pert = synth.copy_wcs(c["perturbed"])
    pert["ap"], pert["bp"], pert["ap_order"], pert["bp_order"] = src["ap"], src["bp"], 4, 4
    tgt, img = c["tgt"], c["images"][0]
    n = 2048
    rng = synth.rng_for(303)
    idx = rng.choice(n * n, n * n // 100, replace=False)
    X = (idx % n).astype(np.float64)
    Y = (idx // n).astype(np.float64)
    # Bilinear interpolation has kinks on the integer lines of the source grid, where its
    # derivative jumps: a pixel whose position lies within the split path's position error of
    # such a line may take the slope of the other side (both are derivatives of the same
    # continuous output). Such pixels (1e-4 px margin, about 4e-4 of the sample) are left out.
    sx, sy, _ = OR.coords(src, tgt, X, Y, inverse="newton")
    far = (np.abs(sx - np.rint(sx)) > 1e-4) & (np.abs(sy - np.rint(sy)) > 1e-4)
    idx, X, Y = idx[far], X[far], Y[far]
    ref, _, _, _ = OR.reproject_pixels(pert, tgt, img, X, Y, "bilinear", inverse="newton")
    o, names = OD.reproject_dual(src, tgt, img, X, Y, "bilinear")
    r = o.v - ref
    g_ref = (2.0 * r * o.d).sum(axis=1)
    go = np.zeros(n * n, np.float32)
    go[idx] = (2.0 * r).astype(np.float32)
    go = go.reshape(n, n)
    for precision in ("fp64", "split"):
        _, gp = dfr().reproject_backward(to_dev(img), src, tgt, to_dev(go), (0, 0, n, n),
                                         "bilinear", precision, exact_inverse=True,
                                         want_src=False)
        torch().cuda.synchronize()
        dfr().device_status()
        _group_check(gp.cpu().numpy(), g_ref, names)


def test_autograd_alignment_descent():
    """torch.autograd through dfr: fitting CRVAL by gradient descent recovers a 0.3 arcsec
    offset of the reference image."""
    T = torch()
    src, tgt, img, _ = _case(n=256, boost=1.0)
    truth = synth.copy_wcs(src)
    truth["crval"] = (src["crval"][0] + 0.3 / 3600, src["crval"][1] - 0.2 / 3600)
    img_d = to_dev(img)
    target_img, _ = dfr().reproject(img_d, truth, tgt, order="bicubic", precision="split",
                                    exact_inverse=True)
    theta0 = dfr().param_vector(src)
    theta = T.tensor(theta0, dtype=T.float64, device="cuda", requires_grad=True)
    bbox = (0, 0, 256, 256)
    scale = T.zeros_like(theta)
    scale[:2] = 1.0 / 3600  # optimise CRVAL only, in arcsec units
    losses = []
    for it in range(60):
        out = dfr().Reproject.apply(img_d, theta, src, tgt, bbox, "bicubic", "split", True)
        loss = ((out - target_img) ** 2).sum()
        theta.grad = None
        loss.backward()
        with T.no_grad():
            g = theta.grad * scale
            step = 0.05 * 0.93 ** it  # arcsec, decaying
            theta -= step * g * scale / max(float(g.abs().max()), 1e-30)
        losses.append(float(loss.detach()))
    err = (theta.detach().cpu().numpy()[:2] - np.array(truth["crval"])) * 3600
    assert losses[-1] < 0.05 * losses[0]
    assert np.all(np.abs(err) < 0.02)


@pytest.mark.parametrize("order", ["nearest", "bilinear", "bicubic"])
@pytest.mark.parametrize("exact", [False, True])
def test_staged_adjoint_matches_per_pixel_kernel(order, exact):
    """The tile-staged split adjoint (TMA source boxes, shared-memory gradient boxes, per-lane
    parameter accumulators) against the per-pixel split adjoint on a ragged bounding box that
    runs off the source (partial tiles, masked taps, pixels outside the footprint)."""
    rng = synth.rng_for(21)
    src = synth.add_sip(synth.tan_wcs(300, 220), 3, 1e-6, rng)
    src["a"] *= 100.0
    src["b"] *= 100.0
    src, _ = OW.with_inverse_sip(src, 4)
    tgt = synth.tan_wcs(340, 260, rho_deg=2.0, crpix=(190.5, 120.5))
    img = synth.sky_image(300, 220, 30, rng)
    bbox = (7, 3, 291, 237)
    x0, y0, w, h = bbox
    g = synth.rng_for(22).standard_normal((h, w)).astype(np.float32)
    img_d, g_d = to_dev(img), to_dev(g)
    gs_a, gp_a = dfr().reproject_backward(img_d, src, tgt, g_d, bbox, order, "split",
                                          exact_inverse=exact)
    gs_b, gp_b = dfr().reproject_backward(img_d, src, tgt, g_d, bbox, order, "split",
                                          exact_inverse=exact, tma=False)
    torch().cuda.synchronize()
    dfr().device_status()
    gs_a, gs_b = gs_a.cpu().numpy(), gs_b.cpu().numpy()
    assert np.abs(gs_b).max() > 0
    assert np.abs(gs_a - gs_b).max() <= 1e-6 * np.abs(gs_b).max()
    gp_a, gp_b = gp_a.cpu().numpy(), gp_b.cpu().numpy()
    if order == "nearest":
        assert np.all(gp_a == 0.0) and np.all(gp_b == 0.0)
        return
    scale = np.abs(gp_b).max()
    assert scale > 0
    assert np.abs(gp_a - gp_b).max() <= 1e-5 * scale
