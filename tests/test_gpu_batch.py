"""GPU batch path (dfr_reproject_batch): the frame-table kernel, CUDA graph replay and autotuned tiles
give exactly the bits of per-frame dfr_reproject calls with the same bounding boxes; sampled
oracle parity at the full 64-frame / 8192^2 batch size."""
import numpy as np
import pytest

import synth
from oracle import wcs as OW

from gpu_util import SPLIT_PX, VALUE_RTOL, coord_check, dfr, gpu, to_dev, torch, value_check

pytestmark = pytest.mark.gpu


def _frames(n=5, seed=21):
    rng = synth.rng_for(seed)
    tgt = synth.tan_wcs(1100, 900, crpix=(550.5, 450.5))
    shapes = [(300, 200), (517, 433), (129, 700), (64, 64), (401, 377)][:n]
    srcs, imgs = [], []
    for k, (w, h) in enumerate(shapes):
        dx, dy = rng.uniform(-50, 50, 2)
        s = synth.tan_wcs(w, h, rho_deg=rng.uniform(-2, 2),
                          crpix=((w + 1) / 2 + dx + 120 * (k - 2), (h + 1) / 2 + dy))
        s = synth.add_sip(s, 3, 1e-6, rng)
        s, _ = OW.with_inverse_sip(s, 4)
        srcs.append(s)
        imgs.append(synth.sky_image(w, h, synth.sources_for_area(w, h, 4000), rng))
    # one frame entirely off the target grid
    off = synth.tan_wcs(50, 50, crval=(151.0, 2.0))
    srcs.insert(2, off)
    imgs.insert(2, np.zeros((50, 50), np.float32))
    return srcs, imgs, tgt


@pytest.mark.parametrize("order", ["nearest", "bilinear", "bicubic", "lanczos3", "bspline3"])
@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_batch_equals_single_bitwise(order, precision):
    srcs, imgs, tgt = _frames()
    imgs_d = [to_dev(i) for i in imgs]
    bbs = [dfr().target_bbox(s, tgt) for s in srcs]
    assert bbs[2] == (0, 0, 0, 0)
    vals, fps = dfr().reproject_batch(imgs_d, srcs, tgt, bbs, order=order, precision=precision)
    torch().cuda.synchronize()
    dfr().device_status()
    for k, (s, bb) in enumerate(zip(srcs, bbs)):
        if bb[2] == 0:
            continue
        v, f = dfr().reproject(imgs_d[k], s, tgt, bbox=bb, order=order, precision=precision)
        assert np.array_equal(vals[k].cpu().numpy(), v.cpu().numpy()), k
        assert np.array_equal(fps[k].cpu().numpy(), f.cpu().numpy()), k


def test_graph_replay_follows_new_inputs():
    srcs, imgs, tgt = _frames()
    bbs = [dfr().target_bbox(s, tgt) for s in srcs]
    a_imgs = [to_dev(i) for i in imgs]
    b_imgs = [to_dev(2.0 * i + 1.0) for i in imgs]
    va, _ = dfr().reproject_batch(a_imgs, srcs, tgt, bbs, order="bilinear")
    vb, _ = dfr().reproject_batch(b_imgs, srcs, tgt, bbs, order="bilinear")
    va2, _ = dfr().reproject_batch(a_imgs, srcs, tgt, bbs, order="bilinear")
    torch().cuda.synchronize()
    for k, bb in enumerate(bbs):
        if bb[2] == 0:
            continue
        a, b, a2 = va[k].cpu().numpy(), vb[k].cpu().numpy(), va2[k].cpu().numpy()
        assert np.array_equal(a, a2)
        v, _ = dfr().reproject(b_imgs[k], srcs[k], tgt, bbox=bb, order="bilinear")
        assert np.array_equal(b, v.cpu().numpy())


def test_batch_frames_match_oracle():
    srcs, imgs, tgt = _frames()
    bbs = [dfr().target_bbox(s, tgt) for s in srcs]
    for k in (0, 3, 5):
        val, fp, cr = gpu(srcs[k], tgt, to_dev(imgs[k]), "bilinear", "split", bbs[k])
        dmax, _ = coord_check(srcs[k], tgt, cr, bbs[k])
        assert dmax < SPLIT_PX
        e, fe = value_check(imgs[k], "bilinear", val, fp, cr, "split")
        assert e <= VALUE_RTOL and fe <= 1e-6


def test_config2_full_batch_sampled():
    """64 exposures (2048-6144 px sides) onto 8192^2 in one persistent graph launch. Every frame
    equals its single-frame call on the same box bit for bit, and 2000 sampled pixels per frame
    match the oracle (coordinates within 1e-3 px, values at the GPU coordinates within 1e-5)."""
    T = torch()
    c = synth.config2()
    tgt = c["tgt"]
    srcs = [OW.with_inverse_sip(s, 4)[0] for s in c["src"]]
    imgs_d = [to_dev(i) for i in c["images"]]
    bbs = [dfr().target_bbox(s, tgt) for s in srcs]
    vals, fps = dfr().reproject_batch(imgs_d, srcs, tgt, bbs, order="bilinear")
    T.cuda.synchronize()
    dfr().device_status()
    rng = synth.rng_for(8)
    for k in range(64):
        x0, y0, w, h = bbs[k]
        v, f, cr = dfr().reproject(imgs_d[k], srcs[k], tgt, bbox=bbs[k], order="bilinear",
                                   precision="split", coords=True)
        assert T.equal(vals[k], v) and T.equal(fps[k], f), k
        iy = T.from_numpy(rng.integers(0, h, 2000)).cuda()
        ix = T.from_numpy(rng.integers(0, w, 2000)).cuda()
        crs = cr[iy, ix].cpu().numpy()[None]
        e, fe = value_check(c["images"][k], "bilinear", v[iy, ix].cpu().numpy()[None],
                            f[iy, ix].cpu().numpy()[None], crs, "split")
        assert e <= VALUE_RTOL and fe <= 1e-6
        from oracle import reproject as OR
        ox, oy, ok = OR.coords(srcs[k], tgt, ix.cpu().numpy() + x0, iy.cpu().numpy() + y0)
        d = np.hypot(crs[0, :, 0] - ox, crs[0, :, 1] - oy)[ok]
        assert d.max() < SPLIT_PX
        del v, f, cr
    del imgs_d, vals, fps


_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import test_gpu_batch as T
from gpu_util import dfr, to_dev, torch
tma = sys.argv[2] == "1"
srcs, imgs, tgt = T._frames()
imgs_d = [to_dev(i) for i in imgs]
bbs = [dfr().target_bbox(s, tgt) for s in srcs]
bad = []
for order in ("bilinear", "bicubic", "lanczos3"):
    vals, fps = dfr().reproject_batch(imgs_d, srcs, tgt, bbs, order=order, tma=tma)
    torch().cuda.synchronize()
    cfg = dfr().last_launch_config()["batch"]
    for k, (s, bb) in enumerate(zip(srcs, bbs)):
        if bb[2] == 0:
            continue
        v, f = dfr().reproject(imgs_d[k], s, tgt, bbox=bb, order=order, tma=tma)
        if not (np.array_equal(vals[k].cpu().numpy(), v.cpu().numpy()) and
                np.array_equal(fps[k].cpu().numpy(), f.cpu().numpy())):
            bad.append((order, k))
dfr().device_status()
print(json.dumps({"cfg": cfg, "bad": bad}))
"""


@pytest.mark.parametrize("form", ["graph", "table"])
@pytest.mark.parametrize("th", [8, 16, 32])
@pytest.mark.parametrize("tma", [True, False])
def test_batch_every_tuned_shape_bitwise(form, th, tma):
    """Every configuration the batch autotuner can pick (launch form, tile height of the staged
    boxes, box staging on or off), pinned in a child process through DFR_BATCH_FORM and
    DFR_TILE_H: the batch gives the bits of per-frame calls."""
    import json
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, DFR_BATCH_FORM=form, DFR_TILE_H=str(th))
    r = subprocess.run([sys.executable, "-c", _CHILD, here, "1" if tma else "0"], env=env,
                       capture_output=True, text=True, timeout=600,
                       cwd=os.path.dirname(here))
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["bad"] == []
    assert out["cfg"]["tile_h"] == th
    assert out["cfg"]["form"] == form
