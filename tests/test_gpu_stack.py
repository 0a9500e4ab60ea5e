"""Stack-scale run (32 exposures of 6000x4000, TAN-SIP order 5 with AP/BP order 6, dithers up to
200 px, rotations up to 3 deg, bicubic onto a 12000x8000 target): one split-precision batch
launch, then the adjoint of every frame in a second pass.

Checks: batch output equals the single-frame call on the same box bit for bit (every frame);
on a seeded random sample of each frame's covered pixels the source positions are within 1e-3 px
of the FP64 oracle (max and RMS printed) and the values at the GPU's coordinates within 1e-5
relative; the backward pass gives finite gradients whose source part passes the dot-product
test against the forward on one frame."""
import numpy as np
import pytest

import synth
from oracle import reproject as OR
from oracle import wcs as OW

from gpu_util import SPLIT_PX, VALUE_RTOL, dfr, to_dev, torch, value_check

pytestmark = pytest.mark.gpu


def test_config4_stack_forward_and_adjoint():
    T = torch()
    c = synth.config4()
    tgt = c["tgt"]
    srcs = [OW.with_inverse_sip(s, 6)[0] for s in c["src"]]
    imgs_d = [to_dev(i) for i in c["images"]]
    bbs = [dfr().target_bbox(s, tgt) for s in srcs]
    vals, fps = dfr().reproject_batch(imgs_d, srcs, tgt, bbs, order="bicubic")
    T.cuda.synchronize()
    dfr().device_status()
    rng = synth.rng_for(404)
    worst, sq, cnt = 0.0, 0.0, 0
    for k in range(32):
        x0, y0, w, h = bbs[k]
        v, f, cr = dfr().reproject(imgs_d[k], srcs[k], tgt, bbox=bbs[k], order="bicubic",
                                   precision="split", coords=True)
        assert T.equal(vals[k], v) and T.equal(fps[k], f), k
        cov = T.nonzero(f.reshape(-1) > 0).reshape(-1)
        pick = cov[T.from_numpy(rng.integers(0, cov.numel(), 4000)).cuda()]
        iy, ix = pick // w, pick % w
        crs = cr[iy, ix].cpu().numpy()[None]
        e, fe = value_check(c["images"][k], "bicubic", v[iy, ix].cpu().numpy()[None],
                            f[iy, ix].cpu().numpy()[None], crs, "split")
        assert e <= VALUE_RTOL and fe <= 1e-6
        ox, oy, ok = OR.coords(srcs[k], tgt, ix.cpu().numpy() + x0, iy.cpu().numpy() + y0)
        d = np.hypot(crs[0, :, 0] - ox, crs[0, :, 1] - oy)[ok]
        worst = max(worst, float(d.max()))
        sq += float(np.sum(d * d))
        cnt += d.size
        del v, f, cr
    print("config4 split coordinate error vs oracle: max %.3g px, rms %.3g px over %d pixels"
          % (worst, (sq / cnt) ** 0.5, cnt))
    assert worst < SPLIT_PX
    # second pass: adjoint of every frame with grad_out ~ N(0, 1)
    g = T.randn((max(b[3] for b in bbs), max(b[2] for b in bbs)), device="cuda",
                generator=T.Generator("cuda").manual_seed(7))
    for k in range(32):
        x0, y0, w, h = bbs[k]
        gs, gp = dfr().reproject_backward(imgs_d[k], srcs[k], tgt, g[:h, :w], bbs[k], "bicubic",
                                          "split")
        assert bool(T.isfinite(gs).all()) and bool(T.isfinite(gp).all())
        if k == 0:
            s = T.randn_like(imgs_d[0])
            ws, _ = dfr().reproject(s, srcs[0], tgt, bbox=bbs[0], order="bicubic")
            lhs = float((ws.double() * g[:h, :w].double()).sum())
            rhs = float((s.double() * gs.double()).sum())
            assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), 1.0)
    T.cuda.synchronize()
    dfr().device_status()
