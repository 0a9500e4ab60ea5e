"""dfr_reproject_batch_noalloc through the C ABI: the batched reprojection for callers that
cannot allocate device memory (it keeps its frame table in a fixed library-owned device array
instead of calling cudaMalloc). Its output must equal dfr_reproject_batch's bit for bit, as its
declaration promises, on two calls in a row (the second call reuses the array that the first
one left behind), for both precisions, with and without TMA staging. This file is collected
last on purpose."""
import pytest

import synth
from oracle import wcs as OW

pytestmark = pytest.mark.gpu



def _inputs(seed):
    rng = synth.rng_for(seed)
    tgt = synth.tan_wcs(900, 700, crpix=(450.5, 350.5))
    srcs, imgs = [], []
    for k, (w, h) in enumerate([(300, 210), (257, 333), (64, 48), (420, 380)]):
        dx, dy = rng.uniform(-40, 40, 2)
        s = synth.tan_wcs(w, h, rho_deg=rng.uniform(-2, 2),
                          crpix=((w + 1) / 2 + dx + 90 * (k - 1), (h + 1) / 2 + dy))
        s = synth.add_sip(s, 3, 1e-6, rng)
        s, _ = OW.with_inverse_sip(s, 4)
        srcs.append(s)
        imgs.append(synth.sky_image(w, h, 10, rng))
    return srcs, imgs, tgt


@pytest.mark.parametrize("tma", [True, False])
@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_noalloc_batch_matches_batch_twice(precision, tma):
    import torch
    import paper_2505_03932_gb300 as dfr

    for call, seed in enumerate((61, 62)):
        srcs, imgs, tgt = _inputs(seed)
        imgs_d = [torch.from_numpy(i).cuda() for i in imgs]
        bbs = [dfr.target_bbox(s, tgt) for s in srcs]
        for order in ("bilinear", "bicubic"):
            ref_v, ref_f = dfr.reproject_batch(imgs_d, srcs, tgt, bbs, order=order,
                                               precision=precision, tma=tma)
            outs = [torch.full((bb[3], bb[2]), -1.0, device="cuda") for bb in bbs]
            fps = [torch.full((bb[3], bb[2]), -1.0, device="cuda") for bb in bbs]
            dfr.reproject_batch_noalloc(imgs_d, srcs, tgt, bbs, outs, fps, order=order,
                                        precision=precision, tma=tma)
            torch.cuda.synchronize()
            dfr.device_status()
            for k in range(len(srcs)):
                assert torch.equal(outs[k], ref_v[k]), (call, order, k)
                assert torch.equal(fps[k], ref_f[k]), (call, order, k)


def test_noalloc_rejects_more_than_64_frames():
    import torch
    import paper_2505_03932_gb300 as dfr

    srcs, imgs, tgt = _inputs(63)
    img = torch.from_numpy(imgs[0]).cuda()
    bb = dfr.target_bbox(srcs[0], tgt)
    out = torch.zeros((bb[3], bb[2]), device="cuda")
    with pytest.raises(dfr.DfrError) as ei:
        dfr.reproject_batch_noalloc([img] * 65, [srcs[0]] * 65, tgt, [bb] * 65, [out] * 65)
    assert ei.value.code == -1 and "64" in str(ei.value)
