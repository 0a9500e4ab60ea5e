"""A bounded wait that runs out, on the GPU (the failure-handling path of the split kernels).

A child process sets DFR_FAULT_TX_EXTRA, so every source-box load of a single-frame split launch
expects 16 bytes more than its copy delivers: the copy completes (nothing writes late) but its
barrier phase never does, and each warp's wait gives up after its time limit. The kernel then
sets the device status word, stops issuing box loads, gathers from global memory and, before it
exits, waits (bounded) for its copies. The test checks that dfr_device_status reports
DFR_ERR_TIMEOUT once (and is clear afterwards) and that value and footprint equal, bit for bit,
those of the launch without TMA staging. Small frame: one wave of CTAs, a few seconds."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, %r)
import numpy as np, torch
import synth
from oracle import wcs as OW
import paper_2505_03932_gb300 as dfr
rng = synth.rng_for(91)
src = synth.add_sip(synth.tan_wcs(160, 120), 3, 1e-6, rng)
src, _ = OW.with_inverse_sip(src, 4)
tgt = synth.tan_wcs(150, 130, rho_deg=0.7, crpix=(src["crpix"][0] + 3.3, src["crpix"][1] - 2.1))
img = torch.from_numpy(synth.sky_image(160, 120, 20, rng)).cuda()
res = {}
v, f = dfr.reproject(img, src, tgt, order="bicubic", precision="split")
torch.cuda.synchronize()
try:
    dfr.device_status()
    res["status"] = 0
except dfr.DfrError as e:
    res["status"] = e.code
try:
    dfr.device_status()
    res["status_after"] = 0
except dfr.DfrError as e:
    res["status_after"] = e.code
v0, f0 = dfr.reproject(img, src, tgt, order="bicubic", precision="split", tma=False)
torch.cuda.synchronize()
dfr.device_status()
res["value_equal"] = bool(torch.equal(v, v0))
res["footprint_equal"] = bool(torch.equal(f, f0))
res["covered"] = float((f0 > 0).float().mean())
print(json.dumps(res))
""" % ROOT


def test_wait_that_runs_out_reports_timeout_and_falls_back():
    env = dict(os.environ, DFR_FAULT_TX_EXTRA="16")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["status"] == -7, res  # DFR_ERR_TIMEOUT
    assert res["status_after"] == 0, res
    assert res["value_equal"] and res["footprint_equal"], res
    assert res["covered"] > 0.5
