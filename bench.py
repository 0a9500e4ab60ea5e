#!/usr/bin/env python3
"""Benchmark: output Mpix/s of TAN-SIP reprojection on GB300 (one JSON line on rank 0).

Workload (the bench step): one 4096x4096 float32 exposure, TAN-SIP order 3 with AP/BP order 4
(fitted by the library), reprojected with bicubic interpolation onto a 4096x4096 TAN target
rotated 1.2 deg, offset (41.3, -17.9) px, 1% larger pixels; split precision (the sky rotation at
one anchor per 32x32 cell in double-float arithmetic, FP32 per pixel); value and footprint
written. One step = one fused launch
over the whole frame. Inputs are synthetic (seeded sky noise + 2000 Gaussian stars).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the launching
stream, with a 512 MB write between steps to flush the 129 MB L2 (the flush is outside the
events); barrier + synchronize around the timed loop; max over ranks. The reference arm
(--impl reference) times the FP64 CPU oracle on a bounded pixel sample of the same workload, on
every host core (one spawned process per core, at most 32).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "output Mpix/s (bicubic, TAN-SIP) split-precision vs all-FP64 at 1e-3 px; % roofline"
WORKLOAD = "4096x4096 TAN-SIP3 (AP/BP 4) -> 4096x4096 TAN, rot 1.2 deg, +1% scale, bicubic"
BYTES_PER_PIX = 12  # 4 B source read + 4 B value + 4 B footprint written


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler (every 200 ms) for the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[2 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _code_of(path):
    """A source file without its comments and blank lines: a change of comments alone leaves
    the compiled kernel, and so a recorded capture of it, valid."""
    import re
    text = open(path, encoding="utf-8").read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", line).rstrip() for line in text.splitlines()]
    return "\n".join(line for line in lines if line.strip()).encode()


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("dfr_fwd.cu", "dfr_fwd_kernels.cuh", "dfr_tile.cuh", "dfr_device.cuh",
              "dfr_internal.h"):
        h.update(_code_of(os.path.join(ROOT, "paper_2505_03932_gb300", "csrc", f)))
    return h.hexdigest()


def _recorded():
    """Counters of the bench kernel from the committed ncu summary (key: value lines), or {} when
    the kernel source has changed since those counters were taken."""
    path = os.path.join(ROOT, "profiles", "split_bicubic_4096.md")
    try:
        rec = {}
        for line in open(path):
            k, sep, v = line.partition(":")
            if sep and k in ("traffic_bytes_per_launch", "kernel_source_sha256",
                             "issue_ipc", "instructions_per_pixel"):
                rec[k] = v.strip()
        if rec.get("kernel_source_sha256") == kernel_source_hash():
            return rec
    except Exception:
        pass
    return {}


def recorded_fp64():
    """FP64 flops per output pixel of the all-FP64 kernel (ncu SASS counts: 2 per DFMA, 1 per
    DADD and DMUL) from the committed summary, or None when the FP64 kernel changed since."""
    path = os.path.join(ROOT, "profiles", "fp64_bicubic_4096.md")
    try:
        rec = {}
        for line in open(path):
            k, sep, v = line.partition(":")
            if sep and k in ("fp64_flops_per_pixel", "fp64_source_sha256"):
                rec[k] = v.strip()
        if rec.get("fp64_source_sha256") == fp64_source_hash():
            return float(rec["fp64_flops_per_pixel"])
    except Exception:
        pass
    return None


def fp64_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("dfr_fwd_kernels.cuh", "dfr_device.cuh"):
        h.update(_code_of(os.path.join(ROOT, "paper_2505_03932_gb300", "csrc", f)))
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes per launch of the bench kernel (ncu), or None (kernel changed since)."""
    rec = _recorded()
    return int(rec["traffic_bytes_per_launch"]) if "traffic_bytes_per_launch" in rec else None


def recorded_issue():
    """The bench kernel's instruction issue rate from the same capture: the kernel is bound by
    instruction issue (4 per SM per cycle), not by HBM; None when the kernel changed since."""
    rec = _recorded()
    if "issue_ipc" not in rec:
        return None
    ipc = float(rec["issue_ipc"])
    return {"ipc": ipc, "peak_ipc": 4.0, "frac": ipc / 4.0,
            "instructions_per_pixel": float(rec["instructions_per_pixel"]), "source": "ncu"}


def workload():
    c = synth.config1()
    return c["src"][0], c["tgt"], c["images"][0]


# ------------------------------------------------------------------------------ reference arm
def oracle_sample_rate(src, tgt, img, npix, seed=7):
    """Run the FP64 CPU oracle on npix random target pixels; returns seconds."""
    from oracle import reproject as OR
    rng = synth.rng_for(seed)
    X = rng.integers(0, tgt["naxis"][0], npix).astype(np.float64)
    Y = rng.integers(0, tgt["naxis"][1], npix).astype(np.float64)
    t0 = time.perf_counter()
    OR.reproject_pixels(src, tgt, img, X, Y, "bicubic", inverse="poly")
    return time.perf_counter() - t0


def oracle_wcs(src):
    from oracle import wcs as OW
    w, _ = OW.with_inverse_sip(src, 4)
    return w


_WORKER = {}


def _oracle_worker_init(barrier):
    """Pool initializer: each worker builds the seeded workload itself (about 1 s), then waits
    until every worker has, so that no start-up time falls inside a timed map."""
    src, tgt, img = workload()
    _WORKER["args"] = (oracle_wcs(src), tgt, img)
    barrier.wait(timeout=600)


def _oracle_worker_run(task):
    npix, seed = task
    return oracle_sample_rate(*_WORKER["args"], npix, seed=seed)


class OraclePool:
    """The oracle run on every host core: one spawned process per core, each evaluating its own
    share of random target pixels (rows of work split statically, like OpenMP static rows)."""

    def __init__(self):
        import multiprocessing as mp
        # every host core, up to 32 processes (each holds the 64 MB frame and ~0.3 GB of
        # oracle temporaries)
        self.cores = min(len(os.sched_getaffinity(0)), 32)
        ctx = mp.get_context("spawn")
        # one thread per worker process: the workers inherit these at spawn
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update({k: "1" for k in saved})
        try:
            self.pool = ctx.Pool(self.cores, initializer=_oracle_worker_init,
                                 initargs=(ctx.Barrier(self.cores),))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        # returns once every worker is past the barrier (bounded: a worker that fails to start
        # is replaced by the pool and would otherwise leave the map waiting)
        self._map([(1000, k) for k in range(self.cores)], timeout=600)

    def _map(self, tasks, timeout):
        return self.pool.map_async(_oracle_worker_run, tasks, chunksize=1).get(timeout=timeout)

    def seconds(self, npix_per_core, seed):
        """Wall seconds for cores x npix_per_core pixels."""
        tasks = [(npix_per_core, seed * 1000 + k) for k in range(self.cores)]
        t0 = time.perf_counter()
        self._map(tasks, timeout=600)
        return time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()


def run_reference(args, rank, world):
    if rank != 0:
        return
    pool = OraclePool()
    try:
        # at most about 0.25 s of each core per step, and about 10 s of each core over all
        # the timed steps (a long timed run takes smaller samples per step)
        per_core = int(min(250_000, max(2_000, 10_000_000 // max(1, args.steps))))
        for k in range(args.warmup):
            pool.seconds(per_core // 4, seed=1 + k)
        secs = [pool.seconds(per_core, seed=100 + k) for k in range(args.steps)]
    finally:
        pool.close()
    npix = per_core * pool.cores
    t = float(np.mean(secs))
    mpix = npix / t / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": mpix, "unit": "Mpix/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_pixels_per_step": npix},
        "cpu_baseline": {"value": mpix, "unit": "Mpix/s", "cores": pool.cores, "kind": "oracle",
                         "sample": "%d random target pixels of the 4096^2 frame per step, "
                                   "%d per core" % (npix, per_core)},
        "e2e": {"value": mpix, "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2505_03932_gb300 as dfr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    src_rec, tgt_rec, img = workload()
    src, fit_max, fit_rms = dfr.fit_inverse_sip(src_rec, 4)
    src, tgt = dfr.to_c(src), dfr.to_c(tgt_rec)  # marshal the WCS records once
    H, W = tgt.naxis[1], tgt.naxis[0]
    npix = H * W
    img_d = torch.from_numpy(img).to(dev)
    out = torch.empty((H, W), dtype=torch.float32, device=dev)
    fpo = torch.empty_like(out)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(precision="split"):
        dfr.reproject(img_d, src, tgt, bbox=(0, 0, W, H), order="bicubic", precision=precision,
                      out=out, fp_out=fpo)

    def timed(k, precision):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        for a, b in evs:
            flush.fill_(1.0)
            a.record(stream)
            step(precision)
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    dfr.device_status()
    clocks = Clocks(local_rank)
    clocks.start()
    time.sleep(0.3)  # let the sampler start before the timed region

    def soak(seconds):
        """Back-to-back bench steps (with the flush) for about `seconds` of device time: the
        continuous load around the timed steps, so that the clock sampler sees the GPU under
        the bench's own load before, during and after them."""
        n = 0
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            for _ in range(64):
                flush.fill_(1.0)
                step()
            n += 64
            torch.cuda.synchronize()
        return n

    for _ in range(max(args.warmup, 3)):  # the GPU idled during the sleep: warm up again
        flush.fill_(1.0)
        step()
    soak_before = soak(0.6)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    times = timed(args.steps, "split")
    wall = time.perf_counter() - t0
    soak_after = soak(0.3)
    clk = clocks.stop()
    clk["window"] = ("%d steps of continuous load before and %d after the %d timed ones"
                     % (soak_before, soak_after, args.steps))
    tuned = dfr.last_launch_config()["single_tile_h"]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    dfr.device_status()
    ms = float(np.mean(times))
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())

    # the plain all-FP64 GPU path on the same workload (its own, shorter timing), and the
    # measured pipe peaks that bound it
    for _ in range(2):
        step("fp64")
    torch.cuda.synchronize()
    ms64 = float(np.mean(timed(max(3, min(args.steps, 5)), "fp64")))
    pipes = dfr.measure_pipe_peaks()
    f64 = recorded_fp64()
    fp64_roof = None
    if f64 is not None:
        ach = f64 * npix / (ms64 * 1e-3)
        fp64_roof = {"bound": "fp64", "achieved": ach / 1e12, "peak": pipes["fp64_fma_flops"] / 1e12,
                     "unit": "TFLOP/s", "frac": ach / pipes["fp64_fma_flops"],
                     "fp64_flops_per_pixel": f64, "peak_source": "measured (dfr_measure_pipe_peaks)"}

    # split vs FP64 coordinate difference over the frame (both GPU paths, FP64 emitted coords)
    _, _, c32 = dfr.reproject(img_d, src, tgt, bbox=(0, 0, W, H), order="bicubic",
                              precision="split", coords=True)
    _, _, c64 = dfr.reproject(img_d, src, tgt, bbox=(0, 0, W, H), order="bicubic",
                              precision="fp64", coords=True)
    d = torch.hypot(c32[..., 0] - c64[..., 0], c32[..., 1] - c64[..., 1])
    d = d[torch.isfinite(d)]
    dmax, drms = float(d.max()), float(torch.sqrt(torch.mean(d * d)))
    del c32, c64, d

    # end to end through the public API with pinned host buffers: H2D source, D2H result
    host_img = torch.from_numpy(img).pin_memory()
    host_out = torch.empty((H, W), dtype=torch.float32).pin_memory()
    host_fp = torch.empty((H, W), dtype=torch.float32).pin_memory()
    # (dfr_reproject_host: bands copied in, computed and copied out on overlapping streams;
    # the call returns once value and footprint are in host memory)
    e2e_steps = max(3, min(args.steps, 10))
    for k in range(e2e_steps + 2):
        if k == 2:
            torch.cuda.synchronize()
            te = time.perf_counter()
        dfr.reproject_host(host_img, src, tgt, bbox=(0, 0, W, H), order="bicubic",
                           out=host_out, fp_out=host_fp)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - te) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())

    peak, peak_src = _peaks()
    achieved = BYTES_PER_PIX * npix / (ms * 1e-3) / 1e9
    value = npix * world / (ms * 1e-3) / 1e6
    traffic = recorded_traffic()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        o_src = oracle_wcs(src_rec)
        npx1 = 3_000_000  # about 3 s of one core
        secs1 = oracle_sample_rate(o_src, tgt_rec, img, npx1)
        pool = OraclePool()
        try:
            per_core = 1_500_000  # about 1.5 s of each core
            secs = pool.seconds(per_core, seed=7)
        finally:
            pool.close()
        npx = per_core * pool.cores
        cpu = {"value": npx / secs / 1e6, "unit": "Mpix/s", "cores": pool.cores, "kind": "oracle",
               "sample": "%d random target pixels of the 4096^2 frame, %d per core (%.1f s)"
                         % (npx, per_core, secs),
               "single_core": {"value": npx1 / secs1 / 1e6, "unit": "Mpix/s",
                               "sample": "%d random target pixels (%.1f s)" % (npx1, secs1)}}

    extra = {}
    if rank == 0 and not args.no_extra:
        extra["batch64"] = measure_batch64(dfr, torch, flush, max(3, min(args.steps, 10)))
        extra["adjoint2048"] = measure_adjoint2048(dfr, torch, flush, max(3, min(args.steps, 10)))
        extra["stack32"] = measure_stack32(dfr, torch, flush, max(3, min(args.steps, 6)))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "ms_per_step_median": float(np.median(times)),
            "ms_steps_first": [round(float(t), 4) for t in times[:16]],
            "ms_steps_p10_p90": [float(np.percentile(times, 10)), float(np.percentile(times, 90))],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "split", "output_mpix": npix / 1e6,
                       "l2": "flushed between steps (512 MB write)", "parallelism": "replicas",
                       "tile": "32 x %d target pixels per staged source box (tuned)" % tuned},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "issue": recorded_issue(),
                         "peak_source": peak_src,
                         "bytes_per_pixel": BYTES_PER_PIX},
            "fp64_path": {"ms_per_step": ms64, "value": npix / (ms64 * 1e-3) / 1e6,
                          "unit": "Mpix/s", "split_speedup": ms64 / ms, "roofline": fp64_roof},
            "pipe_peaks": {k: v / 1e12 for k, v in pipes.items()},
            "pipe_peaks_unit": "T per second (flops, or special-function results)",
            "split_vs_fp64_px": {"max": dmax, "rms": drms},
            "inverse_sip_fit_px": {"max": fit_max, "rms": fit_rms},
            "e2e": {"value": npix * world / e2e_s / 1e6, "unit": "Mpix/s",
                    "h2d_bytes_per_step": int(img.nbytes),
                    "d2h_bytes_per_step": int(2 * npix * 4)},
            "gpu_launches": args.steps,
            "clocks": clk,
            "timed_wall_s": wall,
            "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ other configurations
def _events_time(fn, k, flush=None):
    """Median device time (ms, CUDA events around each call) and median host time of the call
    itself (ms, until it returns). The k calls are enqueued back to back (each after the L2
    flush when one is given), so the host prepares a call while the device runs the previous
    work: the events time the device work, not the host's preparation of it."""
    import torch
    evs, hs = [], []
    torch.cuda.synchronize()
    for _ in range(k):
        if flush is not None:
            flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        t0 = time.perf_counter()
        fn()
        hs.append((time.perf_counter() - t0) * 1e3)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    ts = [a.elapsed_time(b) for a, b in evs]
    return float(np.median(ts)), float(np.median(hs))


def measure_batch64(dfr, torch, flush, steps):
    """The batch configuration: 64 exposures (long side 2048-6144 px, SIP3) onto one 8192^2
    target, bilinear, split precision, value and footprint; dfr_reproject_batch (a CUDA graph of
    single-frame kernels or one kernel over the frame table, tuned on the first call) against 64
    separate dfr_reproject calls."""
    c = synth.config2()
    tgt = dfr.to_c(c["tgt"])
    srcs = [dfr.to_c(dfr.fit_inverse_sip(sw, 4)[0]) for sw in c["src"]]
    imgs = [torch.from_numpy(i).cuda() for i in c["images"]]
    src_bytes = sum(i.numel() * 4 for i in imgs)
    del c
    bbs = [dfr.target_bbox(sw, tgt) for sw in srcs]
    outs = [torch.empty((b[3], b[2]), device="cuda") for b in bbs]
    fps = [torch.empty_like(o) for o in outs]
    npx = sum(b[2] * b[3] for b in bbs)
    batch = lambda: dfr.reproject_batch(imgs, srcs, tgt, bbs, order="bilinear", outs=outs,
                                        fps=fps)
    batch()  # the first call of this kind tunes the launch
    torch.cuda.synchronize()
    cfg = dfr.last_launch_config()["batch"]
    t_batch, h_batch = _events_time(batch, steps, flush)

    def separate():
        for k in range(len(imgs)):
            dfr.reproject(imgs[k], srcs[k], tgt, bbox=bbs[k], order="bilinear", out=outs[k],
                          fp_out=fps[k])
    separate()
    t_sep, h_sep = _events_time(separate, steps, flush)
    dfr.device_status()
    peak = _peaks()[0]
    # algorithmic bytes: every source pixel read once, value and footprint written
    algo = src_bytes + 8 * npx
    return {"workload": "64 frames (2048-6144 px, SIP3) -> 8192^2, bilinear, split",
            "output_mpix": npx / 1e6, "ms": t_batch, "host_call_ms": h_batch,
            "separate_launches_ms": t_sep, "mpix_s": npx / t_batch / 1e3,
            "separate_mpix_s": npx / t_sep / 1e3, "speedup_vs_separate": t_sep / t_batch,
            "roofline": {"bound": "hbm", "achieved": algo / (t_batch * 1e-3) / 1e9,
                         "peak": peak, "unit": "GB/s",
                         "frac": algo / (t_batch * 1e-3) / 1e9 / peak,
                         "bytes": "source read once + 8 B per output pixel"},
            "tuned": cfg}


def measure_adjoint2048(dfr, torch, flush, steps):
    """The differentiation configuration: 2048^2 SIP3 source, bilinear, split, Newton inverse;
    forward (value + footprint) and the adjoint (gradients of the source pixels and of all 24
    WCS parameters) of one frame."""
    c = synth.config3()
    src = dfr.to_c(dfr.fit_inverse_sip(c["src"][0], 4)[0])
    tgt = dfr.to_c(c["tgt"])
    img = torch.from_numpy(c["images"][0]).cuda()
    g = torch.randn((2048, 2048), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    gs = torch.zeros_like(img)
    bb = (0, 0, 2048, 2048)
    npx = 2048 * 2048
    fwd = lambda: dfr.reproject(img, src, tgt, bbox=bb, order="bilinear", exact_inverse=True)
    bwd = lambda: dfr.reproject_backward(img, src, tgt, g, bb, "bilinear", "split",
                                         exact_inverse=True, grad_src=gs)
    fwd()
    bwd()
    t_f = _events_time(fwd, steps, flush)[0]
    t_b = _events_time(bwd, steps, flush)[0]
    dfr.device_status()
    peak = _peaks()[0]
    return {"workload": "2048^2 SIP3 bilinear, Newton inverse, split: forward, adjoint (source "
                        "pixels + 24 parameters)",
            "forward_ms": t_f, "adjoint_ms": t_b, "forward_mpix_s": npx / t_f / 1e3,
            "adjoint_mpix_s": npx / t_b / 1e3,
            "forward_frac_hbm": 12 * npx / (t_f * 1e-3) / 1e9 / peak,
            "adjoint_frac_hbm": 12 * npx / (t_b * 1e-3) / 1e9 / peak,
            "bytes_per_pixel": 12}


def measure_stack32(dfr, torch, flush, steps):
    """The stack configuration: 32 exposures of 6000x4000 (SIP5, AP/BP 6) onto one 12000x8000
    target, bicubic, split precision: the batched forward (value + footprint, one launch form
    tuned on the first call) and, as the second pass, the batched adjoint (source-pixel and
    parameter gradients of all 32 frames in one dfr_reproject_backward_batch call) against 32
    separate dfr_reproject_backward calls."""
    c = synth.config4()
    tgt = dfr.to_c(c["tgt"])
    srcs = [dfr.to_c(dfr.fit_inverse_sip(sw, 6)[0]) for sw in c["src"]]
    imgs = [torch.from_numpy(i).cuda() for i in c["images"]]
    src_bytes = sum(i.numel() * 4 for i in imgs)
    del c
    bbs = [dfr.target_bbox(sw, tgt) for sw in srcs]
    outs = [torch.empty((b[3], b[2]), device="cuda") for b in bbs]
    fps = [torch.empty_like(o) for o in outs]
    npx = sum(b[2] * b[3] for b in bbs)
    fwd = lambda: dfr.reproject_batch(imgs, srcs, tgt, bbs, order="bicubic", outs=outs, fps=fps)
    fwd()
    torch.cuda.synchronize()
    cfg = dfr.last_launch_config()["batch"]
    t_f = _events_time(fwd, steps, flush)[0]
    gen = torch.Generator("cuda").manual_seed(5)
    go = torch.randn((max(b[3] for b in bbs), max(b[2] for b in bbs)), device="cuda",
                     generator=gen)
    gos = [go[:b[3], :b[2]] for b in bbs]
    gs = [torch.zeros_like(i) for i in imgs]
    bwd = lambda: dfr.reproject_backward_batch(imgs, srcs, tgt, gos, bbs, "bicubic", "split",
                                               grad_srcs=gs)

    def bwd_sep():
        for k in range(len(imgs)):
            dfr.reproject_backward(imgs[k], srcs[k], tgt, gos[k], bbs[k], "bicubic", "split",
                                   grad_src=gs[k])
    bwd()
    bwd_sep()
    t_b = _events_time(bwd, max(3, steps // 2), flush)[0]
    t_s = _events_time(bwd_sep, max(3, steps // 2), flush)[0]
    dfr.device_status()
    peak = _peaks()[0]
    algo = src_bytes + 8 * npx
    return {"workload": "32 x 6000x4000 SIP5 -> 12000x8000, bicubic, split: batched forward "
                        "and batched adjoint (source pixels + CRVAL/CD)",
            "output_mpix": npx / 1e6, "forward_ms": t_f, "forward_mpix_s": npx / t_f / 1e3,
            "forward_roofline": {"bound": "hbm", "achieved": algo / (t_f * 1e-3) / 1e9,
                                 "peak": peak, "unit": "GB/s",
                                 "frac": algo / (t_f * 1e-3) / 1e9 / peak,
                                 "bytes": "source read once + 8 B per output pixel"},
            "forward_tuned": cfg,
            "adjoint_batch_ms": t_b, "adjoint_separate_ms": t_s,
            "adjoint_mpix_s": npx / t_b / 1e3,
            "adjoint_speedup_vs_separate": t_s / t_b,
            "adjoint_frac_hbm": 12 * npx / (t_b * 1e-3) / 1e9 / peak,
            "adjoint_bytes_per_pixel": 12}


def measure_configs(dfr, torch, flush, steps):
    """Every workload configuration, split precision and all-FP64, forward with value and
    footprint: 512^2 TAN bilinear (0), the 4096^2 bench frame (1), the 64-frame batch (2), the
    2048^2 differentiation frame with the Newton inverse (3) and the 32-frame stack (4). Batches
    go through dfr_reproject_batch (launch form tuned on the first call of each precision).
    Per configuration and path: ms, output Mpix/s and the HBM fraction at the algorithmic bytes
    (source read once + 8 B per output pixel). One dict per configuration."""
    peak = _peaks()[0]
    rows = []

    def entry(name, npx, src_bytes, t_split, t_fp64, extra=None):
        algo = src_bytes + 8 * npx
        d = {"workload": name, "output_mpix": npx / 1e6}
        for k, t in (("split", t_split), ("fp64", t_fp64)):
            d[k] = {"ms": t, "mpix_s": npx / t / 1e3,
                    "frac_hbm": algo / (t * 1e-3) / 1e9 / peak}
        d["split_speedup"] = t_fp64 / t_split
        d.update(extra or {})
        rows.append(d)

    def single(src, tgt, img, order, exact, bbox, fp64_steps):
        src = dfr.to_c(src)
        tgt = dfr.to_c(tgt)
        img_d = torch.from_numpy(img).cuda()
        w, h = bbox[2], bbox[3]
        o = torch.empty((h, w), device="cuda")
        f = torch.empty_like(o)
        ts = {}
        for prec, k in (("split", steps), ("fp64", fp64_steps)):
            fn = lambda: dfr.reproject(img_d, src, tgt, bbox=bbox, order=order, precision=prec,
                                       exact_inverse=exact, out=o, fp_out=f)
            fn()
            ts[prec] = _events_time(fn, k, flush)[0]
        return w * h, img.nbytes, ts["split"], ts["fp64"]

    def batch(cfg, ideg, fp64_steps):
        tgt = dfr.to_c(cfg["tgt"])
        srcs = [dfr.to_c(dfr.fit_inverse_sip(sw, ideg)[0]) for sw in cfg["src"]]
        imgs = [torch.from_numpy(i).cuda() for i in cfg["images"]]
        bbs = [dfr.target_bbox(sw, tgt) for sw in srcs]
        outs = [torch.empty((b[3], b[2]), device="cuda") for b in bbs]
        fps = [torch.empty_like(o) for o in outs]
        ts, tuned = {}, {}
        for prec, k in (("split", steps), ("fp64", fp64_steps)):
            fn = lambda: dfr.reproject_batch(imgs, srcs, tgt, bbs, order=cfg["order"],
                                             precision=prec, outs=outs, fps=fps)
            fn()
            torch.cuda.synchronize()
            tuned[prec] = dfr.last_launch_config()["batch"]
            ts[prec] = _events_time(fn, k, flush)[0]
        npx = sum(b[2] * b[3] for b in bbs)
        return npx, sum(i.numel() * 4 for i in imgs), ts["split"], ts["fp64"], tuned

    c = synth.config0()
    entry("config 0: 512^2 TAN, bilinear", *single(c["src"][0], c["tgt"], c["images"][0],
                                                   "bilinear", False, (0, 0, 512, 512), steps))
    c = synth.config1()
    src = dfr.fit_inverse_sip(c["src"][0], 4)[0]
    entry("config 1: 4096^2 TAN-SIP3, bicubic", *single(src, c["tgt"], c["images"][0], "bicubic",
                                                        False, (0, 0, 4096, 4096), 3))
    c = synth.config3()
    src = dfr.fit_inverse_sip(c["src"][0], 4)[0]
    entry("config 3: 2048^2 TAN-SIP3, bilinear, Newton inverse",
          *single(src, c["tgt"], c["images"][0], "bilinear", True, (0, 0, 2048, 2048), 3))
    del c
    npx, sb, t1, t2, tuned = batch(synth.config2(), 4, 2)
    entry("config 2: 64 frames (2048-6144 px, SIP3) -> 8192^2, bilinear", npx, sb, t1, t2,
          {"tuned": tuned})
    npx, sb, t1, t2, tuned = batch(synth.config4(), 6, 2)
    entry("config 4: 32 x 6000x4000 SIP5 -> 12000x8000, bicubic", npx, sb, t1, t2,
          {"tuned": tuned})
    dfr.device_status()
    return rows


def run_oracle(args):
    """The FP64 CPU oracle, as it stands, in one process on each configuration (no GPU):
    whole frames for the 512^2 and 2048^2 cases, 1M random pixels of the 4096^2 frame, and a
    seeded 1 % sample of every frame's bounding box for the two batches (Mpix/s of the sample,
    which extrapolates to the whole batch). One JSON line per configuration."""
    from oracle import reproject as OR
    from oracle import wcs as OW
    host = {"cores": 1, "host_cpus": len(os.sched_getaffinity(0)), "machine": os.uname().machine}

    def timed(src, tgt, img, X, Y, order, inverse):
        t0 = time.perf_counter()
        OR.reproject_pixels(src, tgt, img, X, Y, order, inverse=inverse)
        return time.perf_counter() - t0

    def line(name, npx, secs, sample):
        print(json.dumps(dict({"workload": name, "oracle_mpix_s": npx / secs / 1e6,
                               "pixels": int(npx), "seconds": secs, "sample": sample}, **host)),
              flush=True)

    c = synth.config0()
    Y, X = np.mgrid[0:512, 0:512].astype(np.float64)
    line("512^2 TAN bilinear (config 0)", X.size,
         timed(c["src"][0], c["tgt"], c["images"][0], X.ravel(), Y.ravel(), "bilinear", "poly"),
         "whole frame")
    src, tgt, img = workload()
    src = oracle_wcs(src)
    rng = synth.rng_for(7)
    n1 = 1_000_000
    X = rng.integers(0, 4096, n1).astype(np.float64)
    Y = rng.integers(0, 4096, n1).astype(np.float64)
    line("4096^2 TAN-SIP3 bicubic (config 1)", n1,
         timed(src, tgt, img, X, Y, "bicubic", "poly"), "1M random target pixels")
    c = synth.config3()
    Y, X = np.mgrid[0:2048, 0:2048].astype(np.float64)
    line("2048^2 TAN-SIP3 bilinear, Newton inverse (config 3)", X.size,
         timed(c["src"][0], c["tgt"], c["images"][0], X.ravel(), Y.ravel(), "bilinear", "newton"),
         "whole frame")
    for name, cfg, ideg in (("64 frames -> 8192^2 bilinear (config 2)", synth.config2, 4),
                            ("32 x 6000x4000 SIP5 -> 12000x8000 bicubic (config 4)",
                             synth.config4, 6)):
        c = cfg()
        rng = synth.rng_for(8)
        npx = 0
        secs = 0.0
        for f, img in zip(c["src"], c["images"]):
            f = OW.with_inverse_sip(f, ideg)[0]
            x0, y0, w, h = OR.target_bbox(f, c["tgt"])
            k = max(1, (w * h) // 100)
            X = (x0 + rng.integers(0, w, k)).astype(np.float64)
            Y = (y0 + rng.integers(0, h, k)).astype(np.float64)
            secs += timed(f, c["tgt"], img, X, Y, c["order"], "poly")
            npx += k
        line(name, npx, secs, "1 %% of every frame's bounding box (%d frames)" % len(c["src"]))
        del c


def run_extra(args):
    """Secondary measurements (not the bench line): the batch configuration (64 uneven frames
    onto 8192^2, one batch call vs 64 separate launches), the gradient configuration (2048^2,
    forward + adjoint), the stack configuration (32 x 6000x4000 -> 12000x8000, batched forward
    + batched adjoint), every configuration in both precisions, and single-frame variants. One
    JSON line each."""
    import torch
    import paper_2505_03932_gb300 as dfr
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = []
    if args.workload in ("batch64", "all"):
        c = synth.config2()
        tgt = dfr.to_c(c["tgt"])
        srcs = [dfr.to_c(dfr.fit_inverse_sip(s, 4)[0]) for s in c["src"]]
        imgs = [torch.from_numpy(i).cuda() for i in c["images"]]
        bbs = [dfr.target_bbox(s, tgt) for s in srcs]
        outs = [torch.empty((b[3], b[2]), device="cuda") for b in bbs]
        fps = [torch.empty_like(o) for o in outs]
        npx = sum(b[2] * b[3] for b in bbs)
        dfr.reproject_batch(imgs, srcs, tgt, bbs, order="bilinear", outs=outs, fps=fps)
        t_batch, h_batch = _events_time(
            lambda: dfr.reproject_batch(imgs, srcs, tgt, bbs, order="bilinear", outs=outs,
                                        fps=fps), args.steps, flush)

        def separate():
            for k in range(64):
                dfr.reproject(imgs[k], srcs[k], tgt, bbox=bbs[k], order="bilinear",
                              out=outs[k], fp_out=fps[k])
        separate()
        t_sep, h_sep = _events_time(separate, args.steps, flush)
        out.append({"workload": "64 frames (2048-6144 px, SIP3) -> 8192^2, bilinear, split",
                    "output_mpix": npx / 1e6, "batch_graph_ms": t_batch,
                    "batch_host_call_ms": h_batch, "separate_launches_ms": t_sep,
                    "separate_host_calls_ms": h_sep, "batch_mpix_s": npx / t_batch / 1e3,
                    "separate_mpix_s": npx / t_sep / 1e3,
                    "roofline_frac_hbm": (12 * npx / (t_batch * 1e-3)) / 1e9 / _peaks()[0]})
        del imgs, outs, fps
    if args.workload in ("grad2048", "all"):
        c = synth.config3()
        src = dfr.to_c(dfr.fit_inverse_sip(c["src"][0], 4)[0])
        tgt = dfr.to_c(c["tgt"])
        img = torch.from_numpy(c["images"][0]).cuda()
        g = torch.randn((2048, 2048), device="cuda")
        bb = (0, 0, 2048, 2048)
        fwd = lambda: dfr.reproject(img, src, tgt, bbox=bb, order="bilinear", exact_inverse=True)
        bwd = lambda: dfr.reproject_backward(img, src, tgt, g, bb, "bilinear", "split",
                                             exact_inverse=True)
        fwd(); bwd()
        t_f = _events_time(fwd, args.steps, flush)[0]
        t_b = _events_time(bwd, args.steps, flush)[0]
        out.append({"workload": "2048^2 SIP3 bilinear, exact inverse, forward + adjoint (split)",
                    "forward_ms": t_f, "adjoint_ms": t_b,
                    "forward_mpix_s": 4.194304 / t_f * 1e3, "adjoint_mpix_s": 4.194304 / t_b * 1e3})
    if args.workload in ("stack32", "all"):
        out.append(measure_stack32(dfr, torch, flush, max(3, args.steps // 2)))
    if args.workload in ("configs", "all"):
        out.extend(measure_configs(dfr, torch, flush, max(3, min(args.steps, 10))))
    if args.workload in ("adjoint6000", "all"):
        # one 6000x4000 SIP5 exposure of the stack configuration: forward, adjoint with the
        # polynomial inverse (CRVAL and CD gradients), adjoint with the Newton inverse (A/B too)
        c = synth.config4(n_frames=1)
        tgt = dfr.to_c(c["tgt"])
        src = dfr.to_c(dfr.fit_inverse_sip(c["src"][0], 6)[0])
        img = torch.from_numpy(c["images"][0]).cuda()
        bb = dfr.target_bbox(src, tgt)
        npx = bb[2] * bb[3]
        go = torch.randn((bb[3], bb[2]), device="cuda")
        gs = torch.zeros_like(img)
        fwd = lambda: dfr.reproject(img, src, tgt, bbox=bb, order="bicubic")
        bwd = lambda: dfr.reproject_backward(img, src, tgt, go, bb, "bicubic", "split",
                                             grad_src=gs)
        bwx = lambda: dfr.reproject_backward(img, src, tgt, go, bb, "bicubic", "split",
                                             exact_inverse=True, grad_src=gs)
        fwd(); bwd(); bwx()
        t_f = _events_time(fwd, args.steps, flush)[0]
        t_b = _events_time(bwd, args.steps, flush)[0]
        t_x = _events_time(bwx, args.steps, flush)[0]
        out.append({"workload": "6000x4000 SIP5 (AP/BP 6) -> stack target, bicubic, split",
                    "output_mpix": npx / 1e6, "forward_ms": t_f, "adjoint_ms": t_b,
                    "adjoint_exact_ms": t_x, "forward_mpix_s": npx / t_f / 1e3,
                    "adjoint_mpix_s": npx / t_b / 1e3, "adjoint_exact_mpix_s": npx / t_x / 1e3,
                    "adjoint_roofline_frac_hbm": (12 * npx / (t_b * 1e-3)) / 1e9 / _peaks()[0]})
    if args.workload in ("tsip4096", "all"):
        # the bench frame onto a target that carries SIP distortion (order 3) as well
        c = synth.config1()
        src = dfr.to_c(dfr.fit_inverse_sip(c["src"][0], 4)[0])
        tgt_d = synth.add_sip(c["tgt"], 3, 1e-6, synth.rng_for(4096))
        tgt = dfr.to_c(tgt_d)
        img = torch.from_numpy(c["images"][0]).cuda()
        bb = (0, 0, 4096, 4096)
        o = torch.empty((4096, 4096), device="cuda")
        f = torch.empty_like(o)
        fwd = lambda: dfr.reproject(img, src, tgt, bbox=bb, order="bicubic", out=o, fp_out=f)
        fwd()
        t_f = _events_time(fwd, args.steps, flush)[0]
        out.append({"workload": "4096^2 SIP3 -> 4096^2 TAN-SIP3 target, bicubic, split",
                    "forward_ms": t_f, "forward_mpix_s": 16.777216 / t_f * 1e3,
                    "roofline_frac_hbm": (12 * 16777216 / (t_f * 1e-3)) / 1e9 / _peaks()[0]})
    if args.workload in ("lanczos4096", "all"):
        # the bench frame with the Lanczos-3 interpolant (36 taps per pixel)
        c = synth.config1()
        src = dfr.to_c(dfr.fit_inverse_sip(c["src"][0], 4)[0])
        tgt = dfr.to_c(c["tgt"])
        img = torch.from_numpy(c["images"][0]).cuda()
        bb = (0, 0, 4096, 4096)
        o = torch.empty((4096, 4096), device="cuda")
        f = torch.empty_like(o)
        fwd = lambda: dfr.reproject(img, src, tgt, bbox=bb, order="lanczos3", out=o, fp_out=f)
        fwd()
        t_f = _events_time(fwd, args.steps, flush)[0]
        out.append({"workload": "4096^2 SIP3 -> 4096^2 TAN, Lanczos-3, split",
                    "forward_ms": t_f, "forward_mpix_s": 16.777216 / t_f * 1e3,
                    "roofline_frac_hbm": (12 * 16777216 / (t_f * 1e-3)) / 1e9 / _peaks()[0]})
    if args.workload in ("bspline4096", "all"):
        # the bench frame with the cubic B-spline: prefilter once, then reproject the coefficients
        c = synth.config1()
        src = dfr.to_c(dfr.fit_inverse_sip(c["src"][0], 4)[0])
        tgt = dfr.to_c(c["tgt"])
        img = torch.from_numpy(c["images"][0]).cuda()
        coef = torch.empty_like(img)
        bb = (0, 0, 4096, 4096)
        o = torch.empty((4096, 4096), device="cuda")
        f = torch.empty_like(o)
        pre = lambda: dfr.bspline_prefilter(img, out=coef)
        fwd = lambda: dfr.reproject(coef, src, tgt, bbox=bb, order="bspline3", out=o, fp_out=f,
                                    prefiltered=True)
        pre(); fwd()
        t_p = _events_time(pre, args.steps, flush)[0]
        t_f = _events_time(fwd, args.steps, flush)[0]
        out.append({"workload": "4096^2 SIP3 -> 4096^2 TAN, cubic B-spline, split",
                    "prefilter_ms": t_p, "forward_ms": t_f,
                    "forward_mpix_s": 16.777216 / t_f * 1e3,
                    "roofline_frac_hbm": (12 * 16777216 / (t_f * 1e-3)) / 1e9 / _peaks()[0]})
    if args.workload in ("coadd32", "all"):
        # the stack configuration co-added onto its 12000x8000 target, then normalised
        c = synth.config4()
        tgt = dfr.to_c(c["tgt"])
        srcs = [dfr.to_c(dfr.fit_inverse_sip(s, 6)[0]) for s in c["src"]]
        imgs = [torch.from_numpy(i).cuda() for i in c["images"]]
        bbs = [dfr.target_bbox(s, tgt) for s in srcs]
        npx = sum(b[2] * b[3] for b in bbs)
        NX, NY = int(tgt.naxis[0]), int(tgt.naxis[1])
        sv = torch.zeros((NY, NX), device="cuda")
        sf = torch.zeros_like(sv)
        mean = torch.empty_like(sv)

        def co():
            sv.zero_()
            sf.zero_()
            dfr.coadd(imgs, srcs, tgt, bboxes=bbs, order="bicubic", sum_vf=sv, sum_f=sf)
        co()
        t_c = _events_time(co, max(3, args.steps // 2), flush)[0]
        t_z = _events_time(lambda: (sv.zero_(), sf.zero_()), 5, flush)[0]
        nz = lambda: dfr.coadd_normalize(sv, sf, out=mean)
        nz()
        t_n = _events_time(nz, args.steps, flush)[0]
        out.append({"workload": "co-add of 32 x 6000x4000 SIP5 onto 12000x8000, bicubic, split",
                    "frame_mpix": npx / 1e6, "coadd_ms": t_c - t_z, "zero_sums_ms": t_z,
                    "coadd_frame_mpix_s": npx / (t_c - t_z) / 1e3, "normalize_ms": t_n,
                    "normalize_roofline_frac_hbm":
                        (12 * NX * NY / (t_n * 1e-3)) / 1e9 / _peaks()[0]})
    for line in out:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8000,
                    help="timed steps of the bench line (8000: about 0.55 s of kernel time)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave out the batch and adjoint keys of the bench line")
    ap.add_argument("--workload", default="sip3_4096",
                    choices=["sip3_4096", "batch64", "grad2048", "stack32", "adjoint6000", "coadd32",
                             "configs",
                             "tsip4096", "lanczos4096", "bspline4096", "all", "oracle"],
                    help="sip3_4096: the bench line; the others print secondary measurements "
                         "(oracle: the CPU oracle on every configuration, no GPU)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "oracle":
        if rank == 0:
            run_oracle(args)
        return
    if args.workload != "sip3_4096":
        run_extra(args)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
