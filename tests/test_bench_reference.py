"""The CPU arm of bench.py: the oracle timed on every host core prints one well-formed line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Mpix/s"
    cores = min(len(os.sched_getaffinity(0)), 32)
    assert line["cpu_baseline"]["cores"] == cores
    assert line["config"]["sample_pixels_per_step"] == 250_000 * cores
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_recorded_captures_follow_the_kernel_code(tmp_path):
    """The bench line reports a recorded ncu capture only while the kernel sources match it: a
    change of comments keeps the record, a change of code drops it."""
    import importlib.util
    import shutil
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    assert b.recorded_traffic() is not None and b.recorded_fp64() is not None
    csrc = tmp_path / "paper_2505_03932_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2505_03932_gb300", "csrc"), csrc)
    shutil.copytree(os.path.join(ROOT, "profiles"), tmp_path / "profiles")
    b.ROOT = str(tmp_path)
    k = csrc / "dfr_fwd_kernels.cuh"
    text = k.read_text()
    k.write_text("// a comment\n" + text.replace("\n", "\n/* another */\n", 1))
    assert b.recorded_traffic() is not None and b.recorded_fp64() is not None
    k.write_text(text.replace("constexpr int kSplitMinBlocks = 16;",
                              "constexpr int kSplitMinBlocks = 17;"))
    assert b.recorded_traffic() is None and b.recorded_fp64() is None
