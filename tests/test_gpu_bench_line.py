"""The benchmark's JSON line on a small workload: the contract keys are present
and the roofline figures are consistent with the quantities they derive from."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_small_workload():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "2d_const_101",
           "--steps", "3", "--warmup", "3", "--fp64-steps", "1", "--cpu-sample-s", "0",
           "--e2e-steps", "1", "--secondary-2d", "0", "--batched", "0", "--adjoint", "0", "--projection", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, check=True, cwd=ROOT).stdout
    line = json.loads(out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["steps"] == 3 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["gpu_launches"] > 0
    r = line["roofline"]
    # the 101^2 grid is L2-resident: its step kernel is reported against the
    # FP32 pipe, useful FLOPs per update x updates / kernel time
    assert r["bound"] == "alu" and r["l2_resident"] and r["unit"] == "TFLOP/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-9)
    assert 0 < r["frac"] < 1.2
    f = line["fp64_roofline"]
    assert f["bound"] == "alu" and 0 < f["frac"] < 1.2
    e = line["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0


def test_bench_line_hbm_roofline_arithmetic():
    """A grid larger than L2 (3-D 192^3, T cut by the workload's own recipe):
    achieved = algorithmic bytes per launch / average launch time, frac =
    achieved / the measured HBM copy bandwidth, and a kernel option passed by
    --option reaches the solver."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "3d_layered_192",
           "--steps", "1", "--warmup", "3", "--fp64-steps", "0", "--cpu-sample-s", "0",
           "--e2e-steps", "0", "--secondary-2d", "0", "--batched", "0", "--adjoint", "0", "--projection", "0",
           "--option", "s3_stages=5"]
    out = subprocess.run(cmd, capture_output=True, text=True, check=True, cwd=ROOT).stdout
    line = json.loads(out.strip().splitlines()[-1])
    r = line["roofline"]
    assert r["bound"] == "hbm" and not r["l2_resident"]
    assert r["bytes_per_launch"] == 192 ** 3 * 4 * 7
    achieved = r["bytes_per_launch"] / (r["avg_launch_us"] * 1e-6) / 1e9
    assert r["achieved"] == pytest.approx(achieved, rel=1e-9)
    assert r["frac"] == pytest.approx(achieved / r["peak"], rel=1e-9)
    assert 0.3 < r["frac"] < 1.2
    assert line["config"]["options"] == {"s3_stages": 5}
