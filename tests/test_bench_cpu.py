"""The benchmark's CPU legs on a small workload, without a GPU: the oracle
baseline on one core and on every host core (independent copies of the
single-thread oracle in spawned processes), and the reference arm's JSON line."""
import contextlib
import io
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402
import oracle  # noqa: E402


def test_cpu_baseline_single_and_all_cores():
    oracle.build()
    p, _ = bench.make_workload("2d_const_101")
    out = bench.cpu_baseline(p, 0.05)
    cores = len(os.sched_getaffinity(0))
    assert out["kind"] == "oracle" and out["unit"] == "Gupd/s" and out["value"] > 0
    assert out["cores"] == (cores if cores > 1 else 1)
    if cores > 1:
        assert out["single_core_value"] > 0
        # independent copies on several cores do more updates per second than one
        assert out["value"] > out["single_core_value"]
    one = bench.cpu_baseline(p, 0.05, all_cores=False)
    assert one["cores"] == 1 and one["value"] > 0


def test_oracle_steps_count_two_real_updates_per_node():
    oracle.build()
    p, _ = bench.make_workload("2d_const_101")
    o = oracle.Oracle(p, T=1)
    dt, ups = bench.oracle_steps(o, p.F, 3)
    assert dt > 0 and ups == 2 * 101 * 101 * 3


def test_reference_arm_line(monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    args = bench.parse_args(["--impl", "reference", "--workload", "2d_const_101",
                             "--steps", "2", "--warmup", "1"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip())
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "Gupd/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == 1 and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "Gupd/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "2d_const_101"


def test_kernel_option_parsing():
    args = bench.parse_args(["--option", "s3_zchunk=32", "--option", "tb_form=3"])
    assert bench.kernel_options(args) == {"s3_zchunk": 32, "tb_form": 3}
    with pytest.raises(SystemExit):
        bench.kernel_options(bench.parse_args(["--option", "s3_zchunk"]))


def test_default_workload_is_the_largest_single_gpu_config():
    assert bench.parse_args([]).workload == "3d_layered_256"


def test_traffic_records_follow_the_kernel_source(tmp_path, monkeypatch):
    """Each ncu traffic record holds while the kernel's region of its source file
    is the one captured, also after edits elsewhere in the file, and turns
    null once the region changes."""
    import shutil
    for key, rec in bench.NCU_TRAFFIC.items():
        assert bench.ncu_traffic(key, rec["nodes"]) == rec["bytes"], key
    csrc = tmp_path / "paper_2006_16861_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(ROOT, "paper_2006_16861_gb300", "csrc", "htd_tblock.cu")
    shutil.copy(src, csrc / "htd_tblock.cu")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = bench.NCU_TRAFFIC["tb2d_pair"]
    text = (csrc / "htd_tblock.cu").read_text()
    (csrc / "htd_tblock.cu").write_text(text + "\n// an edit outside the kernel\n")
    assert bench.ncu_traffic("tb2d_pair", rec["nodes"]) == rec["bytes"]
    i = text.index(rec["begin"])
    (csrc / "htd_tblock.cu").write_text(text[:i + 5] + "x" + text[i + 5:])
    assert bench.ncu_traffic("tb2d_pair", rec["nodes"]) is None


def test_oracle_solves_the_101_configuration_for_the_cpu_leg():
    """The CPU leg's whole-solve figure for the 101^2 configuration: the oracle's
    FGMRES(20) with Table 1 reaches 1e-6 in a handful of iterations."""
    oracle.build()
    out = bench.cpu_config1_solve()
    assert out["kind"] == "oracle" and out["cores"] == 1
    assert 1 <= out["iterations"] <= 20 and out["time_to_tol_ms"] > 0
