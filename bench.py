#!/usr/bin/env python
"""Benchmark of the time-domain preconditioned FGMRES solver on one GB300.

One step = one complete solve of H U = F to a true relative residual of 1e-6
(preconditioner split, T n_P recurrence steps per application, snapshot /
join, true-operator residual, FP64 Arnoldi and Givens, solution update) on the
2-D 1001 x 1001 heterogeneous workload: h = 1/1000, c a seeded smooth Gaussian
random field (correlation length 0.05, clipped to [1.5, 4.5]), omega for 8
points per wavelength at min c, 40-cell absorbing layer, one centre point
source, T = 125 periods, n_P = 12 (1500 steps per application), FGMRES(20),
FP32 recurrence with FP64 Krylov ("mixed").

Printed (one JSON line on rank 0):
  value       recurrence grid-point updates per second over the whole solve,
              all ranks (Gupd/s), device time (CUDA events on the solve stream),
              L2 flushed (256 MiB write) between timed steps;
  roofline    the step kernel: algorithmic bytes per launch / average launch
              time, measured live (events around every preconditioner
              application), against the measured HBM copy bandwidth; with the
              ncu DRAM bytes per launch (`traffic`, null once the kernel source
              differs from the captured one) and, for the blocked kernel, the
              one-step-equivalent bandwidth and its fraction (`effective_*`);
  fp64_roofline the FP64 step kernel of the plain form against the FP64 pipe;
  e2e         the same metric through htd_gmres_solve_host with pinned host
              buffers, host<->device copies inside the timed region;
  time_to_tol_ms / fp64_time_to_tol_ms / speedup_vs_fp64
              the solve time in mixed and in plain FP64 mode on the same GPU;
  secondary_3d the FP32 recurrence on the 3-D 256^3 layered workload and its
              HBM roofline (the HBM-bound case);
  batched     the 96-system batched workload solved in lockstep;
  cpu_baseline the FP64 CPU oracle on a bounded sample of the same workload;
  clocks, gpu_launches  SM clocks sampled during the timed region; kernels
              launched by the library in it.

--impl reference times the oracle on the same workload and metric.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "recurrence Gpt-updates/s & %HBM peak; GMRES time-to-1e-6 vs FP64 plain"
UNIT = "Gupd/s"
TOL = 1e-6
# algorithmic bytes per node of one step-kernel launch (FP32): a one-step launch
# reads u_j, u_{j-1}, q*kappa, d, Re F, Im F and writes u_{j+1} (7 words); a
# B-step temporally blocked launch reads the same 6 planes once and writes the
# last two states (8 words)
WORDS_ONE_STEP, WORDS_BLOCKED = 7, 8
# FP64 recurrence: FLOPs per point update as the step kernels compute it (FMA =
# 2): 2-D 12 FMA + 20 add/mul; 3-D 57 FMA + 21 add/mul (27 coefficients and 27
# products of the stencil sum, 19 cell sums, forcing and update); FP64 pipe
# peak 2 DFMA per clock per SM x 152 SMs x 2 x 2.07e9
FP64_FLOPS_PER_UPDATE = {2: 44, 3: 135}
FP64_PEAK_TFLOPS = 2 * 152 * 2 * 2.07e9 / 1e12

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
# capture, valid only for the kernel source it was taken on (sha256 prefix of the
# file); scaled by node count to other grid sizes.  The captures are summarised
# under profiles/.
NCU_TRAFFIC = {
    "tb2d_pair": {"file": "htd_tblock.cu", "sha16": "b9afe2271fc20c85", "bytes": 25192448 + 1792,
                  "nodes": 1001 * 1001},
    "stream3d": {"file": "htd_stream3d.cu", "sha16": "4f289c964d28aa22",
                 "bytes": 193680896 + 18157568, "nodes": 192 ** 3},
    "stream3d_pair": {"file": "htd_stream3d_pair.cu", "sha16": "8c6bdafcd9f39e71",
                      "bytes": 201089536 + 15837696, "nodes": 192 ** 3},
}


def step_kernel_name(prm, ndim):
    """(name, traffic key) of the recurrence kernel a context uses."""
    sk = prm.get("step_kernel")
    if sk == 1:
        if prm["tile"][2] == 2:
            return f"tb2d_pair_kernel<{prm['steps_per_launch']}>", "tb2d_pair"
        return f"tb2d_kernel<float,{prm['steps_per_launch']}>", "tb2d"
    if sk == 2:
        if list(prm["tile"][:2]) == [64, 8]:
            return "stream3d_pair_kernel", "stream3d_pair"
        return "stream3d_kernel", "stream3d"
    return ("step2d_kernel<float>" if ndim == 2 else "step3d_kernel<float>"), None


def ncu_traffic(key, nodes):
    """Measured DRAM bytes per launch for `nodes` nodes, or None if the kernel
    source changed since the capture."""
    import hashlib
    rec = NCU_TRAFFIC.get(key)
    if rec is None:
        return None
    path = os.path.join(ROOT, "paper_2006_16861_gb300", "csrc", rec["file"])
    try:
        with open(path, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    if sha != rec["sha16"]:
        return None
    return rec["bytes"] * nodes / rec["nodes"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2d_grf_1001",
                    choices=["2d_grf_1001", "3d_layered_256", "3d_layered_192", "2d_const_101",
                             "3d_paper_shape", "3d_paper_shape_4hz", "3d_paper_shape_6hz"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-s", type=float, default=10.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--restart", type=int, default=20)
    ap.add_argument("--batched", type=int, default=1,
                    help="also time the batched workload (96 systems, lockstep FGMRES)")
    ap.add_argument("--secondary-3d", type=int, default=1,
                    help="also time the FP32 recurrence on the 3-D 256^3 workload (HBM-bound)")
    return ap.parse_args(argv)


def make_workload(name, rank=0):
    from paper_2006_16861_gb300 import workloads as W
    if name == "2d_grf_1001":
        p = W.config_2d_heterogeneous(1001)
        desc = ("2-D 1001x1001 heterogeneous (GRF c in [1.5,4.5], corr 0.05), h=1/1000, "
                "8 ppw at min c, 40-cell layer R0=2w, point source, T=125, rho=0.25")
    elif name == "3d_layered_256":
        p = W.config_3d_layered(256)
        desc = ("3-D 256^3 4-layer c [1.5..4.5] x (1+0.1 GRF), h=1/255, 8 ppw at min c, "
                "24-cell layer R0=2w, point source, T=32, rho=0.25")
    elif name == "3d_layered_192":
        p = W.config_3d_layered(192, layer=18)
        desc = ("3-D 192^3 (profiling size) 4-layer c [1.5..4.5] x (1+0.1 GRF), h=1/191, "
                "8 ppw at min c, 18-cell layer R0=2w, point source, T=24, rho=0.25")
    elif name == "3d_paper_shape":
        p = W.config_3d_paper_shape()
        desc = ("3-D 200x200x106 (the paper's smallest 3-D example size), 4-layer model in place "
                "of SEG/EAGE salt, 6 ppw at min c, 16-cell layer R0=2w, point source, T=25")
    elif name == "3d_paper_shape_4hz":
        p = W.config_3d_paper_shape(shape=(130, 280, 280), T=40)
        desc = ("3-D 280x280x130 (the paper's second 3-D example size), 4-layer model in place "
                "of SEG/EAGE salt, 6 ppw at min c, 16-cell layer R0=2w, point source, T=40")
    elif name == "3d_paper_shape_6hz":
        p = W.config_3d_paper_shape(shape=(165, 392, 392), T=60)
        desc = ("3-D 392x392x165 (the paper's largest 3-D example size), 4-layer model in place "
                "of SEG/EAGE salt, 6 ppw at min c, 16-cell layer R0=2w, point source, T=60")
    else:
        p = W.config_2d_constant(101)
        desc = "2-D 101x101 constant c=1, h=0.01, 10 ppw, 20-cell layer, point source, T=10"
    if rank:
        # weak scaling: every rank solves its own independent instance (source moved)
        pos = tuple((m - 1) // 2 + (rank * 7) % max(1, m // 4) for m in p.n)
        p.F = W.point_source(p.ndim, p.n, p.h, pos=pos)
    return p, desc


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001 - fall back to the recipe's figure
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001 - no nvidia-smi: no clock record
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [x for x in sm if x >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(p, budget_s):
    """The FP64 oracle (single thread) on a bounded sample: one Table 1 application
    with T_sample periods on the same grid.  Returns (Gupd/s, description)."""
    import oracle
    o1 = oracle.Oracle(p, T=1)
    t0 = time.perf_counter()
    o1.precond(p.F)
    t1 = time.perf_counter() - t0
    T_sample = int(max(1, min(p.T, math.floor(budget_s / max(t1, 1e-3)))))
    o = oracle.Oracle(p, T=T_sample)
    t0 = time.perf_counter()
    o.precond(p.F)
    dt = time.perf_counter() - t0
    ups = math.prod(p.n) * o.params.nsteps
    return ups / dt / 1e9, (f"oracle Table-1 preconditioner, {T_sample} periods "
                            f"({o.params.nsteps} steps) on the full grid, {dt:.1f} s")


def secondary_3d(htd, stream, flush, peaks):
    """Time preconditioner applications (T = 4, 48 steps each) on 3d_layered_256 with
    CUDA events; report Gupd/s and the step kernel's HBM roofline fraction."""
    import torch
    from paper_2006_16861_gb300 import workloads as W
    p3 = W.config_3d_layered(256, T=4)
    N3 = math.prod(p3.n)
    s3 = htd.Solver(p3, precision="mixed", restart=1)
    prm = s3.params
    F3 = torch.from_numpy(np.ascontiguousarray(p3.F)).cuda()
    U3 = torch.zeros_like(F3)
    s3.precond(F3, U3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(3):
        flush.fill_(4)
        e0.record(stream)
        htd.htd_apply_precond(s3.handle, F3, U3, stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    s3.close()
    ms = statistics.mean(times)
    us_step = 1e3 * ms / prm["steps"]
    bytes_step = N3 * 4 * WORDS_ONE_STEP
    peak, kind = peaks()
    achieved = bytes_step / (us_step * 1e-6) / 1e9
    kern, tkey = step_kernel_name(prm, 3)
    return {"workload": "3d_layered_256 (T=4, 48 steps per application)",
            "value": N3 * prm["steps"] / (ms * 1e-3) / 1e9, "unit": UNIT,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": ncu_traffic(tkey, N3) if tkey else None,
                         "tile": prm["tile"],
                         "kernel": kern,
                         "bytes_per_launch": bytes_step, "avg_launch_us": us_step,
                         "peak_kind": f"{kind} HBM copy bandwidth"}}


def secondary_batched(htd, stream, flush, sub_rhs=4, sub_inst=4):
    """Batched workload: the 3-D layered model at 128^3 with 32 seeded point sources
    as 32 right-hand sides of one handle, plus 64 2-D instances with sides uniform in
    [200, 1000] -- 96 systems, one CUDA-graph launch per preconditioner round,
    lockstep FGMRES(20) to 1e-6.  CUDA events on the solve stream: one warm-up solve
    (it also builds the graph), then one timed solve.  The plain FP64 GPU form is
    timed on a sub-batch (the 3-D handle with `sub_rhs` sources and `sub_inst` 2-D
    instances) next to the mixed form on the same sub-batch."""
    import torch
    from paper_2006_16861_gb300 import workloads as W
    setup = W.config_batched()

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()

    def run(precision, probs, Fs, reps):
        solvers = [htd.Solver(p, precision=precision, max_rhs=F.shape[0], restart=20)
                   for p, F in zip(probs, Fs)]
        b = htd.Batch(solvers, [F.shape[0] for F in Fs])
        Fd = [dev(F) for F in Fs]
        Us = b.zeros()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        times, infos = [], None
        for r in range(reps + 1):
            for U in Us:
                U.zero_()
            flush.fill_(5)
            e0.record(stream)
            Us, infos = b.solve(Fd, Us, tol=TOL, max_iters=400, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if r > 0 or reps == 0:
                times.append(e0.elapsed_time(e1))
        ups, k = 0, 0
        for p, F in zip(probs, Fs):
            for _ in range(F.shape[0]):
                ups += p.N * infos[k]["steps"]
                k += 1
        b.close()
        for sv in solvers:
            sv.close()
        return min(times), ups, infos

    ms, ups, infos = run("mixed", setup.probs, setup.F, 1)
    its = [i["iterations"] for i in infos]
    sub_p = setup.probs[:1 + sub_inst]
    sub_F = [setup.F[0][:sub_rhs]] + setup.F[1:1 + sub_inst]
    ms_m, _, _ = run("mixed", sub_p, sub_F, 1)
    ms_f, _, inf_f = run("fp64", sub_p, sub_F, 0)
    return {"workload": "batched: 3d_layered_128 x 32 sources + 64 2-D instances (sides 200..1000)",
            "systems": len(infos),
            "unknowns": int(sum(p.N * F.shape[0] for p, F in zip(setup.probs, setup.F))),
            "value": ups / (ms * 1e-3) / 1e9, "unit": UNIT, "time_to_tol_ms": ms,
            "iterations_min": min(its), "iterations_max": max(its),
            "rel_res_true_max": max(i["rel_res_true"] for i in infos),
            "graph": "one launch per preconditioner round (65 child graphs)",
            "fp64_sub_batch": {"systems": sub_rhs + sub_inst, "mixed_ms": ms_m, "fp64_ms": ms_f,
                               "speedup_vs_fp64": ms_f / ms_m,
                               "fp64_rel_res_true_max": max(i["rel_res_true"] for i in inf_f)}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    p, desc = make_workload(args.workload)
    # each step: a bounded sample (2 periods of the recurrence) of the workload
    o = oracle.Oracle(p, T=2)
    ups = math.prod(p.n) * o.params.nsteps
    for _ in range(args.warmup):
        o.precond(p.F)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.precond(p.F)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = ups * len(times) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "description": desc,
                                        "sample": "2 periods of the recurrence per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"oracle Table-1 preconditioner, 2 periods "
                                   f"({o.params.nsteps} steps) per step, full grid"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def all_reduce_scalar(x, op, world, device):
    """One float reduced over the ranks (op: a torch.distributed.ReduceOp); the
    value itself when there is one rank.  device: "cuda" under NCCL, "cpu" under
    gloo."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2006_16861_gb300 import htd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def allmax(x):
        return all_reduce_scalar(x, dist.ReduceOp.MAX, world, "cuda")

    def allsum(x):
        return all_reduce_scalar(x, dist.ReduceOp.SUM, world, "cuda")

    p, desc = make_workload(args.workload, rank)
    N = math.prod(p.n)
    stream = torch.cuda.current_stream()
    F = torch.from_numpy(np.ascontiguousarray(p.F)).cuda()
    U = torch.zeros_like(F)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    solver = htd.Solver(p, precision="mixed", mode="table1", krylov="fgmres",
                        restart=args.restart)
    prm = solver.params

    def solve_once():
        U.zero_()
        return htd.htd_gmres_solve(solver.handle, F, U, TOL, 400, stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        solve_once()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(local)
    gpu_id = f"GPU-{props.uuid}" if hasattr(props, "uuid") else str(local)
    clocks = ClockSampler(gpu_id)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ms_steps, ups, launches, ms_prec, steps_run, its, rels = [], 0, 0, 0.0, 0, [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.fill_(2)                       # evict L2 between timed steps
        e0.record(stream)
        info = solve_once()
        e1.record(stream)
        e1.synchronize()
        ms_steps.append(e0.elapsed_time(e1))
        ups += N * info["steps"]
        launches += info["launches"]
        ms_prec += info["ms_precond"]
        steps_run += info["steps"]
        its.append(info["iterations"])
        rels.append(info["rel_res_true"])
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = allmax(sum(ms_steps))
    all_ups = allsum(ups)
    value = all_ups / (total_ms * 1e-3) / 1e9

    # roofline of the step kernel: algorithmic bytes per launch / average launch time
    spl = max(1, int(prm.get("steps_per_launch", 1) or 1))
    runs = steps_run // prm["steps"]
    step_launches = runs * (-(-prm["steps"] // spl))
    avg_launch_s = ms_prec * 1e-3 / max(1, step_launches)
    bytes_per_launch = N * 4 * (WORDS_ONE_STEP if spl == 1 else WORDS_BLOCKED)
    achieved = bytes_per_launch / avg_launch_s / 1e9
    peak, peak_kind = peaks()
    l2_resident = bytes_per_launch < 96 * (1 << 20)

    # e2e: host buffers through the C ABI (copies inside the timed region)
    e2e = None
    if args.e2e_steps > 0:
        Fh = torch.from_numpy(np.ascontiguousarray(p.F)).pin_memory()
        Uh = torch.zeros_like(Fh).pin_memory()
        Fn, Un = Fh.numpy(), Uh.numpy()
        Un[...] = 0
        htd.htd_gmres_solve_host(solver.handle, Fn, Un, TOL, 400, stream)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e_ups = 0
        for _ in range(args.e2e_steps):
            Un[...] = 0
            info = htd.htd_gmres_solve_host(solver.handle, Fn, Un, TOL, 400, stream)
            e_ups += N * info["steps"]
        torch.cuda.synchronize()
        wall = allmax(time.perf_counter() - t0)
        e2e = {"value": allsum(e_ups) / wall / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 2 * Fn.nbytes, "d2h_bytes_per_step": Un.nbytes,
               "ms_per_step": 1e3 * wall / args.e2e_steps}
    solver.close()

    # plain FP64 GPU form on the same workload: time to 1e-6
    fp64_ms = None
    fp64_info = None
    fp64_roof = None
    if args.fp64_steps > 0:
        s64 = htd.Solver(p, precision="fp64", mode="table1", krylov="fgmres",
                         restart=args.restart)
        U.zero_()
        htd.htd_gmres_solve(s64.handle, F, U, TOL, 400, stream)
        t = []
        for _ in range(args.fp64_steps):
            flush.fill_(3)
            U.zero_()
            e0.record(stream)
            fp64_info = htd.htd_gmres_solve(s64.handle, F, U, TOL, 400, stream)
            e1.record(stream)
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        fp64_ms = allmax(statistics.mean(t))
        s64.close()
        # the FP64 step kernel against the FP64 pipe (it is ALU-bound on GB300):
        # FLOPs per point update of step2d/step3d as written (FMA = 2)
        fp_upd = FP64_FLOPS_PER_UPDATE[p.ndim]
        upd = N * fp64_info["steps"]
        tflops = fp_upd * upd / (fp64_info["ms_precond"] * 1e-3) / 1e12
        fp64_roof = {"bound": "alu", "kernel": f"step{p.ndim}d_kernel<double>",
                     "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": tflops / FP64_PEAK_TFLOPS, "flops_per_update": fp_upd,
                     "peak_kind": "FP64 pipe: 2 DFMA per clock per SM x 152 SMs x 2.07 GHz"}

    # secondary: the recurrence alone on the 3-D 256^3 layered workload, whose
    # working set (470 MB per step) is far larger than L2
    sec = None
    if args.secondary_3d and p.ndim == 2:
        sec = secondary_3d(htd, stream, flush, peaks)
    batched = None
    if args.batched and p.ndim == 2:
        batched = secondary_batched(htd, stream, flush)

    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample_s > 0:
        import oracle
        oracle.build()
        v, sample = cpu_baseline(p, args.cpu_sample_s)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}

    ms_per_step = total_ms / args.steps
    kern, tkey = step_kernel_name(prm, p.ndim)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "dtype_detail": "recurrence f32; Arnoldi, Givens, true residual f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "n": list(p.n),
                       "T": prm["T"], "nP": prm["nP"], "steps_per_apply": prm["steps"],
                       "krylov": f"FGMRES({args.restart})", "tol": TOL, "mode": "table1",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"independent instance per GPU x{world}"},
            "time_to_tol_ms": ms_per_step,
            "fp64_time_to_tol_ms": fp64_ms,
            "speedup_vs_fp64": (fp64_ms / ms_per_step) if fp64_ms else None,
            "iterations": its[-1], "rel_res_true": max(rels),
            "fp64_iterations": fp64_info["iterations"] if fp64_info else None,
            "fp64_roofline": fp64_roof,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": ncu_traffic(tkey, N) if tkey else None,
                         "effective_single_step_gbs": N * 4 * WORDS_ONE_STEP * spl / avg_launch_s / 1e9,
                         "effective_frac": N * 4 * WORDS_ONE_STEP * spl / avg_launch_s / 1e9 / peak,
                         "kernel": kern,
                         "steps_per_launch": spl,
                         "bytes_per_launch": bytes_per_launch,
                         "avg_launch_us": avg_launch_s * 1e6,
                         "peak_kind": f"{peak_kind} HBM copy bandwidth",
                         "l2_resident": l2_resident},
            "cpu_baseline": cpu,
            "secondary_3d": sec,
            "batched": batched,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
