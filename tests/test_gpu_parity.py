"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (relative L2 over the whole output unless stated):
  FP64 recurrence, operator, fixed-iteration FGMRES: 1e-10 (plus max-abs
      1e-10 * max|ref|).  The two sides differ only in summation order and FMA
      contraction; each step is a fixed short sum, so the error stays near
      steps * 1e-16 * growth.
  Mixed mode (FP32 recurrence): the preconditioner output is compared at the
      FP32 level (tolerance in the test), and GMRES solutions must reach a true
      relative residual <= 1e-6, computed by the oracle's own FP64 operator.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2006_16861_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2006_16861_gb300 import htd  # noqa: E402


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def assert_close64(got, ref, tol=1e-10):
    got, ref = np.asarray(got).reshape(-1), np.asarray(ref).reshape(-1)
    assert rel_l2(got, ref) <= tol, rel_l2(got, ref)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def het_problem(ndim, n, T=3, layer=3, seed=11, ppw=7.0, rho=0.25):
    n = tuple(n)
    h = 1.0 / (max(n) - 1) if max(n) > 1 else 0.1
    cells = tuple(m + 1 for m in n)
    g = W.gaussian_random_field(seed, cells, 2.5)
    c = np.clip(2.0 + 0.6 * g, 1.0, 3.5)
    omega = 2 * math.pi * c.min() / (ppw * h)
    R = W.damping_profile(ndim, n, layer, 2.0 * omega) if min(n) > 2 * layer else \
        np.full(n, 0.3 * omega)
    F = W.point_source(ndim, n, h)
    return W.Problem(f"het{n}", ndim, n, h, c, R, omega, F, T, rho)


PRECOND_CASES = [
    ("cfg1_101", lambda: W.config_2d_constant(101), "q1mix"),
    ("2d_ragged", lambda: het_problem(2, (37, 45)), "q1mix"),
    ("2d_ragged_fd5", lambda: het_problem(2, (33, 70)), "fd5"),
    ("2d_1x1", lambda: het_problem(2, (1, 1), T=2), "q1mix"),
    ("2d_1x7", lambda: het_problem(2, (1, 7), T=2), "q1mix"),
    ("2d_3x2", lambda: het_problem(2, (3, 2), T=2), "q1mix"),
    ("3d_ragged", lambda: het_problem(3, (13, 17, 19), T=2), "q1mix"),
    ("3d_ragged_fd5", lambda: het_problem(3, (9, 11, 35), T=2), "fd5"),
    ("3d_2x2x2", lambda: het_problem(3, (2, 2, 2), T=2), "q1mix"),
    ("3d_1x3x1", lambda: het_problem(3, (1, 3, 1), T=2), "q1mix"),
]


@pytest.mark.parametrize("name,mk,stencil", PRECOND_CASES, ids=[c[0] for c in PRECOND_CASES])
@pytest.mark.parametrize("mode", ["table1", "exact"])
def test_precond_fp64_matches_oracle(name, mk, stencil, mode):
    p = mk()
    s = htd.Solver(p, precision="fp64", mode=mode, stencil=stencil)
    o = oracle.Oracle(p, stencil)
    assert s.params["nP"] == o.params.nP and s.params["steps"] == o.params.nsteps
    for F in (p.F, W.random_rhs(5, p.n)):
        ref = o.precond(F, mode)
        got = host(s.precond(dev(F)))
        assert_close64(got, ref)


@pytest.mark.parametrize("name,mk,stencil", PRECOND_CASES[:3] + PRECOND_CASES[6:8],
                         ids=[c[0] for c in PRECOND_CASES[:3] + PRECOND_CASES[6:8]])
def test_apply_H_and_residual_match_oracle(name, mk, stencil):
    p = mk()
    s = htd.Solver(p, stencil=stencil)
    o = oracle.Oracle(p, stencil)
    X = W.random_rhs(8, p.n)
    assert_close64(host(s.apply_H(dev(X))), o.apply_H(X), 1e-13)
    F = W.random_rhs(9, p.n)
    rel = htd.htd_residual_norm(s.handle, dev(F), dev(X))
    ref = np.linalg.norm(F - o.apply_H(X)) / np.linalg.norm(F)
    assert rel == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("krylov,mode", [("fgmres", "table1"), ("fgmres", "exact"),
                                         ("left", "exact"), ("left", "table1")])
def test_gmres_fp64_fixed_iterations_match_oracle(krylov, mode):
    """A fixed number of Arnoldi steps (no early exit, crossing a restart)."""
    p = het_problem(2, (29, 31), T=2)
    s = htd.Solver(p, precision="fp64", mode=mode, krylov=krylov, restart=4)
    o = oracle.Oracle(p)
    ref, rinfo = o.gmres(p.F, krylov, mode, tol=0.0, restart=4, maxit=7, fixed=True)
    U, info = s.solve(dev(p.F), tol=0.0, max_iters=7)
    assert info["iterations"] == 7 == rinfo["iterations"]
    assert info["restarts"] == rinfo["restarts"] == 2
    assert_close64(host(U), ref)
    np.testing.assert_allclose(info["hist"], rinfo["hist"], rtol=1e-8)


def test_gmres_fp64_config1_converges_to_direct_solution():
    p = W.config_2d_constant(101)
    s = htd.Solver(p, precision="fp64")
    o = oracle.Oracle(p)
    U, info = s.solve(dev(p.F), tol=1e-10, max_iters=200)
    Ug = host(U)
    assert info["converged"] and info["rel_res_true"] <= 1e-10
    assert np.linalg.norm(p.F - o.apply_H(Ug)) / np.linalg.norm(p.F) <= 1e-10
    Ud = o.direct_solve(p.F)
    assert rel_l2(Ug.reshape(-1), Ud.reshape(-1)) <= 1e-8
    Uo, oinfo = o.gmres(p.F, "fgmres", "table1", tol=1e-10, restart=20, maxit=200)
    assert info["iterations"] == oinfo["iterations"]


TB_CASES = [(37, 45), (1, 7), (3, 2), (130, 67), (101, 101), (64, 300)]
TB_CONFIGS = [(4, 12, 0, 0), (4, 10, 0, 0), (8, 6, 0, 0), (8, 20, 0, 0), (4, 10, 1, 0),
              (4, 12, 1, 0), (8, 6, 1, 0), (8, 12, 1, 0), (4, 8, 1, 1), (8, 8, 1, 1),
              (8, 10, 1, 1), (None, None, None, None)]


def tb_options(B, rpt, pair, sd):
    """Options forcing one blocked 2-D configuration (depth, rows per thread, form)."""
    if B is None:
        return {}
    form = htd.TB_COLUMN if not pair else (htd.TB_PAIR_SD if sd else htd.TB_PAIR)
    return dict(tblock=B, tb_rows=rpt, tb_form=form)


@pytest.mark.parametrize("n", TB_CASES, ids=[f"{a}x{b}" for a, b in TB_CASES])
@pytest.mark.parametrize("B,rpt,pair,sd", TB_CONFIGS,
                         ids=[f"B{b}_r{r}_p{q}_d{d}" for b, r, q, d in TB_CONFIGS])
@pytest.mark.parametrize("mode", ["table1", "exact"])
def test_temporal_blocking_matches_one_step(n, B, rpt, pair, sd, mode):
    """The 2-D FP32 recurrence with B steps per launch (shared-memory tiles with a
    halo of B, rows per thread rpt, one column per thread or node pairs in
    paired FP32 instructions, d in registers or staged in shared memory)
    against the one-step-per-launch kernel, bit for bit (the same roundings in
    the same order), and the FP64 oracle; None = the autotuner's own choice.
    Step counts that are not multiples of B and snapshots inside a launch
    included."""
    p = het_problem(2, n, T=3) if min(n) > 1 else het_problem(2, n, T=2)
    s0 = htd.Solver(p, precision="mixed", mode=mode, tblock=1)
    assert s0.params["steps_per_launch"] == 1
    s1 = htd.Solver(p, precision="mixed", mode=mode, **tb_options(B, rpt, pair, sd))
    if B is not None:
        assert s1.params["steps_per_launch"] == B
        assert s1.params["tile"][2] == (2 if pair else 1)
        groups = (20, 16, 8) if pair else ((16,) if rpt in (6, 10) else (8,))
        assert s1.params["tile"][1] in [g * rpt - 2 * B for g in groups]
    o = oracle.Oracle(p)
    for F in (p.F, W.random_rhs(6, p.n)):
        a = host(s0.precond(dev(F))).reshape(-1)
        b = host(s1.precond(dev(F))).reshape(-1)
        assert np.array_equal(b, a), rel_l2(b, a)
        assert rel_l2(b, o.precond(F, mode).reshape(-1)) <= 2e-5


S3_CASES = [(13, 17, 19), (40, 9, 70), (1, 3, 1), (2, 2, 2), (64, 16, 33), (5, 33, 65)]


S3_KERNELS = {"0": htd.S3_NODE_32x8, "1": htd.S3_NODE_64x4, "2": htd.S3_NODE_128x2,
              "3": htd.S3_PAIR}


def s3_options(tile):
    """Options forcing a streamed 3-D kernel ("0".."2" one node per thread on
    32 x 8, 64 x 4, 128 x 2 tiles; "3" node pairs), ":k" = k ring stages."""
    o = dict(s3_kernel=S3_KERNELS[tile.split(":")[0]])
    if ":" in tile:
        o["s3_stages"] = int(tile.split(":")[1])
    return o


@pytest.mark.parametrize("n", S3_CASES, ids=["x".join(map(str, c)) for c in S3_CASES])
@pytest.mark.parametrize("mode", ["table1", "exact"])
@pytest.mark.parametrize("tile", ["0", "1", "2", "3", "3:4", "3:6", "3:7"])
def test_streamed_3d_step_matches_register_kernel(n, mode, tile):
    """The TMA-streamed 3-D FP32 step (one node per thread on 32 x 8, 64 x 4 or
    128 x 2 column tiles, or node pairs in paired FP32 instructions on 64 x 8
    tiles; z chunks, a ring of shared-memory stages fed by a producer warp)
    against the register z-march kernel and the FP64 oracle, on ragged grids
    (odd nx leaves the last pair half-used) and several z chunks (16 planes per
    chunk at these sizes); "3:4", "3:6" and "3:7" run the pair kernel with 4, 6
    or 7 ring stages instead of the default 5."""
    p = het_problem(3, n, T=2)
    s0 = htd.Solver(p, precision="mixed", mode=mode, s3_kernel=htd.S3_ZMARCH)
    assert s0.params["step_kernel"] == 0
    s1 = htd.Solver(p, precision="mixed", mode=mode, **s3_options(tile))
    assert s1.params["step_kernel"] == 2
    o = oracle.Oracle(p)
    for F in (p.F, W.random_rhs(7, p.n)):
        a = host(s0.precond(dev(F))).reshape(-1)
        b = host(s1.precond(dev(F))).reshape(-1)
        assert rel_l2(b, a) <= 1e-6, rel_l2(b, a)
        assert rel_l2(b, o.precond(F, mode).reshape(-1)) <= 2e-5


@pytest.mark.parametrize("zchunk", [1, 5, 7])
@pytest.mark.parametrize("tile", ["0", "3"])
def test_streamed_3d_forced_z_chunks(zchunk, tile):
    """Short and ragged z chunks (19 planes as 19 x 1, 5+5+5+4, 7+7+5): every
    chunk boundary re-reads its two halo planes, and the result is the same as
    one-chunk streaming and the register z-march kernel, to rounding."""
    p = het_problem(3, (37, 21, 19), T=2)
    s0 = htd.Solver(p, precision="mixed", s3_kernel=htd.S3_ZMARCH)
    s1 = htd.Solver(p, precision="mixed", s3_zchunk=zchunk, **s3_options(tile))
    assert s1.params["step_kernel"] == 2
    assert s1.params["tile"][2] == zchunk
    F = W.random_rhs(8, p.n)
    a = host(s0.precond(dev(F))).reshape(-1)
    b = host(s1.precond(dev(F))).reshape(-1)
    assert rel_l2(b, a) <= 1e-6, rel_l2(b, a)


def test_mixed_precond_is_fp32_accurate():
    """FP32 recurrence against the FP64 oracle: the relative error stays at the
    FP32 level (unit roundoff 6e-8 times a modest growth over 120 steps)."""
    p = W.config_2d_constant(101)
    s = htd.Solver(p, precision="mixed")
    o = oracle.Oracle(p)
    for F in (p.F, W.random_rhs(3, p.n)):
        err = rel_l2(host(s.precond(dev(F))).reshape(-1), o.precond(F).reshape(-1))
        assert err <= 2e-5, err


@pytest.mark.parametrize("mk", [lambda: W.config_2d_constant(101),
                                lambda: het_problem(3, (21, 19, 23), T=3)])
def test_mixed_gmres_reaches_1e6_true_residual(mk):
    p = mk()
    s = htd.Solver(p, precision="mixed")
    o = oracle.Oracle(p)
    U, info = s.solve(dev(p.F), tol=1e-6, max_iters=200)
    Ug = host(U)
    rel = np.linalg.norm(p.F - o.apply_H(Ug)) / np.linalg.norm(p.F)
    assert info["converged"] and rel <= 1e-6
    Ud = o.direct_solve(p.F)
    # error against the exact discrete solution, bounded by cond(H) * 1e-6
    assert rel_l2(Ug.reshape(-1), Ud.reshape(-1)) <= 1e-4


def test_host_buffer_solve_equals_device_solve():
    p = het_problem(2, (40, 33), T=2)
    s = htd.Solver(p, precision="mixed")
    Ud, infod = s.solve(dev(p.F), tol=1e-8, max_iters=100)
    Fh = np.ascontiguousarray(p.F, dtype=np.complex128)
    Uh = np.zeros_like(Fh)
    infoh = htd.htd_gmres_solve_host(s.handle, Fh, Uh, 1e-8, 100)
    assert infoh["iterations"] == infod["iterations"]
    assert np.array_equal(Uh, host(Ud))


def test_errors_are_reported():
    p = het_problem(2, (20, 20), T=2)
    s = htd.Solver(p)
    U, info = s.solve(dev(p.F), tol=1e-14, max_iters=2, allow_not_converged=True)
    assert info["status"] == "HTD_ERR_NOT_CONVERGED" and info["iterations"] == 2
    with pytest.raises(htd.HtdError):
        s.solve(dev(p.F), tol=1e-14, max_iters=2)
    bad = p.F.copy()
    bad[3, 3] = np.nan
    with pytest.raises(htd.HtdError) as e:
        s.solve(dev(bad), tol=1e-6, max_iters=5)
    assert e.value.status == 5
    Z = torch.zeros(p.n, dtype=torch.complex128, device="cuda")
    U, info = s.solve(Z, tol=1e-6, max_iters=5)
    assert info["converged"] and float(U.abs().max()) == 0.0


# ---------------------------------------------------------------------------
# full-size configurations, in the launch configuration the benchmark times
# ---------------------------------------------------------------------------

def test_config_2d_1001_full_size():
    """2-D 1001 x 1001 heterogeneous case: an FP64 preconditioner application
    (T = 12 periods, 144 steps, to keep the oracle's time down; same grid and
    kernel launch shape as the benchmark) against the oracle element by
    element, and the mixed-precision FGMRES solve to 1e-6 at the full T, whose
    true residual the oracle's FP64 operator checks."""
    p = W.config_2d_heterogeneous(1001)
    o = oracle.Oracle(p)
    o12 = oracle.Oracle(p, T=12)
    s64 = htd.Solver(p, precision="fp64", T=12, restart=2)
    assert_close64(host(s64.precond(dev(p.F))), o12.precond(p.F))
    s64.close()
    sm = htd.Solver(p, precision="mixed")
    U, info = sm.solve(dev(p.F), tol=1e-6, max_iters=200)
    Ug = host(U)
    rel = np.linalg.norm(p.F - o.apply_H(Ug)) / np.linalg.norm(p.F)
    assert info["converged"] and rel <= 1e-6


def test_config_3d_256_full_size():
    """3-D 256^3 layered case: the FP64 operator over the whole grid against the
    oracle, a short FP64 recurrence (T = 1) against the oracle, and the mixed
    FGMRES solve to 1e-6 checked by the oracle's operator."""
    p = W.config_3d_layered(256)
    o = oracle.Oracle(p, T=1)
    s1 = htd.Solver(p, precision="fp64", T=1, restart=2)
    X = W.random_rhs(4, p.n)
    assert_close64(host(s1.apply_H(dev(X))), o.apply_H(X), 1e-13)
    assert_close64(host(s1.precond(dev(p.F))), o.precond(p.F))
    s1.close()
    sm = htd.Solver(p, precision="mixed")
    U, info = sm.solve(dev(p.F), tol=1e-6, max_iters=100)
    Ug = host(U)
    rel = np.linalg.norm(p.F - o.apply_H(Ug)) / np.linalg.norm(p.F)
    assert info["converged"] and rel <= 1e-6


@pytest.mark.parametrize("ndim,n", [(2, (130, 67)), (2, (1001, 1001)), (3, (37, 70, 41))],
                         ids=["2d-130x67", "2d-1001", "3d-37x70x41"])
def test_overlapped_launches_change_nothing(ndim, n):
    """Consecutive step launches overlap (programmatic dependent launch: the next
    launch reads the coefficients while the previous one drains, and waits for
    it before touching a state plane).  The outputs equal those of plain
    stream-ordered launches bit for bit, captured graph and direct launches."""
    p = het_problem(ndim, n, T=2)
    # 2-D: the blocked kernel (the tuner may prefer the resident-grid one, a
    # single launch per run with nothing to overlap)
    kw = dict(tblock=8) if ndim == 2 else {}
    s0 = htd.Solver(p, precision="mixed", launch=htd.LAUNCH_NO_OVERLAP, **kw)
    F2 = W.random_rhs(5, p.n)
    ref = [host(s0.precond(dev(F))) for F in (p.F, F2)]
    s1 = htd.Solver(p, precision="mixed", **kw)
    assert s1.params["step_kernel"] in (1, 2)           # blocked 2-D or streamed 3-D
    for r in range(3):
        for F, want in zip((p.F, F2), ref):
            assert np.array_equal(host(s1.precond(dev(F))), want)
    s2 = htd.Solver(p, precision="mixed", launch=htd.LAUNCH_NO_GRAPH, **kw)
    assert np.array_equal(host(s2.precond(dev(p.F))), ref[0])
    for s in (s0, s1, s2):
        s.close()


@pytest.mark.parametrize("stages", ["5", "7"])
def test_pair_streamed_kernel_matches_one_node_kernel_bitwise(stages):
    """The node-pair streamed 3-D kernel reads each stored plane once and pushes
    it into the sums of the three node planes it touches; the terms reach each
    sum in the order of the one-node streamed kernel, and paired instructions
    round each lane like scalar ones, so the outputs agree bit for bit (ragged
    x: the last pair half-used)."""
    p = het_problem(3, (29, 45, 37), T=2)
    s0 = htd.Solver(p, precision="mixed", s3_kernel=htd.S3_NODE_32x8)
    s1 = htd.Solver(p, precision="mixed", **s3_options("3:" + stages))
    assert s0.params["step_kernel"] == s1.params["step_kernel"] == 2
    assert s1.params["tile"][:2] == [64, 8] and s0.params["tile"][:2] != [64, 8]
    for F in (p.F, W.random_rhs(9, p.n)):
        assert np.array_equal(host(s0.precond(dev(F))), host(s1.precond(dev(F))))
    s0.close()
    s1.close()
