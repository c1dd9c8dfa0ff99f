"""The resident-grid 2-D kernel (HTD_TB_RESIDENT, step kernel 4), FP32 and FP64.

One cooperative launch runs a whole preconditioner run with the grid held in
shared memory across the SMs; neighbouring tiles swap their edge values through
tagged 64-bit words every step.  Per node it evaluates the same expression as
the one-step kernel (Def. of I_acd with Table 1's forcing and read-out), so:

- its preconditioner output is bit-identical to the one-step kernel's and the
  blocked kernel's, on grids whose tilings reach every degenerate case (tiles one
  node wide or high, one tile row or column, ragged last tiles) and at the
  1001^2 configuration's size, in Table 1 and exact read-out;
- an FGMRES solve through it repeats the one-step solve exactly;
- a neighbour wait that runs out (stall test) ends the launch with
  HTD_ERR_TIMEOUT and leaves the handle usable;
- a handle that joins a batch leaves it for its blocked configuration and the
  batch's preconditioner equals the handle's own.
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

TIMEOUT = 7


def _problem(n, T=None, seed=17):
    """2-D heterogeneous problem on an n[0] x n[1] grid (the workloads' recipe:
    c = clip(3 + 0.75 g), 8 points per wavelength at the slowest speed, damping
    layer of 12 nodes) with a few point sources."""
    h = 1.0 / (max(n) - 1)
    g = W.gaussian_random_field(seed, tuple(m + 1 for m in n), 0.05 / h)
    c = np.clip(3.0 + 0.75 * g, 1.5, 4.5)
    omega = 2 * math.pi * c.min() / (8 * h)
    R = W.damping_profile(2, n, min(12, max(1, min(n) // 4)), 2 * omega)
    if T is None:
        T = W.periods_for(max(n), h, float(c.min()), omega)
    F = W.point_source(2, n, h)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        pos = tuple(int(rng.integers(0, m)) for m in n)
        F[pos] += (1.0 - 0.5j) / (h * h)
    return W.Problem("res2d", 2, tuple(n), h, c, R, omega, F, T)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def precond(p, mode="table1", **kw):
    s = htd.Solver(p, precision="mixed", mode=mode, **kw)
    U = s.precond(dev(p.F)).cpu().numpy()
    prm = s.params
    s.close()
    return U, prm


# shapes whose tilings (at most one tile per SM) give tiles 2 nodes wide with a
# last column 1 wide, a single tile row, a single tile column, square and
# ragged tiles
SHAPES = [(37, 29), (5, 700), (700, 5), (4, 3000), (130, 257), (257, 130), (64, 64)]


@pytest.mark.parametrize("n", SHAPES)
def test_resident_equals_one_step_kernel_bit_for_bit(n):
    p = _problem(n, T=2)
    U1, prm1 = precond(p, tblock=1)
    Ur, prmr = precond(p, tb_form=htd.TB_RESIDENT)
    assert prm1["step_kernel"] == 0
    assert prmr["step_kernel"] == 4
    assert prmr["steps_per_launch"] == prmr["steps"]
    assert prmr["tile"][2] == 2 and prmr["ctas_per_sm"] == 1
    assert np.isfinite(Ur).all() and np.abs(Ur).max() > 0
    assert np.array_equal(Ur, U1), float(np.abs(Ur - U1).max())


def test_resident_equals_blocked_and_one_step_at_1001():
    """The 1001^2 configuration (one period per run, 12 steps) through the
    resident kernel, the blocked pair kernel and the one-step kernel."""
    p = W.config_2d_heterogeneous(1001, T=1)
    Ur, prmr = precond(p, tb_form=htd.TB_RESIDENT)
    Ub, prmb = precond(p, tblock=8, tb_rows=8, tb_form=htd.TB_PAIR_SD)
    U1, _ = precond(p, tblock=1)
    assert prmr["step_kernel"] == 4 and prmb["step_kernel"] == 1
    W_, H_ = prmr["tile"][:2]
    assert W_ % 2 == 0 and math.ceil(1001 / W_) * math.ceil(1001 / H_) <= 152 * 4
    assert np.array_equal(Ub, U1)
    assert np.array_equal(Ur, U1)


@pytest.mark.parametrize("n", [(37, 29), (130, 257)])
def test_resident_exact_mode_equals_one_step(n):
    p = _problem(n, T=2)
    U1, _ = precond(p, mode="exact", tblock=1)
    Ur, prm = precond(p, mode="exact", tb_form=htd.TB_RESIDENT)
    assert prm["step_kernel"] == 4
    assert np.array_equal(Ur, U1)


def test_resident_full_run_matches_the_oracle():
    """All T n_P steps of one application on a 129 x 161 grid against the FP64
    oracle: the FP32 recurrence's 2e-5 (relative L2 and maximum norm)."""
    p = _problem((129, 161))
    Ur, prm = precond(p, tb_form=htd.TB_RESIDENT)
    assert prm["step_kernel"] == 4 and prm["steps"] > 100
    ref = oracle.Oracle(p).precond(p.F)
    a, b = Ur.reshape(-1), ref.reshape(-1)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 2e-5
    assert np.abs(a - b).max() / np.abs(b).max() <= 2e-5


def test_resident_solve_repeats_the_one_step_solve():
    p = _problem((129, 161))
    F = dev(p.F)
    out = []
    for kw in (dict(tblock=1), dict(tb_form=htd.TB_RESIDENT)):
        s = htd.Solver(p, precision="mixed", **kw)
        U, info = s.solve(F, tol=1e-6, max_iters=300)
        assert info["converged"]
        out.append((U.cpu().numpy(), info["iterations"], info["rel_res_true"]))
        s.close()
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert np.array_equal(out[0][0], out[1][0])


def test_resident_wait_runs_out_then_the_handle_solves():
    p = _problem((129, 161))
    s = htd.Solver(p, precision="mixed", tb_form=htd.TB_RESIDENT)
    assert s.params["step_kernel"] == 4
    F = dev(p.F)
    htd.htd_set_wait_limit(s.handle, 1_000_000, stall_test=True)     # 1 ms, stalled
    U = s.zeros()
    with pytest.raises(htd.HtdError) as e:
        htd.htd_gmres_solve(s.handle, F, U, 1e-6, 2)
    assert e.value.status == TIMEOUT
    htd.htd_set_wait_limit(s.handle, 0, stall_test=False)
    U.zero_()
    info = htd.htd_gmres_solve(s.handle, F, U, 1e-6, 300)
    assert info["converged"]
    rel = np.linalg.norm(p.F - oracle.Oracle(p).apply_H(U.cpu().numpy())) / np.linalg.norm(p.F)
    assert rel <= 1e-6
    s.close()


def test_a_resident_handle_joining_a_batch_uses_its_blocked_configuration():
    p = _problem((130, 257), T=2)
    q = _problem((64, 64), T=2, seed=5)
    s = htd.Solver(p, precision="mixed", tb_form=htd.TB_RESIDENT)
    t = htd.Solver(q, precision="mixed", tb_form=htd.TB_RESIDENT)
    assert s.params["step_kernel"] == 4 and t.params["step_kernel"] == 4
    Up = s.precond(dev(p.F)).cpu().numpy()
    Uq = t.precond(dev(q.F)).cpu().numpy()
    b = htd.Batch([s, t], [1, 1])
    assert htd.htd_get_params(s.handle)["step_kernel"] in (0, 1)
    Us = b.precond([dev(p.F)[None], dev(q.F)[None]])
    assert np.array_equal(Us[0][0].cpu().numpy(), Up)
    assert np.array_equal(Us[1][0].cpu().numpy(), Uq)
    # the handle alone now runs the blocked (or one-step) kernel: same result
    assert np.array_equal(s.precond(dev(p.F)).cpu().numpy(), Up)
    b.close()
    s.close()
    t.close()


# ---- the plain FP64 recurrence -------------------------------------------------

@pytest.mark.parametrize("n", [(37, 29), (5, 700), (130, 257), (101, 101)])
def test_fp64_resident_equals_the_fp64_one_step_kernel(n):
    """FP64: each exchanged value travels as two tagged 32-bit halves; the
    arithmetic per node is the one-step FP64 kernel's, so the outputs agree bit
    for bit (Table 1 and exact read-out)."""
    p = _problem(n, T=2)
    for mode in ("table1", "exact"):
        s1 = htd.Solver(p, precision="fp64", mode=mode, tblock=1)
        sr = htd.Solver(p, precision="fp64", mode=mode, tb_form=htd.TB_RESIDENT)
        assert s1.params["step_kernel"] == 0 and sr.params["step_kernel"] == 4
        U1 = s1.precond(dev(p.F)).cpu().numpy()
        Ur = sr.precond(dev(p.F)).cpu().numpy()
        s1.close()
        sr.close()
        assert np.isfinite(Ur).all() and np.abs(Ur).max() > 0
        assert np.array_equal(Ur, U1), (mode, float(np.abs(Ur - U1).max()))


def test_fp64_resident_config1_solve_matches_the_oracle():
    """The 101^2 configuration in plain FP64 through the resident kernel: one
    full application within 1e-10 of the oracle, and FGMRES(20) to 1e-6 with the
    one-step kernel's iterates exactly."""
    p = W.config_2d_constant(101)
    sr = htd.Solver(p, precision="fp64", tb_form=htd.TB_RESIDENT)
    assert sr.params["step_kernel"] == 4
    U = sr.precond(dev(p.F)).cpu().numpy()
    ref = oracle.Oracle(p).precond(p.F)
    a, b = U.reshape(-1), ref.reshape(-1)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-10
    assert np.abs(a - b).max() / np.abs(b).max() <= 1e-10
    Ur, ir = sr.solve(dev(p.F), tol=1e-6)
    s1 = htd.Solver(p, precision="fp64", tblock=1)
    U1, i1 = s1.solve(dev(p.F), tol=1e-6)
    assert ir["converged"] and ir["iterations"] == i1["iterations"]
    assert np.array_equal(Ur.cpu().numpy(), U1.cpu().numpy())
    sr.close()
    s1.close()


def test_fp64_resident_wait_runs_out_then_the_handle_solves():
    p = W.config_2d_constant(101)
    s = htd.Solver(p, precision="fp64", tb_form=htd.TB_RESIDENT)
    assert s.params["step_kernel"] == 4
    F = dev(p.F)
    htd.htd_set_wait_limit(s.handle, 1_000_000, stall_test=True)
    U = s.zeros()
    with pytest.raises(htd.HtdError) as e:
        htd.htd_gmres_solve(s.handle, F, U, 1e-6, 2)
    assert e.value.status == TIMEOUT
    htd.htd_set_wait_limit(s.handle, 0, stall_test=False)
    U.zero_()
    assert htd.htd_gmres_solve(s.handle, F, U, 1e-6, 100)["converged"]
    s.close()


# ---- projection read-out inside the resident run --------------------------------

@pytest.mark.parametrize("precision,periods", [("mixed", 1), ("mixed", 2), ("fp64", 1)])
def test_resident_projection_matches_the_oracle(precision, periods):
    """PROJECT mode on the resident kernel: the window's states are accumulated
    inside the launch (compensated sums, compact order, after each window
    step's barrier) and finished by the same kernel as the other paths.
    Against the oracle (2e-5 FP32, 1e-10 FP64) and against the one-step path."""
    p = _problem((129, 161), T=3)
    tol = 2e-5 if precision == "mixed" else 1e-10
    sr = htd.Solver(p, precision=precision, mode="project", proj_periods=periods,
                    tb_form=htd.TB_RESIDENT)
    s1 = htd.Solver(p, precision=precision, mode="project", proj_periods=periods, tblock=1)
    assert sr.params["step_kernel"] == 4 and s1.params["step_kernel"] == 0
    o = oracle.Oracle(p)
    for F in (p.F, W.random_rhs(3, p.n)):
        Ur = sr.precond(dev(F)).cpu().numpy()
        U1 = s1.precond(dev(F)).cpu().numpy()
        ref = o.precond(F, "project", periods)
        a, b = Ur.reshape(-1), ref.reshape(-1)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= tol
        assert np.abs(a - b).max() / np.abs(b).max() <= tol
        c = U1.reshape(-1)
        assert np.linalg.norm(a - c) / np.linalg.norm(c) <= (1e-6 if precision == "mixed"
                                                             else 1e-13)
    sr.close()
    s1.close()
