"""GPU tests of the batch calls (htd_batch_*): several right-hand sides of one
handle and several handles of different sizes, kernels and step counts, run
as one batch.

A batch only schedules; every system keeps the arithmetic of the single-system
calls.  So the batched preconditioner must reproduce each handle's own
htd_apply_precond bit for bit (same kernels, same configuration, only the
right-hand-side slot differs), the batched FGMRES must take the same
iterations and give the same solution as htd_gmres_solve per system, and
both are tied to the FP64 oracle as in test_gpu_parity.
"""
import numpy as np
import pytest

import oracle
from paper_2006_16861_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2006_16861_gb300 import htd  # noqa: E402
from test_gpu_parity import dev, het_problem, host, rel_l2  # noqa: E402


def rhs_stack(p, nrhs, seed):
    """nrhs right-hand sides: the problem's point source, then seeded random fields."""
    F = [p.F] + [W.random_rhs(seed + k, p.n) for k in range(nrhs - 1)]
    return np.stack(F).astype(np.complex128)


CASES = [  # (ndim, n, precision, mode)
    (2, (45, 37), "fp64", "table1"),
    (2, (70, 66), "mixed", "table1"),
    (2, (41, 29), "mixed", "exact"),
    (3, (13, 17, 19), "fp64", "table1"),
    (3, (21, 70, 33), "mixed", "table1"),
    (3, (11, 9, 15), "mixed", "exact"),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{'x'.join(map(str, c[1]))}-{c[2]}-{c[3]}"
                                             for c in CASES])
def test_rhs_batch_precond_equals_single(case):
    """Three right-hand sides of one handle (max_rhs 4, so one slot idles) in one
    batched application: each equals the handle's single application exactly,
    and the FP64 ones equal the oracle to 1e-10."""
    ndim, n, precision, mode = case
    p = het_problem(ndim, n, T=2)
    s = htd.Solver(p, precision=precision, mode=mode, max_rhs=4)
    F = rhs_stack(p, 3, 40)
    b = htd.Batch([s], [3])
    U = b.precond([dev(F)])[0]
    Ub = host(U)
    o = oracle.Oracle(p)
    for r in range(3):
        single = host(s.precond(dev(F[r])))
        assert np.array_equal(Ub[r], single), rel_l2(Ub[r].reshape(-1), single.reshape(-1))
        ref = o.precond(F[r], mode).reshape(-1)
        tol = 1e-10 if precision == "fp64" else 2e-5
        assert rel_l2(Ub[r].reshape(-1), ref) <= tol
    b.close()


def test_multi_instance_batch_precond():
    """Handles of different dimension, size, precision and step count (a 3-D
    handle with two right-hand sides, 2-D handles with one) in one graph launch:
    each output equals that handle's own application."""
    setup = W.config_batched(n3=20, nsrc=2, ninst=3, side_lo=30, side_hi=90)
    precisions = ["mixed", "mixed", "fp64", "mixed"]
    solvers = [htd.Solver(p, precision=pr, max_rhs=F.shape[0])
               for p, F, pr in zip(setup.probs, setup.F, precisions)]
    assert len({s.params["steps"] for s in solvers}) > 1      # different step counts
    b = htd.Batch(solvers, [F.shape[0] for F in setup.F])
    Us = b.precond([dev(F) for F in setup.F])
    for s, F, U in zip(solvers, setup.F, Us):
        Ub = host(U)
        for r in range(F.shape[0]):
            single = host(s.precond(dev(F[r])))
            assert np.array_equal(Ub[r], single)
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_gmres_matches_single_solves(precision):
    """Lockstep FGMRES over a 3-D handle with three right-hand sides (which
    converge after different numbers of steps, so slots go idle) and two 2-D
    handles: per system the same iteration count as htd_gmres_solve, the same
    solution bit for bit (identical operations; the host-side Givens and
    triangular solve are shared code built without FMA contraction), and a true
    residual <= 1e-6 by the oracle's FP64 operator."""
    setup = W.config_batched(n3=18, nsrc=2, ninst=2, side_lo=40, side_hi=80)
    Fs = [np.concatenate([F, W.random_rhs(7, F.shape[1:])[None]]) if k == 0 else F
          for k, F in enumerate(setup.F)]
    solvers = [htd.Solver(p, precision=precision, max_rhs=F.shape[0], restart=8)
               for p, F in zip(setup.probs, Fs)]
    b = htd.Batch(solvers, [F.shape[0] for F in Fs])
    Us, infos = b.solve([dev(F) for F in Fs], tol=1e-6, max_iters=200)
    k = 0
    its = []
    for s, p, F, U in zip(solvers, setup.probs, Fs, Us):
        Ub = host(U)
        o = oracle.Oracle(p)
        for r in range(F.shape[0]):
            info = infos[k]
            k += 1
            Us1, info1 = s.solve(dev(F[r]), tol=1e-6, max_iters=200)
            assert info["converged"] and info1["converged"]
            assert info["iterations"] == info1["iterations"]
            its.append(info["iterations"])
            assert np.array_equal(Ub[r], host(Us1))
            res = np.linalg.norm(F[r] - o.apply_H(Ub[r])) / np.linalg.norm(F[r])
            assert res <= 1e-6
    assert len(set(its)) > 1                  # systems left the batch at different steps
    b.close()


def test_batch_rejects_bad_arguments():
    p = het_problem(2, (20, 22), T=2)
    s1 = htd.Solver(p, precision="mixed", max_rhs=2)
    s2 = htd.Solver(p, precision="mixed", krylov="left")
    for handles, nrhs in (([s1.handle, s1.handle], [1, 1]),   # repeated handle
                          ([s1.handle], [3]),                  # more rhs than max_rhs
                          ([s1.handle], [0]),
                          ([s2.handle], [1])):                 # left GMRES
        with pytest.raises(htd.HtdError) as e:
            htd.htd_batch_create(handles, nrhs)
        assert e.value.status == 1
    b = htd.Batch([s1], [2])
    F = dev(rhs_stack(p, 2, 3))
    with pytest.raises(htd.HtdError) as e:
        htd.htd_batch_gmres_solve(b.handle, [F], [F], 1e-6, 10, 2)     # F aliases U
    assert e.value.status == 1
    b.close()


def test_config_batched_full_size():
    """The full batched configuration (3-D 128^3 layered model with 32 seeded
    point sources as right-hand sides of one handle, plus 64 2-D instances with
    sides in [200, 1000]) in the launch configuration the benchmark times: one
    lockstep FGMRES(20) solve of all 96 systems; every solution reaches a true
    relative residual <= 1e-6 by the oracle's FP64 operator."""
    setup = W.config_batched()
    solvers = [htd.Solver(p, precision="mixed", max_rhs=F.shape[0], restart=20)
               for p, F in zip(setup.probs, setup.F)]
    b = htd.Batch(solvers, [F.shape[0] for F in setup.F])
    Us, infos = b.solve([dev(F) for F in setup.F], tol=1e-6, max_iters=400)
    assert len(infos) == 96
    k = 0
    for p, F, U in zip(setup.probs, setup.F, Us):
        Ub = host(U)
        o = oracle.Oracle(p)
        for r in range(F.shape[0]):
            assert infos[k]["converged"], (k, infos[k])
            res = np.linalg.norm(F[r] - o.apply_H(Ub[r])) / np.linalg.norm(F[r])
            assert res <= 1e-6, (k, res)
            k += 1
    b.close()
    for s in solvers:
        s.close()


GROUP_SIZES = [(1, 7), (3, 2), (37, 45), (130, 67), (64, 300), (101, 101), (211, 97)]


def test_group_launch_equals_per_handle_launches():
    """2-D FP32 handles of many sizes (ragged; one tile of 1 x 7 and 3 x 2 nodes;
    up to 5 x 2 tiles), step counts and right-hand-side slots (one handle with
    three of four slots used, one with two, one in exact mode) run by the one
    persistent group launch: every output equals that handle's own
    application bit for bit, on two applications in a row (graph replay), and
    a 3-D handle in the same batch runs beside the group as its own child graph."""
    Ts = [2, 2, 3, 2, 3, 2, 4]
    probs = [het_problem(2, n, T=T) for n, T in zip(GROUP_SIZES, Ts)]
    modes = ["table1", "table1", "table1", "table1", "table1", "exact", "table1"]
    nrhs = [1, 1, 3, 1, 2, 1, 1]
    caps = [1, 1, 4, 1, 2, 1, 1]
    solvers = [htd.Solver(p, precision="mixed", mode=m, max_rhs=c)
               for p, m, c in zip(probs, modes, caps)]
    p3 = het_problem(3, (21, 17, 19), T=2)
    solvers.append(htd.Solver(p3, precision="mixed", max_rhs=2))
    probs.append(p3)
    nrhs.append(2)
    assert len({s.params["steps"] for s in solvers}) > 2
    b = htd.Batch(solvers, nrhs)
    b.set_form(2)                                  # the group's persistent launch
    Fs = [rhs_stack(p, r, 60 + 7 * k) for k, (p, r) in enumerate(zip(probs, nrhs))]
    for rep in range(2):
        Us = b.precond([dev(F) for F in Fs])
        if rep == 0:
            d = b.describe()
            assert d["grouped"] == 7 and d["group_ctas"] > 0 and d["group_steps_per_task"] in (4, 8)
            assert d["form"] == 2
        for s, F, U in zip(solvers, Fs, Us):
            Ub = host(U)
            for r in range(F.shape[0]):
                single = host(s.precond(dev(F[r])))
                assert np.array_equal(Ub[r], single), rel_l2(Ub[r].reshape(-1), single.reshape(-1))
    b.close()
    for s in solvers:
        s.close()


def test_group_launch_solve_equals_single_solves():
    """Lockstep FGMRES over five 2-D FP32 handles of different sizes and step
    counts run by the group launch (systems leave the batch at different
    iterations, so the group's slots go idle one by one): the same iterations
    and the same solutions bit for bit as htd_gmres_solve per handle."""
    # five 2-D instances of the batched workload's recipe (smooth random c, a
    # layer of 4 % of the side, T = side in wavelengths), sides 60 .. 200
    probs = W.config_batched(n3=12, nsrc=1, ninst=5, side_lo=60, side_hi=200).probs[1:]
    assert len({p.n for p in probs}) > 1
    solvers = [htd.Solver(p, precision="mixed", restart=10) for p in probs]
    b = htd.Batch(solvers, [1] * len(solvers))
    singles = [s.solve(dev(p.F), tol=1e-7, max_iters=300) for s, p in zip(solvers, probs)]
    # the group form throughout, then the form chosen by timing the first rounds
    for form in (2, 0):
        b.set_form(form)
        Us, infos = b.solve([dev(p.F[None]) for p in probs], tol=1e-7, max_iters=300)
        d = b.describe()
        assert d["grouped"] == len(solvers)
        if form == 2:
            assert d["form"] == 2
        else:
            assert d["form"] in (1, 2)
            assert d["ns_per_update_plain"] > 0 and d["ns_per_update_group"] > 0
        its = []
        for (U1, info1), U, info in zip(singles, Us, infos):
            assert info["converged"] and info1["converged"]
            assert info["iterations"] == info1["iterations"]
            its.append(info["iterations"])
            assert np.array_equal(host(U)[0], host(U1))
        assert len(set(its)) > 1
    b.close()


@pytest.mark.parametrize("nrhs", [2, 5, 6])
def test_two_rhs_per_cta_equals_one(nrhs):
    """The streamed 3-D pair kernel with two right-hand sides per CTA (q*kappa, d
    and every stencil coefficient loaded or computed once for both) gives each
    right-hand side the bits of one-per-CTA launches and of the handle's own
    single application; an odd count leaves the last CTA with one, and a
    handle with six slots carrying fewer leaves slots idle."""
    p = het_problem(3, (45, 37, 29), T=2)
    s1 = htd.Solver(p, precision="mixed", max_rhs=6, s3_rhs_per_cta=1)
    s2 = htd.Solver(p, precision="mixed", max_rhs=6, s3_rhs_per_cta=2)
    assert s1.params["rhs_per_cta"] == 1 and s2.params["rhs_per_cta"] == 2
    assert s1.params["step_kernel"] == s2.params["step_kernel"] == 2
    F = rhs_stack(p, nrhs, 90)
    b1 = htd.Batch([s1], [nrhs])
    b2 = htd.Batch([s2], [nrhs])
    for rep in range(2):
        U1 = host(b1.precond([dev(F)])[0])
        U2 = host(b2.precond([dev(F)])[0])
        assert np.array_equal(U1, U2), rel_l2(U1.reshape(-1), U2.reshape(-1))
    for r in range(nrhs):
        assert np.array_equal(U2[r], host(s1.precond(dev(F[r]))))
    b1.close()
    b2.close()


def test_rhs_per_cta_is_tuned_for_multi_rhs_handles():
    """A 3-D handle with several right-hand sides times one and two per CTA at
    create and reports its choice; a one-rhs handle uses one."""
    p = het_problem(3, (64, 48, 40), T=2)
    s = htd.Solver(p, precision="mixed", max_rhs=8)
    assert s.params["rhs_per_cta"] in (1, 2)
    s1 = htd.Solver(p, precision="mixed")
    assert s1.params["rhs_per_cta"] == 1
    F = rhs_stack(p, 8, 120)
    b = htd.Batch([s], [8])
    Ub = host(b.precond([dev(F)])[0])
    for r in (0, 7):
        assert np.array_equal(Ub[r], host(s1.precond(dev(F[r]))))
    b.close()
