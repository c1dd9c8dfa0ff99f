"""GPU tests of the backward-differences scheme I_abd (Sec. 6) and of the
non-diagonal cell-mass damping it makes usable, against the FP64 oracle.

Tolerances as in test_gpu_parity: 1e-10 relative L2 in FP64, 5e-5 in mixed
precision (FP32 recurrence; I_abd's smaller time step means more steps per
period than I_acd), 1e-12 for the FP64 operator.
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


def abd_problem(ndim, n, T=2, layer=3, seed=11):
    """het_problem with its damping scaled by 1/4: I_abd needs lambda_max(Im H)
    below about 2 k_max^2 (Sec. 6.1), and the layer profile adds up over the
    axes at edges and corners."""
    p = het_problem(ndim, n, T=T, layer=layer, seed=seed)
    return W.Problem(p.name, p.ndim, p.n, p.h, p.c_cell, 0.25 * p.R_node, p.omega, p.F, p.T,
                     p.rho)


CASES = [  # (ndim, n, damping, mode, precision)
    (2, (41, 37), "node", "table1", "fp64"),
    (2, (33, 45), "cell", "table1", "fp64"),
    (2, (30, 28), "cell", "exact", "fp64"),
    (3, (13, 11, 15), "cell", "table1", "fp64"),
    (3, (12, 14, 9), "node", "exact", "fp64"),
    (2, (70, 66), "cell", "table1", "mixed"),
    (3, (21, 17, 19), "cell", "table1", "mixed"),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{'x'.join(map(str, c[1]))}-{c[2]}-{c[3]}-{c[4]}"
                                             for c in CASES])
def test_abd_precond_matches_oracle(case):
    ndim, n, damping, mode, precision = case
    p = abd_problem(ndim, n)
    s = htd.Solver(p, precision=precision, mode=mode, integrator="abd", damping=damping)
    o = oracle.Oracle(p, integrator="abd", damping=damping)
    assert s.params["step_kernel"] == 3 and s.params["nP"] == o.params.nP
    tol = 1e-10 if precision == "fp64" else 5e-5
    for F in (p.F, W.random_rhs(12, p.n)):
        got = host(s.precond(dev(F))).reshape(-1)
        ref = o.precond(F, mode).reshape(-1)
        assert rel_l2(got, ref) <= tol, rel_l2(got, ref)


@pytest.mark.parametrize("ndim,n", [(2, (29, 31)), (3, (9, 12, 10))])
def test_cell_damping_operator_matches_oracle(ndim, n):
    p = abd_problem(ndim, n)
    s = htd.Solver(p, precision="fp64", integrator="abd", damping="cell")
    o = oracle.Oracle(p, integrator="abd", damping="cell")
    X = W.random_rhs(5, p.n)
    got = host(s.apply_H(dev(X))).reshape(-1)
    ref = o.apply_H(X).reshape(-1)
    assert rel_l2(got, ref) <= 1e-12


def test_projection_with_abd():
    p = abd_problem(2, (40, 36), T=3)
    s = htd.Solver(p, precision="fp64", mode="project", proj_periods=2, integrator="abd",
                   damping="cell")
    o = oracle.Oracle(p, integrator="abd", damping="cell")
    got = host(s.precond(dev(p.F))).reshape(-1)
    assert rel_l2(got, o.precond(p.F, "project", periods=2).reshape(-1)) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fgmres_with_abd_and_cell_damping_reaches_1e6(precision):
    p = abd_problem(2, (60, 57), T=4)
    s = htd.Solver(p, precision=precision, integrator="abd", damping="cell")
    U, info = s.solve(dev(p.F), tol=1e-6, max_iters=300)
    o = oracle.Oracle(p, integrator="abd", damping="cell")
    Ug = host(U)
    res = np.linalg.norm(p.F - o.apply_H(Ug)) / np.linalg.norm(p.F)
    assert info["converged"] and res <= 1e-6
    Ud = o.direct_solve(p.F)
    assert rel_l2(Ug.reshape(-1), Ud.reshape(-1)) <= 1e-4


def test_abd_batch_equals_single():
    p = abd_problem(3, (13, 15, 11))
    s = htd.Solver(p, precision="mixed", integrator="abd", damping="cell", max_rhs=2)
    F = np.stack([p.F, W.random_rhs(6, p.n)]).astype(np.complex128)
    b = htd.Batch([s], [2])
    Ub = host(b.precond([dev(F)])[0])
    for r in range(2):
        assert np.array_equal(Ub[r], host(s.precond(dev(F[r]))))
    b.close()


def test_gradients_reject_what_they_do_not_cover():
    p = abd_problem(2, (20, 18))
    F = dev(p.F[None])
    rec = np.arange(5, dtype=np.int64)
    d = dev(np.zeros((1, 5)))
    sc = htd.Solver(p, precision="fp64", integrator="abd", damping="cell")
    with pytest.raises(htd.HtdError):
        sc.grad(F, rec, d)                        # dH/dR is not diagonal
    sn = htd.Solver(p, precision="fp64", integrator="abd")
    with pytest.raises(htd.HtdError):
        sn.grad_td(F, rec, d)                     # the recurrence adjoint covers I_acd
