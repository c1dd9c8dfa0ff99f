"""GPU tests of the projection read-out (mode "project"): Table 1's real-field
run read out as (2 / n_acc) sum_j e^{-i 2 pi j / n_P} u_j over its last whole
periods, summed on the GPU with compensated (Kahan) additions in the
recurrence precision, against the FP64 oracle's plain sum.

Tolerances as in test_gpu_parity: 1e-10 relative L2 in FP64 (summation order
and FMA contraction only), 2e-5 in mixed precision (FP32 recurrence over a few
hundred steps).
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

CASES = [  # (ndim, n, T, periods, precision)
    (2, (45, 37), 3, 1, "fp64"),
    (2, (30, 41), 4, 3, "fp64"),
    (3, (13, 11, 15), 2, 2, "fp64"),
    (2, (150, 131), 3, 1, "mixed"),       # blocked 2-D kernel, then one-step tail
    (2, (97, 140), 4, 2, "mixed"),
    (3, (40, 9, 70), 2, 1, "mixed"),      # streamed 3-D kernel
    (3, (21, 33, 19), 3, 3, "mixed"),     # all steps projected (periods = T)
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{'x'.join(map(str, c[1]))}-T{c[2]}-p{c[3]}-{c[4]}"
                                             for c in CASES])
def test_projection_matches_oracle(case):
    ndim, n, T, periods, precision = case
    p = het_problem(ndim, n, T=T)
    # 2-D mixed: the blocked kernel (depth 4) carries the bulk
    kw = dict(tblock=4) if precision == "mixed" and ndim == 2 else {}
    s = htd.Solver(p, precision=precision, mode="project", proj_periods=periods, **kw)
    if precision == "mixed" and ndim == 2:
        assert s.params["step_kernel"] == 1
    if precision == "mixed" and ndim == 3:
        assert s.params["step_kernel"] == 2
    o = oracle.Oracle(p)
    tol = 1e-10 if precision == "fp64" else 2e-5
    for F in (p.F, W.random_rhs(9, p.n)):
        got = host(s.precond(dev(F))).reshape(-1)
        ref = o.precond(F, "project", periods=periods).reshape(-1)
        assert rel_l2(got, ref) <= tol, rel_l2(got, ref)
    # repeated applications start from zero sums
    again = host(s.precond(dev(p.F))).reshape(-1)
    assert np.array_equal(again, host(s.precond(dev(p.F))).reshape(-1))


def test_projection_differs_from_table1_and_approaches_it_at_steady_state():
    """Both read-outs sample the same run: they agree where the run is close to
    time-harmonic (large T, strong damping) and differ in the transient."""
    p = het_problem(2, (41, 39), T=12, layer=6)
    sp = htd.Solver(p, precision="fp64", mode="project")
    st = htd.Solver(p, precision="fp64", mode="table1")
    a = host(sp.precond(dev(p.F))).reshape(-1)
    b = host(st.precond(dev(p.F))).reshape(-1)
    assert 1e-12 < rel_l2(a, b) < 0.1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fgmres_with_projection_reaches_1e6(precision):
    p = het_problem(2, (70, 66), T=4)
    s = htd.Solver(p, precision=precision, mode="project", proj_periods=2)
    U, info = s.solve(dev(p.F), tol=1e-6, max_iters=200)
    o = oracle.Oracle(p)
    Ug = host(U)
    res = np.linalg.norm(p.F - o.apply_H(Ug)) / np.linalg.norm(p.F)
    assert info["converged"] and res <= 1e-6


def test_projection_batch_equals_single():
    p = het_problem(3, (21, 17, 23), T=2)
    s = htd.Solver(p, precision="mixed", mode="project", proj_periods=2, max_rhs=3)
    F = np.stack([p.F, W.random_rhs(4, p.n), W.random_rhs(5, p.n)]).astype(np.complex128)
    b = htd.Batch([s], [3])
    Ub = host(b.precond([dev(F)])[0])
    for r in range(3):
        assert np.array_equal(Ub[r], host(s.precond(dev(F[r]))))
    b.close()
