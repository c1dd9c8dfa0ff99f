"""GPU parity for the stencil family (HTD_STENCIL_FAMILY) and the tblock option.

The family mixes the Q1 element stiffness with the edge (FD5) stiffness and the
consistent Q1 mass with the lumped mass, per Hamming distance of App. A's cell
kernel.  Only host tables change; the kernels take them as coefficients.  So
the FP64 recurrence must match the oracle at 1e-10 like the built-in stencils,
the mixed form must solve to a true residual of 1e-6 by the oracle's FP64
operator, and the blocked 2-D FP32 kernel must reproduce the one-step kernel
bit for bit whatever the options.tblock choice.
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
from test_gpu_parity import assert_close64, dev, het_problem, host, rel_l2  # noqa: E402

FAMILY = [(0.3, 0.6), (1.0, 0.0), (0.0, 1.0)]
GRIDS = [(2, (45, 37)), (3, (13, 11, 9))]


@pytest.mark.parametrize("ndim,n", GRIDS, ids=["2d", "3d"])
@pytest.mark.parametrize("a,g", FAMILY, ids=[f"a{a}_g{g}" for a, g in FAMILY])
@pytest.mark.parametrize("mode", ["table1", "exact"])
def test_family_fp64_precond_matches_oracle(ndim, n, a, g, mode):
    p = het_problem(ndim, n, T=2)
    s = htd.Solver(p, precision="fp64", mode=mode, stencil="family", stencil_a=a,
                   stencil_gamma=g)
    o = oracle.Oracle(p, "family", stencil_a=a, stencil_gamma=g)
    assert s.params["nP"] == o.params.nP
    for F in (p.F, W.random_rhs(3, p.n)):
        assert_close64(host(s.precond(dev(F))), o.precond(F, mode))
    X = W.random_rhs(4, p.n)
    assert_close64(host(s.apply_H(dev(X))), o.apply_H(X), tol=1e-12)
    s.close()


@pytest.mark.parametrize("ndim,n", GRIDS, ids=["2d", "3d"])
@pytest.mark.parametrize("a,g", FAMILY[:2], ids=[f"a{a}_g{g}" for a, g in FAMILY[:2]])
def test_family_mixed_solve_reaches_tolerance(ndim, n, a, g):
    p = het_problem(ndim, n, T=3)
    s = htd.Solver(p, precision="mixed", stencil="family", stencil_a=a, stencil_gamma=g)
    o = oracle.Oracle(p, "family", stencil_a=a, stencil_gamma=g)
    ref = o.precond(p.F, "table1")
    assert rel_l2(host(s.precond(dev(p.F))).reshape(-1), ref.reshape(-1)) <= 2e-5
    U, info = s.solve(dev(p.F), tol=1e-6, max_iters=200)
    Ub = host(U)
    res = np.linalg.norm(p.F - o.apply_H(Ub)) / np.linalg.norm(p.F)
    assert info["converged"] and res <= 1e-6
    s.close()


@pytest.mark.parametrize("tblock", [4, 8])
def test_tblock_option_matches_one_step_bitwise(tblock):
    """options.tblock = 1 gives one step per launch, 4 or 8 that blocking depth;
    the blocked outputs equal the one-step outputs bit for bit (FAMILY stencil)."""
    p = het_problem(2, (70, 53), T=3)
    kw = dict(precision="mixed", stencil="family", stencil_a=0.3, stencil_gamma=0.6)
    s1 = htd.Solver(p, tblock=1, **kw)
    sb = htd.Solver(p, tblock=tblock, **kw)
    assert s1.params["steps_per_launch"] == 1
    assert sb.params["steps_per_launch"] == tblock
    for F in (p.F, W.random_rhs(8, p.n)):
        assert np.array_equal(host(s1.precond(dev(F))), host(sb.precond(dev(F))))
    s1.close()
    sb.close()
