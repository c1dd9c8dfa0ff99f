"""GPU gradient (htd_grad, adjoint state) against the FP64 oracle's gradient
(direct solves) on small grids, and against central finite differences of the
GPU misfit at the full 512 x 512, 8-source configuration.

Tolerances: the GPU solves run to a true relative residual of 1e-11 (small
grids) / 1e-10 (512^2); misfit and gradient then agree with the exact-solve
oracle to about cond(H) * 1e-11, tested at 1e-7 (misfit) and 1e-5 (relative L2
of the gradient).  Finite differences: relative error < 1e-4 along smooth
random directions.
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


def small_case(ndim, n, nsrc, seed=5):
    n = tuple(n)
    h = 1.0 / (max(n) - 1)
    cells = tuple(m + 1 for m in n)
    g = W.gaussian_random_field(seed, cells, 3.0)
    c = np.clip(2.0 + 0.4 * g, 1.2, 3.0)
    omega = 2 * math.pi * c.min() / (8 * h)
    R = W.damping_profile(ndim, n, 3, 2.0 * omega)
    F = W.seeded_sources(seed + 1, ndim, n, h, nsrc, 3)
    rec = np.arange(3 * n[-1], 4 * n[-1], dtype=np.int64)
    d = 1e-2 * (W.white_noise(seed + 2, (nsrc, rec.size)) + 1j * W.white_noise(seed + 3, (nsrc, rec.size)))
    p = W.Problem("g", ndim, n, h, c, R, omega, F[0], 3, 0.25)
    return p, F, rec, d


@pytest.mark.parametrize("ndim,n", [(2, (41, 37)), (3, (13, 11, 15))])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_matches_oracle(ndim, n, precision):
    p, F, rec, d = small_case(ndim, n, 3)
    s = htd.Solver(p, precision=precision)
    J, gm, gR, info = s.grad(dev(F), rec, dev(d), tol=1e-11, max_iters=600)
    Jo, gmo, gRo = oracle.Oracle(p).grad(F, rec, d)
    assert J == pytest.approx(Jo, rel=1e-7)
    gm, gR = gm.cpu().numpy(), gR.cpu().numpy()
    assert np.linalg.norm(gm - gmo) <= 1e-5 * np.linalg.norm(gmo)
    assert np.linalg.norm(gR - gRo) <= 1e-5 * np.linalg.norm(gRo)
    # misfit only (no adjoint solves)
    J2, g1, g2, _ = s.grad(dev(F), rec, dev(d), tol=1e-11, max_iters=600, want_grad=False)
    assert g1 is None and J2 == pytest.approx(J, rel=1e-9)


def test_gradient_rejects_bad_receivers():
    p, F, rec, d = small_case(2, (21, 19), 1)
    s = htd.Solver(p)
    bad = rec.copy()
    bad[0] = p.N
    with pytest.raises(htd.HtdError) as e:
        s.grad(dev(F), bad, dev(d))
    assert e.value.status == 1


def test_config_adjoint_512_finite_differences():
    """2-D 512^2 smooth random c, 8 seeded point sources, receivers on the first
    row inside the top absorbing layer, data from the model with a 5 % Gaussian
    blob; the gradient along smooth directions against central differences."""
    from paper_2006_16861_gb300.autograd import receiver_misfit
    st = W.config_adjoint(512)
    p = st.prob
    F = dev(st.F)
    # data d_s = P U_s(c_true), computed with the library (this test compares the
    # GPU gradient with GPU misfits only; the oracle is not involved at this size)
    pt = W.Problem(p.name, 2, p.n, p.h, st.c_true, p.R_node, p.omega, p.F, p.T, p.rho)
    strue = htd.Solver(pt, precision="mixed")
    d = []
    for s in range(st.F.shape[0]):
        U, _ = strue.solve(F[s].contiguous(), tol=1e-10, max_iters=600)
        d.append(U.reshape(-1)[torch.from_numpy(st.rec_idx).cuda()])
    d = torch.stack(d).contiguous()
    strue.close()
    m = torch.from_numpy(p.c_cell ** -2.0).requires_grad_(True)
    R = torch.from_numpy(p.R_node.copy()).requires_grad_(True)
    J = receiver_misfit(m, R, p, F, st.rec_idx, d, tol=1e-10)
    J.backward()
    gm, gR = m.grad.numpy(), R.grad.numpy()
    assert J.item() > 0 and np.isfinite(gm).all() and np.isfinite(gR).all()
    n1 = p.n[0] + 1
    xs = (np.arange(n1) - 0.5) * p.h
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    # localized smooth directions (a global change of m shifts the phase over the
    # whole 64-wavelength domain and puts central differences in the nonlinear range)
    dirs_m = [np.exp(-((X - 0.4) ** 2 + (Y - 0.6) ** 2) / 0.02),
              np.exp(-((X - 0.7) ** 2 + (Y - 0.3) ** 2) / 0.005)]
    for v in dirs_m:
        v = v * m.detach().numpy()
        eps = 1e-3
        Jp = receiver_misfit(torch.from_numpy(m.detach().numpy() + eps * v), R.detach(), p, F,
                             st.rec_idx, d, tol=1e-10).item()
        Jm = receiver_misfit(torch.from_numpy(m.detach().numpy() - eps * v), R.detach(), p, F,
                             st.rec_idx, d, tol=1e-10).item()
        fd = (Jp - Jm) / (2 * eps)
        assert abs(np.sum(gm * v) - fd) <= 1e-4 * abs(fd)
    # a bump inside the top absorbing layer, proportional to R so that R stays >= 0
    w = p.R_node * np.exp(-((X[:-1, :-1] - 0.02) ** 2 + (Y[:-1, :-1] - 0.5) ** 2) / 0.01)
    eps = 1e-3
    Jp = receiver_misfit(m.detach(), torch.from_numpy(p.R_node + eps * w), p, F, st.rec_idx, d,
                         tol=1e-10).item()
    Jm = receiver_misfit(m.detach(), torch.from_numpy(p.R_node - eps * w), p, F, st.rec_idx, d,
                         tol=1e-10).item()
    fd = (Jp - Jm) / (2 * eps)
    assert abs(np.sum(gR * w) - fd) <= 1e-4 * abs(fd)
