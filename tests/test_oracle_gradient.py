"""Pin of the oracle's misfit gradient against central finite differences of the
oracle's own misfit (both from direct solves): the adjoint formula, the mass
weights in dRe H/dm and the omega factors must agree with the derivative of
J = 1/2 sum_s ||P H^{-1} F_s - d_s||^2."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_16861_gb300 import workloads as W


def small_setup(ndim, n, nsrc=2, seed=3, stencil="q1mix"):
    n = tuple(n)
    h = 1.0 / (max(n) - 1)
    cells = tuple(m + 1 for m in n)
    g = W.gaussian_random_field(seed, cells, 2.0)
    c = np.clip(2.0 + 0.4 * g, 1.2, 3.0)
    omega = 2 * math.pi * c.min() / (7 * h)
    R = W.damping_profile(ndim, n, 2, 2.0 * omega)
    F = W.seeded_sources(seed + 5, ndim, n, h, nsrc, 2)
    rec = np.arange(0, int(np.prod(n)), 7, dtype=np.int64)
    d = 1e-3 * (W.white_noise(seed + 9, (nsrc, rec.size)) + 1j * W.white_noise(seed + 10, (nsrc, rec.size)))
    p = W.Problem("g", ndim, n, h, c, R, omega, F[0], 2, 0.25)
    return p, F, rec, d


def misfit(p, F, rec, d, c=None, R=None):
    q = W.Problem(p.name, p.ndim, p.n, p.h, p.c_cell if c is None else c,
                  p.R_node if R is None else R, p.omega, p.F, p.T, p.rho)
    return oracle.Oracle(q).grad(F, rec, d)[0]


@pytest.mark.parametrize("ndim,n", [(2, (11, 9)), (3, (5, 6, 4))])
def test_gradient_matches_central_differences(ndim, n):
    p, F, rec, d = small_setup(ndim, n)
    J, gm, gR = oracle.Oracle(p).grad(F, rec, d)
    m = p.c_cell ** -2.0
    rng = np.random.default_rng(1)
    for _ in range(3):
        v = rng.standard_normal(m.shape) * m
        eps = 1e-5
        Jp = misfit(p, F, rec, d, c=(m + eps * v) ** -0.5)
        Jm = misfit(p, F, rec, d, c=(m - eps * v) ** -0.5)
        fd = (Jp - Jm) / (2 * eps)
        assert np.sum(gm * v) == pytest.approx(fd, rel=1e-6)
        w = rng.standard_normal(p.n) * (p.R_node.max() + 1.0)
        Jp = misfit(p, F, rec, d, R=p.R_node + eps * w)
        Jm = misfit(p, F, rec, d, R=p.R_node - eps * w)
        fd = (Jp - Jm) / (2 * eps)
        assert np.sum(gR * w) == pytest.approx(fd, rel=1e-6)


def test_misfit_is_zero_for_exact_data_and_gradient_vanishes():
    p, F, rec, _ = small_setup(2, (9, 8))
    o = oracle.Oracle(p)
    U = np.stack([o.direct_solve(f).reshape(-1) for f in F])
    d = U[:, rec]
    J, gm, gR = o.grad(F, rec, d)
    assert J < 1e-20 and np.abs(gm).max() < 1e-8 and np.abs(gR).max() < 1e-8


# ---- gradient through the recurrence (the preconditioner's own solution) ------

def misfit_td(p, base, F, rec, d, mode, c=None, R=None):
    """Misfit of the perturbed model with the base model's omega, dt and n_P."""
    q = W.Problem(p.name, p.ndim, p.n, p.h, p.c_cell if c is None else c,
                  p.R_node if R is None else R, p.omega, p.F, p.T, p.rho)
    return oracle.Oracle(q).with_params(base).grad_td(F, rec, d, mode)[0]


@pytest.mark.parametrize("ndim,n,mode", [(2, (11, 9), "table1"), (2, (10, 12), "exact"),
                                         (3, (5, 6, 4), "table1")])
def test_recurrence_gradient_matches_central_differences(ndim, n, mode):
    """J = 1/2 sum_s ||P(P F_s) - d_s||^2 with P the preconditioner itself: the
    reverse-time adjoint recurrence and the K / L derivatives must agree with
    central differences of the same misfit (recurrence parameters frozen)."""
    p, F, rec, d = small_setup(ndim, n)
    base = oracle.Oracle(p)
    J, gm, gR = base.grad_td(F, rec, d, mode)
    assert J > 0
    m = p.c_cell ** -2.0
    rng = np.random.default_rng(2)
    for _ in range(3):
        v = rng.standard_normal(m.shape) * m
        eps = 1e-5
        fd = (misfit_td(p, base, F, rec, d, mode, c=(m + eps * v) ** -0.5)
              - misfit_td(p, base, F, rec, d, mode, c=(m - eps * v) ** -0.5)) / (2 * eps)
        assert np.sum(gm * v) == pytest.approx(fd, rel=1e-6)
        w = rng.standard_normal(p.n) * (p.R_node.max() + 1.0)
        fd = (misfit_td(p, base, F, rec, d, mode, R=p.R_node + eps * w)
              - misfit_td(p, base, F, rec, d, mode, R=p.R_node - eps * w)) / (2 * eps)
        assert np.sum(gR * w) == pytest.approx(fd, rel=1e-6)


def test_recurrence_misfit_uses_the_preconditioner_output():
    """J of the recurrence gradient is the misfit of P F (not of H^{-1} F): zero
    for data taken from P F itself, with a vanishing gradient."""
    p, F, rec, _ = small_setup(2, (9, 8))
    o = oracle.Oracle(p)
    d = np.stack([o.precond(f, "table1").reshape(-1)[rec] for f in F])
    J, gm, gR = o.grad_td(F, rec, d, "table1")
    assert J < 1e-24 and np.abs(gm).max() < 1e-10 and np.abs(gR).max() < 1e-10
