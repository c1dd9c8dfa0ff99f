"""Pins of the oracle's backward-differences scheme I_abd (Sec. 6) and of the
non-diagonal (cell-mass) damping it is meant for, against identities of the
paper and the mathematics: the time-harmonic reproduction of the proposition
of Sec. 6.1 (exact one-step identity), the energy of Sec. 6.2 (conserved
without damping, non-increasing with it), the stability conditions at the
chosen parameters (dense eigenvalues on tiny grids), symmetry / positivity /
row sums of the damping operator, and convergence of S_T^abd to H^{-1}."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_16861_gb300 import workloads as W
from test_oracle_pins import make_problem


def dense_H(o):
    return o.H_sparse().toarray()


def abd_problem(*args, **kw):
    """make_problem with the absorbing layer at R0 = omega instead of 2 omega: the
    backward-differences scheme needs lambda_max(Im H) below about 2 omega^2
    (its CFL-type condition of Sec. 6.1 tends to 2 lambda_max(Im H) / k_max^2 < 4
    for small omega dt)."""
    p = make_problem(*args, **kw)
    return W.Problem(p.name, p.ndim, p.n, p.h, p.c_cell, 0.5 * p.R_node, p.omega, p.F, p.T,
                     p.rho)


@pytest.mark.parametrize("d,n", [(2, (9, 8)), (3, (5, 4, 6))])
@pytest.mark.parametrize("damping", ["node", "cell"])
def test_abd_reproduces_time_harmonic_solutions_exactly(d, n, damping):
    """With H U = F, u_j = e^{i omega j dt} U and f_j = e^{i omega j dt} F satisfy
    u_{n+1} = I_abd(u_n, u_{n-1}, f_n) exactly (to rounding), for the scheme's
    own omega, dt, alpha, beta and either damping form."""
    p = abd_problem(d, n, het=True, layer=2)
    o = oracle.Oracle(p, integrator="abd", damping=damping)
    q = o.params
    rng = np.random.default_rng(3)
    U = (rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n))
    F = o.apply_H(U)
    e = lambda j: np.exp(1j * q.omega * j * q.dt)
    j = 7
    got = o.abd_step(e(j) * U, e(j - 1) * U, e(j) * F)
    assert np.abs(got - e(j + 1) * U).max() <= 1e-10 * np.abs(U).max()


@pytest.mark.parametrize("stencil", ["q1mix", "fd5"])
def test_cell_damping_operator(stencil):
    """Cell-mass damping: symmetric, positive semidefinite, equal to omega R on
    interior constants for constant R; with the lumped mass (FD5) diagonal."""
    n = (9, 8)
    p = make_problem(2, n, R=3.0)
    o = oracle.Oracle(p, stencil, damping="cell")
    Hm = dense_H(o)
    B = Hm.imag
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(B).min() >= -1e-10 * np.abs(B).max()
    ones = np.ones(p.n)
    v = o.apply_imH(ones)
    assert np.allclose(v[1:-1, 1:-1], p.omega * 3.0, rtol=1e-13)
    assert np.allclose(B, np.diag(np.diag(B))) == (stencil == "fd5")
    # apply_imH is the operator that assembles into Im H
    u = np.random.default_rng(1).standard_normal(p.n)
    assert np.allclose(o.apply_imH(u).reshape(-1), B @ u.reshape(-1), rtol=1e-12, atol=0)


@pytest.mark.parametrize("damping", ["node", "cell"])
def test_abd_parameters_satisfy_the_stability_conditions(damping):
    """K positive semidefinite and 4 I - K - 2 L positive definite at the chosen
    omega, dt (Sec. 6.1), by dense eigenvalues."""
    p = abd_problem(2, (10, 9), het=True, layer=3)
    o = oracle.Oracle(p, integrator="abd", damping=damping)
    q = o.params
    Hm = dense_H(o)
    A = Hm.real + q.omega ** 2 * np.eye(p.N)
    B = Hm.imag / q.omega
    th = q.omega * q.dt
    K = q.dt ** 2 / q.alpha * A - q.dt * q.beta * (1 - math.cos(th)) / q.alpha * B
    L = q.beta * q.dt / q.alpha * B
    assert np.linalg.eigvalsh(K).min() >= -1e-10
    assert np.linalg.eigvalsh(4 * np.eye(p.N) - K - 2 * L).min() > 0
    assert q.integrator == 1 and q.nP % 4 == 0


@pytest.mark.parametrize("R", ["zero", "layer"])
def test_abd_energy(R):
    """E_bd = <D,(4I-K)D> + <S,K S> - 2<D,L D> (D = u_n - u_{n-1}, S = u_n + u_{n-1})
    is conserved by the homogeneous recursion without damping and does not
    grow with it (Sec. 6.2)."""
    p = abd_problem(2, (10, 9), het=True, layer=3, R=R)
    o = oracle.Oracle(p, integrator="abd", damping="cell")
    q = o.params
    Hm = dense_H(o)
    A = Hm.real + q.omega ** 2 * np.eye(p.N)
    B = Hm.imag / q.omega
    th = q.omega * q.dt
    K = q.dt ** 2 / q.alpha * A - q.dt * q.beta * (1 - math.cos(th)) / q.alpha * B
    L = q.beta * q.dt / q.alpha * B
    I4 = 4 * np.eye(p.N)

    def E(un, um):
        D, S = un - um, un + um
        return D @ (I4 - K) @ D + S @ K @ S - 2 * D @ L @ D

    rng = np.random.default_rng(4)
    um = rng.standard_normal(p.N)
    un = rng.standard_normal(p.N)
    zero = np.zeros(p.N, dtype=complex)
    Es = [E(un, um)]
    for _ in range(60):
        up = o.abd_step(un.astype(complex), um.astype(complex), zero).real.reshape(-1)
        um, un = un, up
        Es.append(E(un, um))
    Es = np.array(Es)
    if R == "zero":
        assert np.abs(Es - Es[0]).max() <= 1e-11 * abs(Es[0])
    else:
        assert np.all(np.diff(Es) <= 1e-11 * Es[0]) and Es[-1] < Es[0]


def test_abd_ST_converges_to_Hinv_with_cell_damping():
    p = abd_problem(2, (21, 21), c=1.0, layer=5, ppw=8)
    o0 = oracle.Oracle(p, integrator="abd", damping="cell")
    U = o0.direct_solve(p.F)
    errs = []
    for T in (2, 4, 8, 16, 32):
        o = oracle.Oracle(p, T=T, integrator="abd", damping="cell")
        errs.append(np.linalg.norm(o.precond(p.F, "exact") - U) / np.linalg.norm(U))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * errs[0]


def test_acd_refuses_non_diagonal_damping():
    p = make_problem(2, (9, 8))
    o = oracle.Oracle(p, damping="cell")
    with pytest.raises(ValueError):
        o.precond(p.F)
