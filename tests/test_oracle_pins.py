"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself: a
closed form, a textbook derivation done independently in the test (Gauss
quadrature of Q1 elements, tensor-product sine eigenvalues), a library routine
(scipy spsolve / gmres, numpy eigvalsh), an exact identity of the paper
(Prop. 1, Theorem 1's energy identity, Theorem 3's Green's-function sum) or a
number the paper prints (tests/golden/paper_facts.json).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import oracle
from paper_2006_16861_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def make_problem(ndim, n, c=1.0, ppw=6.0, R="layer", layer=4, T=4, rho=0.25, seed=7,
                 het=False):
    n = (n,) * ndim if np.isscalar(n) else tuple(n)
    h = 1.0 / (max(n) - 1)
    cells = tuple(m + 1 for m in n)
    if het:
        g = W.gaussian_random_field(seed, cells, 2.0)
        cc = np.clip(2.0 + 0.5 * g, 1.0, 3.0)
    else:
        cc = np.full(cells, float(c))
    omega = 2 * math.pi * cc.min() / (ppw * h)
    if R == "layer":
        RR = W.damping_profile(ndim, n, layer, 2.0 * omega)
    elif R == "zero":
        RR = np.zeros(n)
    else:
        RR = np.full(n, float(R))
    F = W.point_source(ndim, n, h)
    return W.Problem("t", ndim, n, h, cc, RR, omega, F, T, rho)


# ----------------------------------------------------------------------------
# stencil tables: textbook Q1 element matrices by Gauss quadrature
# ----------------------------------------------------------------------------

def q1_element_matrices(d):
    """Q1 stiffness and consistent mass on the unit cell by 2-point Gauss quadrature."""
    gp = np.array([0.5 - 0.5 / math.sqrt(3), 0.5 + 0.5 / math.sqrt(3)])
    gw = np.array([0.5, 0.5])
    corners = [tuple((b >> (d - 1 - t)) & 1 for t in range(d)) for b in range(1 << d)]

    def phi(b, x):
        return np.prod([x[t] if b[t] else 1 - x[t] for t in range(d)])

    def dphi(b, x, a):
        v = 1.0 if b[a] else -1.0
        return v * np.prod([(x[t] if b[t] else 1 - x[t]) for t in range(d) if t != a])

    nc = len(corners)
    K = np.zeros((nc, nc))
    Mc = np.zeros((nc, nc))
    for idx in np.ndindex(*(2,) * d):
        x = gp[list(idx)]
        w = np.prod(gw[list(idx)])
        for i, b in enumerate(corners):
            for j, g in enumerate(corners):
                K[i, j] += w * sum(dphi(b, x, a) * dphi(g, x, a) for a in range(d))
                Mc[i, j] += w * phi(b, x) * phi(g, x)
    ham = np.array([[sum(bi != gi for bi, gi in zip(b, g)) for g in corners] for b in corners])
    return K, Mc, ham


@pytest.mark.parametrize("d", [2, 3])
def test_q1mix_tables_are_q1_element_matrices(d):
    K, Mc, ham = q1_element_matrices(d)
    Ml = np.diag(Mc.sum(axis=1))                     # row-sum lumping
    Mmix = 0.5 * Mc + 0.5 * Ml
    S, M = oracle.tables(d, "q1mix")
    for s in range(d + 1):
        sel = ham == s
        assert np.allclose(K[sel], K[sel][0]) and np.allclose(Mmix[sel], Mmix[sel][0])
        assert K[sel][0] == pytest.approx(S[s], abs=1e-14)
        assert Mmix[sel][0] == pytest.approx(M[s], abs=1e-14)
    # App. A requirement used for lambda_min: 0 <= M~ <= 2^{-d} I per cell, S~ PSD
    Mk = M[ham]
    Sk = S[ham]
    ev_m = np.linalg.eigvalsh(Mk)
    assert ev_m.min() >= -1e-14 and ev_m.max() <= 2.0 ** -d + 1e-14
    assert np.linalg.eigvalsh(Sk).min() >= -1e-14


FAMILY = [(0.3, 0.6), (1.0, 0.0), (0.0, 1.0), (0.8, 0.25)]


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("a,g", FAMILY)
def test_family_tables_mix_q1_element_matrices_and_edge_stiffness(d, a, g):
    """FAMILY(a, gamma): gamma x (Q1 element stiffness, Gauss quadrature) +
    (1 - gamma) x (edge stiffness: weight 2^{1-d} per cell edge), a x (consistent
    Q1 mass) + (1 - a) x (row-sum lumped mass); each entry depends only on the
    Hamming distance, the stiffness kernel is PSD and 0 <= mass <= 2^-d."""
    K, Mc, ham = q1_element_matrices(d)
    w = 2.0 ** (1 - d)
    Kfd = np.where(ham == 1, -w, 0.0)
    Kfd[np.diag_indices_from(Kfd)] = -Kfd.sum(axis=1)              # edge graph Laplacian
    Ml = np.diag(Mc.sum(axis=1))
    Kf = g * K + (1 - g) * Kfd
    Mf = a * Mc + (1 - a) * Ml
    S, M = oracle.tables(d, "family", a, g)
    for s in range(d + 1):
        sel = ham == s
        assert np.allclose(Kf[sel], Kf[sel][0]) and np.allclose(Mf[sel], Mf[sel][0])
        assert Kf[sel][0] == pytest.approx(S[s], abs=1e-14)
        assert Mf[sel][0] == pytest.approx(M[s], abs=1e-14)
    assert np.linalg.eigvalsh(S[ham]).min() >= -1e-14
    ev_m = np.linalg.eigvalsh(M[ham])
    assert ev_m.min() >= -1e-14 and ev_m.max() <= 2.0 ** -d + 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_family_corners_are_q1mix_and_fd5(d):
    for st, a, g in (("q1mix", 0.5, 1.0), ("fd5", 0.0, 0.0)):
        S0, M0 = oracle.tables(d, st)
        S1, M1 = oracle.tables(d, "family", a, g)
        assert np.array_equal(S0, S1) and np.array_equal(M0, M1)
    for a, g in ((-0.1, 0.5), (0.5, 1.2), (np.nan, 0.5)):
        with pytest.raises(ValueError):
            oracle.tables(d, "family", a, g)


@pytest.mark.parametrize("d", [2, 3])
def test_fd5_constant_k_is_the_papers_5_point_operator(d):
    """Sec. 3.1: (HU) = h^-2 (2d U - sum of axis neighbours) - k^2 U + i Im H U."""
    n = (7, 6) if d == 2 else (5, 4, 6)
    p = make_problem(d, n, c=1.3, R="layer", layer=2)
    o = oracle.Oracle(p, "fd5")
    H = o.H_sparse().toarray()
    k = p.omega / 1.3
    lap1 = [sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1]) for m in n]
    Id = [sp.identity(m) for m in n]
    L = None
    for a in range(d):
        term = None
        for b in range(d):
            f = lap1[b] if a == b else Id[b]
            term = f if term is None else sp.kron(term, f)
        L = term if L is None else L + term
    Href = (L.toarray() / p.h ** 2 - k * k * np.eye(o.N)
            + 1j * np.diag(p.omega * p.R_node.reshape(-1)))
    assert np.allclose(H, Href, rtol=0, atol=1e-10 * np.abs(Href).max())


def _sine_mode(n, m):
    v = None
    for a, (na, ma) in enumerate(zip(n, m)):
        th = math.pi * ma / (na + 1)
        s = np.sin(th * (np.arange(na) + 1))
        v = s if v is None else np.multiply.outer(v, s)
    return v


def sine_eigenvalue(stencil, n, m, h, kappa, a=0.5, g=1.0):
    """Eigenvalue of Re H (constant kappa = (hk)^2, zero Dirichlet) on sine mode m.

    Q1 finite elements assemble to tensor products of the 1-D stiffness
    tridiag(-1, 2, -1) and 1-D consistent mass tridiag(1, 4, 1)/6; lumped mass
    assembles to the identity.  FD5 is the textbook Laplacian minus k^2.  The
    family mixes the two stiffnesses with weights g, 1 - g and the two masses
    with weights a, 1 - a (Q1MIX: a = 1/2, g = 1).
    """
    th = [math.pi * ma / (na + 1) for na, ma in zip(n, m)]
    k1 = [2 - 2 * math.cos(t) for t in th]
    m1 = [(4 + 2 * math.cos(t)) / 6 for t in th]
    d = len(n)
    if stencil == "fd5":
        return (sum(k1) - kappa) / h ** 2
    stiff = sum(k1[a_] * np.prod([m1[b] for b in range(d) if b != a_]) for a_ in range(d))
    stiff = g * stiff + (1 - g) * sum(k1)
    mass = a * np.prod(m1) + (1 - a)
    return (stiff - kappa * mass) / h ** 2


@pytest.mark.parametrize("d,stencil", [(2, "q1mix"), (3, "q1mix"), (2, "fd5"), (3, "fd5")])
def test_sine_modes_diagonalise_constant_coefficient_operator(d, stencil):
    n = (9, 7) if d == 2 else (5, 6, 4)
    p = make_problem(d, n, c=0.8, R="zero")
    o = oracle.Oracle(p, stencil)
    kappa = (p.h * p.omega / 0.8) ** 2
    rng = np.random.default_rng(1)
    for _ in range(6):
        m = tuple(int(rng.integers(1, na + 1)) for na in n)
        v = _sine_mode(n, m)
        lam = sine_eigenvalue(stencil, n, m, p.h, kappa)
        Hv = o.apply_reH(v)
        assert np.abs(Hv - lam * v).max() <= 1e-10 * abs(lam) * np.abs(v).max() + 1e-9


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("a,g", FAMILY)
def test_sine_modes_diagonalise_family_operator(d, a, g):
    n = (8, 7) if d == 2 else (5, 4, 6)
    p = make_problem(d, n, c=0.9, R="zero")
    o = oracle.Oracle(p, "family", stencil_a=a, stencil_gamma=g)
    kappa = (p.h * p.omega / 0.9) ** 2
    rng = np.random.default_rng(2)
    for _ in range(6):
        m = tuple(int(rng.integers(1, na + 1)) for na in n)
        v = _sine_mode(n, m)
        lam = sine_eigenvalue("family", n, m, p.h, kappa, a, g)
        Hv = o.apply_reH(v)
        assert np.abs(Hv - lam * v).max() <= 1e-10 * abs(lam) * np.abs(v).max() + 1e-9


@pytest.mark.parametrize("d,n", [(2, (9, 8)), (3, (5, 4, 5))])
@pytest.mark.parametrize("a,g", FAMILY)
def test_family_required_properties_and_bounds(d, n, a, g):
    """Re H symmetric with lambda_min >= -k_max^2 and lambda_max below the
    symbol-vertex bound; K >= 0 and 4 I - K > 0 at the chosen time step."""
    p = make_problem(d, n, het=True, R="layer", layer=2)
    o = oracle.Oracle(p, "family", stencil_a=a, stencil_gamma=g)
    reH = o.H_sparse().toarray().real
    assert np.allclose(reH, reH.T, atol=1e-9)
    ev = np.linalg.eigvalsh(reH)
    q = o.params
    assert ev.min() >= -q.k_max ** 2 * (1 + 1e-12)
    assert ev.max() <= q.lam_max_reH * (1 + 1e-12)
    evK = np.linalg.eigvalsh(q.dt ** 2 / q.alpha * (reH + q.omega ** 2 * np.eye(o.N)))
    assert evK.min() >= -1e-12 and evK.max() < 4.0


# ----------------------------------------------------------------------------
# properties required of H (Sec. 1) and the bounds used for omega, dt (App. A)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("d,n", [(2, (11, 9)), (3, (5, 6, 5))])
@pytest.mark.parametrize("stencil", ["q1mix", "fd5"])
def test_required_properties_and_eigenvalue_bounds(d, n, stencil):
    p = make_problem(d, n, het=True, R="layer", layer=2)
    o = oracle.Oracle(p, stencil)
    H = o.H_sparse().toarray()
    reH, imH = H.real, H.imag
    assert np.allclose(reH, reH.T, atol=1e-9)                       # Re H symmetric
    assert np.count_nonzero(imH - np.diag(np.diag(imH))) == 0       # Im H diagonal
    assert np.diag(imH).min() >= 0                                  # Im H PSD
    ev = np.linalg.eigvalsh(reH)
    q = o.params
    assert ev.min() >= -q.k_max ** 2 * (1 + 1e-12)                   # App. A lower bound
    assert ev.max() <= q.lam_max_reH * (1 + 1e-12)                   # symbol-vertex bound
    # K >= 0 and 4I - K > 0 (stability conditions of Theorem 1)
    K = q.dt ** 2 / q.alpha * (reH + q.omega ** 2 * np.eye(o.N))
    evK = np.linalg.eigvalsh(K)
    assert evK.min() >= -1e-12 and evK.max() < 4.0


def test_lambda_max_bound_is_tight_for_constant_speed():
    p = make_problem(2, (40, 40), c=1.0, R="zero")
    o = oracle.Oracle(p, "q1mix")
    ev = np.linalg.eigvalsh(o.H_sparse().toarray().real)
    assert ev.max() <= o.params.lam_max_reH
    assert ev.max() >= 0.98 * o.params.lam_max_reH


def test_parameter_formulas():
    facts = json.load(open(GOLDEN))
    p = make_problem(2, (31, 31), het=True)
    o = oracle.Oracle(p)
    q = o.params
    # omega = k_max (per-cell bound), dt = 2 pi / (omega n_P)
    assert q.omega == pytest.approx(p.omega / p.c_cell.min(), rel=1e-14)
    assert q.dt * q.omega * q.nP == pytest.approx(2 * math.pi, rel=1e-14)
    x = q.omega * q.dt
    assert q.alpha == pytest.approx(x * x / (2 - 2 * math.cos(x)), rel=1e-12)
    assert q.beta == pytest.approx(x / math.sin(x), rel=1e-12)
    # n_P: multiple of 4 (Sec. 2.3), strict CFL (Eq. define_Deltat_ImH_diagonal), minimal
    m4 = facts["steps_per_period_multiple_of"]["value"]
    assert q.nP % m4 == 0
    assert q.dt < 2 / q.omega * math.asin(q.omega / math.sqrt(q.lam_max_A))
    if q.nP > m4:
        dt_prev = 2 * math.pi / (q.omega * (q.nP - m4))
        assert not dt_prev < 2 / q.omega * math.asin(q.omega / math.sqrt(q.lam_max_A))
    # rho = 0 means a ramp over one period (Sec. 5.1)
    o0 = oracle.Oracle(p, rho=0.0, T=8)
    assert o0.params.rho == pytest.approx(1.0 / 8)
    # a requested n_P below the CFL bound is refused
    with pytest.raises(ValueError):
        oracle.Oracle(p, nP=4)
    with pytest.raises(ValueError):
        oracle.Oracle(p, nP=q.nP + 2)


def test_six_points_per_wavelength_gives_eight_steps_per_period():
    """Sec. 5.1: 6 points per wavelength resulted in 8 time steps per period."""
    facts = json.load(open(GOLDEN))
    want = facts["steps_per_period_at_6_points_per_wavelength"]["value"]
    for n in (101, 321):
        p = W.config_2d_constant(n, ppw=6.0)
        assert oracle.Oracle(p).params.nP == want
    p3 = make_problem(3, 24, ppw=6.0)
    assert oracle.Oracle(p3).params.nP == want


def test_window_is_admissible():
    facts = json.load(open(GOLDEN))["window_sine_squared_limits"]["value"]
    p = make_problem(2, 11)
    o = oracle.Oracle(p)
    for rho in (0.1, 0.25, 0.5, 0.75, 1.0):
        assert o.window(0.0, rho) == facts["chi_at_0"]
        assert o.window(1.0, rho) == facts["chi_at_1"]
        assert o.window(1.5, rho) == 0.0
        s = np.linspace(0, 1, 2001)
        v = np.array([o.window(x, rho) for x in s])
        assert np.all(np.diff(v) <= 1e-15)                       # non-increasing on [0, 1]
        assert all(o.window(-x, rho) == o.window(x, rho) for x in s[::50])   # even
        # continuous and C^1 at both ends of the taper: one-sided slopes agree
        for s0 in (1 - rho, 1.0):
            e = 1e-6
            left = (o.window(s0, rho) - o.window(s0 - e, rho)) / e
            right = (o.window(s0 + e, rho) - o.window(s0, rho)) / e
            assert abs(left - right) < 1e-4 * (1 + 1 / rho)
        # sine squared: half-way through the taper chi = sin^2(pi/4) = 1/2
        assert o.window(1 - rho / 2, rho) == pytest.approx(0.5, abs=1e-14)


# ----------------------------------------------------------------------------
# the time integrator: Prop. 1 and Theorem 1
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("d,n", [(2, (13, 11)), (3, (6, 5, 7))])
def test_prop1_time_harmonic_solutions_are_reproduced_exactly(d, n):
    """Prop. 1: u_n = e^{i w n dt} U, f_n = e^{i w n dt} F solve I_acd iff H U = F."""
    p = make_problem(d, n, het=True, R="layer", layer=2)
    o = oracle.Oracle(p)
    H = o.H_sparse().tocsc()
    F = W.random_rhs(3, n).reshape(-1)
    U = sla.spsolve(H, F)
    w, dt = o.params.omega, o.params.dt
    e = lambda k: np.exp(1j * w * k * dt)
    u2 = o.acd_step(e(1) * U, e(0) * U, e(1) * F).reshape(-1)
    assert np.linalg.norm(u2 - e(2) * U) <= 1e-10 * np.linalg.norm(U)
    # and a non-solution is not reproduced
    U2 = U + 1e-3 * np.linalg.norm(U) / math.sqrt(U.size)
    u2b = o.acd_step(e(1) * U2, e(0) * U2, e(1) * F).reshape(-1)
    assert np.linalg.norm(u2b - e(2) * U2) > 1e-6 * np.linalg.norm(U)


def test_theorem1_energy_identity():
    """Homogeneous recursion: E(n+1/2) - E(n-1/2) = -2 <D, L D>, D = u_{n+1} - u_{n-1}."""
    n = (12, 10)
    p = make_problem(2, n, het=True, R="layer", layer=3)
    o = oracle.Oracle(p)
    q = o.params
    reH = o.H_sparse().real.toarray()
    K = q.dt ** 2 / q.alpha * (reH + q.omega ** 2 * np.eye(o.N))
    L = q.beta * q.dt / q.alpha * (p.omega * p.R_node.reshape(-1) / q.omega)
    rng = np.random.default_rng(5)
    um1 = rng.standard_normal(o.N)
    u0 = rng.standard_normal(o.N)
    E = lambda a, b: (a - b) @ ((4 * np.eye(o.N) - K) @ (a - b)) + (a + b) @ (K @ (a + b))
    zero = np.zeros(o.N)
    for _ in range(20):
        u1 = o.acd_step(u0, um1, zero).reshape(-1).real
        D = u1 - um1
        dE = E(u1, u0) - E(u0, um1)
        assert dE == pytest.approx(-2 * D @ (L * D), rel=1e-9, abs=1e-9 * abs(E(u0, um1)))
        assert dE <= 1e-12 * abs(E(u0, um1))
        um1, u0 = u0, u1


# ----------------------------------------------------------------------------
# the preconditioner: Theorem 3's Green's-function sum on sine modes
# ----------------------------------------------------------------------------

def chi_sine_squared(s, rho):
    s = abs(s)
    if s >= 1:
        return 0.0
    if s <= 1 - rho:
        return 1.0
    return math.sin(math.pi * (1 - s) / (2 * rho)) ** 2


def scalar_preconditioner(lam, ell, q, F, mode, periods=1):
    """Scalar S_T (or Table 1) by the Green's-function sum of Theorem 3.

    k = dt^2/alpha (lam + omega^2); Lambda_+- from Eq. Lambda_pm_stability;
    impulse response G_j = (L+^j - L-^j) / ((1 + ell/2)(L+ - L-)).
    """
    k = q.dt ** 2 / q.alpha * (lam + q.omega ** 2)
    disc = complex(-k + k * k / 4 + ell * ell / 4)
    lp = ((1 - k / 2) + np.sqrt(disc)) / (1 + ell / 2)
    lm = ((1 - k / 2) - np.sqrt(disc)) / (1 + ell / 2)
    ns = q.nsteps
    j = np.arange(ns + 1)
    G = (lp ** j - lm ** j) / ((1 + ell / 2) * (lp - lm))
    chi = np.array([chi_sine_squared(1 - m / ns, q.rho) for m in range(ns)])
    c = q.dt ** 2 / q.alpha
    m = np.arange(ns)
    if mode == "exact":
        f = chi * np.exp(1j * q.omega * m * q.dt) * F
        u = np.sum(G[ns - m] * c * f)
        return np.exp(-2j * math.pi * q.T) * u
    f = chi * (np.cos(2 * math.pi * m / q.nP) * F.real - np.sin(2 * math.pi * m / q.nP) * F.imag)
    if mode == "project":
        # u_j = sum_{m < j} G_{j-m} c f_m for the states of the last `periods` periods
        n_acc = periods * q.nP
        acc = 0j
        for jj in range(ns - n_acc + 1, ns + 1):
            uj = np.sum(G[jj - m[:jj]] * c * f[:jj]).real
            acc += np.exp(-2j * math.pi * jj / q.nP) * uj
        return 2.0 * acc / n_acc
    u_end = np.sum(G[ns - m] * c * f).real
    jim = ns - q.nP // 4
    mm = np.arange(jim)
    u_im = np.sum(G[jim - mm] * c * f[:jim]).real
    return u_end + 1j * u_im


@pytest.mark.parametrize("d,stencil", [(2, "q1mix"), (3, "q1mix"), (2, "fd5")])
@pytest.mark.parametrize("R", ["zero", 40.0])
@pytest.mark.parametrize("mode", ["table1", "exact"])
def test_preconditioner_on_sine_mode_equals_greens_sum(d, stencil, R, mode):
    n = (15, 13) if d == 2 else (7, 6, 5)
    p = make_problem(d, n, c=1.0, R=R, T=3, rho=0.3)
    o = oracle.Oracle(p, stencil)
    q = o.params
    kappa = (p.h * p.omega) ** 2
    ell = q.beta * q.dt / q.alpha * (p.omega * float(p.R_node.flat[0]) / q.omega)
    for m, Fs in [((1,) * d, 1.0 + 0.0j), ((2, 3) + (1,) * (d - 2), 0.3 - 0.7j),
                  (tuple(n), -0.2 + 1.1j)]:
        v = _sine_mode(n, m)
        lam = sine_eigenvalue(stencil, n, m, p.h, kappa)
        U = o.precond(Fs * v, mode)
        s = scalar_preconditioner(lam, ell, q, Fs, mode)
        assert np.abs(U - s * v).max() <= 1e-10 * max(abs(s), 1e-30) * np.abs(v).max()


@pytest.mark.parametrize("d,stencil", [(2, "q1mix"), (3, "q1mix")])
@pytest.mark.parametrize("R", ["zero", 40.0])
@pytest.mark.parametrize("periods", [1, 2])
def test_projection_on_sine_mode_equals_greens_sum(d, stencil, R, periods):
    """The projection read-out on a sine mode (constant k): the grid recurrence
    acts as a scalar, equal to the Green's-function sum of Theorem 3 projected
    by hand over the last `periods` periods."""
    n = (15, 13) if d == 2 else (7, 6, 5)
    p = make_problem(d, n, c=1.0, R=R, T=3, rho=0.3)
    o = oracle.Oracle(p, stencil)
    q = o.params
    kappa = (p.h * p.omega) ** 2
    ell = q.beta * q.dt / q.alpha * (p.omega * float(p.R_node.flat[0]) / q.omega)
    for m, Fs in [((1,) * d, 1.0 + 0.0j), ((2, 3) + (1,) * (d - 2), 0.3 - 0.7j)]:
        v = _sine_mode(n, m)
        lam = sine_eigenvalue(stencil, n, m, p.h, kappa)
        U = o.precond(Fs * v, "project", periods=periods)
        s = scalar_preconditioner(lam, ell, q, Fs, "project", periods)
        assert np.abs(U - s * v).max() <= 1e-10 * max(abs(s), 1e-30) * np.abs(v).max()


@pytest.mark.parametrize("nP,periods,j_first", [(4, 1, 0), (8, 2, 37), (12, 3, 1500)])
def test_projection_recovers_time_harmonic_amplitude(nP, periods, j_first):
    """For exactly time-harmonic states u_j = Re(U e^{i 2 pi j / n_P}) the
    projection over whole periods returns U (the e^{-2 i theta} terms cancel);
    over a part of a period it does not, which is why the read-out uses whole
    periods."""
    rng = np.random.default_rng(5)
    U = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    j = j_first + np.arange(periods * nP)
    states = np.real(U[None, :] * np.exp(2j * np.pi * j / nP)[:, None])
    got = oracle.project_states(states, nP, j_first)
    assert np.abs(got - U).max() <= 1e-13 * np.abs(U).max()
    part = oracle.project_states(states[: nP // 2 + 1], nP, j_first)
    assert np.abs(part - U).max() > 1e-3 * np.abs(U).max()


def test_projection_converges_to_Hinv_with_T():
    """The projected read-out of the damped recurrence approaches H^{-1} F as
    T grows, like S_T (Theorem 4)."""
    p = make_problem(2, (25, 25), c=1.0, R="layer", layer=5, ppw=8)
    U = oracle.Oracle(p).direct_solve(p.F)
    errs = []
    for T in (2, 4, 8, 16, 32):
        o = oracle.Oracle(p, T=T)
        errs.append(np.linalg.norm(o.precond(p.F, "project") - U) / np.linalg.norm(U))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * errs[0]


def test_table1_real_part_is_exact_real_part_and_linearity():
    """Re of Table 1's output is u_{T n_P} of the real-field run = Re S_T F.  S_T is
    C-linear; Table 1 is only R-linear (its imaginary part is the quarter-period
    snapshot), which is why the flexible Krylov method is the default."""
    p = make_problem(2, (17, 15), het=True)
    o = oracle.Oracle(p)
    F = W.random_rhs(11, p.n)
    Ut = o.precond(F, "table1")
    Ue = o.precond(F, "exact")
    scale = np.abs(Ue).max()
    assert np.abs(Ut.real - Ue.real).max() <= 1e-12 * scale
    Ue_i = o.precond(1j * F, "exact")
    assert np.abs(Ue_i - 1j * Ue).max() <= 1e-12 * scale
    Ut_i = o.precond(1j * F, "table1")
    assert np.abs(Ut_i - 1j * Ut).max() > 1e-6 * scale


RATE_T = (12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 128)


def st_error_envelope_slope(stencil_mode, Ts=RATE_T):
    """Least-squares slope of log(envelope of |s_T(lambda) lambda - 1|) against
    log T, with s_T(lambda) read off the oracle's S_T applied to a sine mode of
    a constant-k grid without damping (an eigenvector of Re H), and the last
    error.  The envelope max_{T' >= T} err(T') removes the oscillation that the
    aliasing and pole terms of the convolution formula put on the error."""
    n, m = stencil_mode
    p = make_problem(2, n, c=1.0, R="zero", T=4, rho=0.25, ppw=6)
    kappa = (p.h * p.omega) ** 2
    lam = sine_eigenvalue("q1mix", n, m, p.h, kappa)
    v = _sine_mode(n, m)
    errs = []
    for T in Ts:
        U = oracle.Oracle(p, T=int(T)).precond(v, "exact")
        s = (U * v).sum() / (v * v).sum()
        errs.append(abs(s * lam - 1.0))
    env = [max(errs[i:]) for i in range(len(errs))]
    return np.polyfit(np.log(Ts), np.log(env), 1)[0], errs[-1], lam


@pytest.mark.parametrize("m", [(2, 1), (8, 1), (18, 1), (24, 1)],
                         ids=["caseI-near-minus-omega2", "caseI", "caseII", "caseII-large"])
def test_theorem5_rate_of_ST_on_sine_modes(m):
    """Theorem 5 (speed of convergence, Im H = 0): S_T acts on an eigenvector of
    Re H as the scalar s_T(lambda), and |s_T(lambda) - 1/lambda| decays like a
    power of T fixed by the smoothness of the window chi.  The sin^2 window of
    Sec. 2.3 is piecewise smooth with jumps in its second derivative, so chi-hat
    decays like |sigma|^-3 (N_1 = 3 in the theorem's decay assumption, by the
    rule that jumps in the k-th derivative give N_1 = k + 1); chi = 1 near 0
    makes every moment of chi-hat vanish, and the integrability half of the
    moment condition then allows N_2 = 1, so the theorem guarantees at least
    T^-1 in both of its cases (lambda < 0 and lambda > 0, away from 0).  The
    |sigma|^-3 tails of chi-hat give an error envelope of order T^-2; a window
    that is only continuous (a kink at its ends, N_1 = 2) gives T^-1 (planted in
    test_oracle_mutants.py).  Modes in case I (lambda in [-omega^2, gamma],
    gamma < 0) and in case II (lambda > 0)."""
    slope, last, lam = st_error_envelope_slope(((31, 31), m))
    assert slope <= -1.8, (lam, slope)
    assert last <= 3e-3, (lam, last)


def test_theorem4_ST_converges_to_Hinv():
    p = make_problem(2, (25, 25), c=1.0, R="layer", layer=5, ppw=8)
    o0 = oracle.Oracle(p)
    U = o0.direct_solve(p.F)
    errs = []
    for T in (2, 4, 8, 16, 32):
        o = oracle.Oracle(p, T=T)
        errs.append(np.linalg.norm(o.precond(p.F, "exact") - U) / np.linalg.norm(U))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * errs[0]


# ----------------------------------------------------------------------------
# direct solve and GMRES
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("d,n", [(2, (23, 19)), (3, (7, 6, 8))])
def test_direct_solve_matches_scipy(d, n):
    p = make_problem(d, n, het=True)
    o = oracle.Oracle(p)
    F = W.random_rhs(2, n).reshape(-1)
    U = o.direct_solve(F).reshape(-1)
    Uref = sla.spsolve(o.H_sparse().tocsc(), F)
    assert np.linalg.norm(U - Uref) <= 1e-10 * np.linalg.norm(Uref)
    HU = o.apply_H(U).reshape(-1)
    assert np.linalg.norm(HU - o.H_sparse() @ U) <= 1e-12 * np.linalg.norm(HU)


def test_gmres_unpreconditioned_matches_scipy_residual_history():
    p = make_problem(2, (15, 13), het=True)
    o = oracle.Oracle(p)
    F = W.random_rhs(4, p.n).reshape(-1)
    m = 10
    hist = []
    sla.gmres(o.H_sparse(), F, rtol=1e-14, atol=0.0, restart=m, maxiter=2,
              callback=lambda r: hist.append(r), callback_type="pr_norm")
    for kr in ("fgmres", "left"):
        _, info = o.gmres(F, kr, "identity", tol=0.0, restart=m, maxit=2 * m, fixed=True)
        mine = np.array(info["hist"][: len(hist)])
        assert len(mine) == len(hist) == 2 * m
        assert np.allclose(mine, hist, rtol=1e-8)


def test_gmres_with_exact_inverse_converges_in_one_step():
    p = make_problem(2, (15, 17), het=True)
    o = oracle.Oracle(p)
    for kr in ("fgmres", "left"):
        U, info = o.gmres(p.F, kr, "direct", tol=1e-10, restart=5, maxit=5)
        assert info["iterations"] == 1 and info["rel_res_true"] < 1e-12


@pytest.mark.parametrize("kr,pc", [("fgmres", "table1"), ("fgmres", "exact"), ("left", "exact")])
def test_gmres_recovers_manufactured_solution(kr, pc):
    p = make_problem(2, (21, 19), het=True, T=3)
    o = oracle.Oracle(p)
    Ustar = W.random_rhs(9, p.n)
    F = o.apply_H(Ustar)
    U, info = o.gmres(F, kr, pc, tol=1e-11, restart=20, maxit=200)
    assert info["converged"] and info["rel_res_true"] <= 1e-11
    assert np.linalg.norm(U - Ustar) <= 1e-7 * np.linalg.norm(Ustar)
