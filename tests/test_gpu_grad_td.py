"""GPU gradient through the recurrence (htd_grad_td): misfit of the
preconditioner's own output and its reverse-time adjoint gradient with
checkpoints, against the FP64 oracle's (all states kept) on small grids.

Tolerances: FP64 1e-10 on the misfit and 1e-8 (relative L2) on the gradients
(summation order only); mixed precision (FP32 states and multipliers, FP64
sums) 1e-5 on the misfit and 2e-4 on the gradients.  The checkpoint interval
changes only which states are recomputed, not any arithmetic: gradients for
different intervals are identical.
"""
import numpy as np
import pytest

import oracle
from paper_2006_16861_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2006_16861_gb300 import autograd as AG  # noqa: E402
from paper_2006_16861_gb300 import htd  # noqa: E402
from test_gpu_gradient import dev, small_case  # noqa: E402

CASES = [  # (ndim, n, mode, precision)
    (2, (41, 37), "table1", "fp64"),
    (2, (33, 40), "exact", "fp64"),
    (3, (13, 11, 15), "table1", "fp64"),
    (2, (70, 66), "table1", "mixed"),
    (3, (13, 11, 15), "exact", "mixed"),
]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{'x'.join(map(str, c[1]))}-{c[2]}-{c[3]}"
                                             for c in CASES])
def test_recurrence_gradient_matches_oracle(case):
    ndim, n, mode, precision = case
    p, F, rec, d = small_case(ndim, n, 2)
    s = htd.Solver(p, precision=precision, mode=mode)
    J, gm, gR = s.grad_td(dev(F), rec, dev(d))
    Jo, gmo, gRo = oracle.Oracle(p).grad_td(F, rec, d, mode)
    fp64 = precision == "fp64"
    assert J == pytest.approx(Jo, rel=1e-10 if fp64 else 1e-5)
    assert rel(gm.cpu().numpy(), gmo) <= (1e-8 if fp64 else 2e-4)
    assert rel(gR.cpu().numpy(), gRo) <= (1e-8 if fp64 else 2e-4)
    J2, g1, g2 = s.grad_td(dev(F), rec, dev(d), want_grad=False)
    assert g1 is None and J2 == J


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_interval_does_not_change_the_gradient(precision):
    p, F, rec, d = small_case(2, (30, 28), 1)
    s = htd.Solver(p, precision=precision)
    ns = s.params["steps"]
    ref = s.grad_td(dev(F), rec, dev(d), checkpoint_every=0)
    for C in (1, 7, ns - 1, ns, ns + 5):
        J, gm, gR = s.grad_td(dev(F), rec, dev(d), checkpoint_every=C)
        assert J == ref[0]
        assert torch.equal(gm, ref[1]) and torch.equal(gR, ref[2])


def test_autograd_and_finite_differences_fp64():
    """preconditioner_misfit's backward equals htd_grad_td, and the gradient
    matches central differences of the GPU misfit along directions that leave
    the recurrence parameters (chosen from min / max c) unchanged."""
    p, F, rec, d = small_case(2, (36, 34), 2)
    m = torch.tensor(p.c_cell ** -2.0, dtype=torch.float64, device="cuda", requires_grad=True)
    R = torch.tensor(p.R_node, dtype=torch.float64, device="cuda", requires_grad=True)
    Fd, dd = dev(F), dev(d)
    J = AG.preconditioner_misfit(m, R, p, Fd, rec, dd, precision="fp64")
    J.backward()
    s = htd.Solver(p, precision="fp64")
    J0, gm, gR = s.grad_td(Fd, rec, dd)
    assert float(J.detach()) == pytest.approx(J0, rel=1e-14)
    assert torch.allclose(m.grad, gm, rtol=1e-12, atol=0) and torch.allclose(R.grad, gR, rtol=1e-12,
                                                                            atol=0)
    params0 = s.params
    mm = p.c_cell ** -2.0
    # a smooth bump away from the extreme cells of c
    cells = np.indices(mm.shape).astype(float)
    cen = np.array(mm.shape) * np.array([0.4, 0.6])
    bump = np.exp(-((cells[0] - cen[0]) ** 2 + (cells[1] - cen[1]) ** 2) / 8.0)
    bump[mm == mm.max()] = 0.0
    bump[mm == mm.min()] = 0.0
    v = 1e-3 * bump * mm
    eps = 1e-3

    def J_at(mv=None, Rv=None):
        q = W.Problem(p.name, p.ndim, p.n, p.h, (mm if mv is None else mv) ** -0.5,
                      p.R_node if Rv is None else Rv, p.omega, p.F, p.T, p.rho)
        sq = htd.Solver(q, precision="fp64")
        assert sq.params["nP"] == params0["nP"] and sq.params["dt"] == params0["dt"]
        assert sq.params["omega_c"] == params0["omega_c"]
        return sq.grad_td(Fd, rec, dd, want_grad=False)[0]

    fd = (J_at(mv=mm + eps * v) - J_at(mv=mm - eps * v)) / (2 * eps)
    assert float(np.sum(gm.cpu().numpy() * v)) == pytest.approx(fd, rel=1e-5)
    w = 1e-3 * p.R_node * np.exp(-((np.indices(p.n)[0] - 1.0) ** 2) / 4.0)
    fd = (J_at(Rv=p.R_node + eps * w) - J_at(Rv=p.R_node - eps * w)) / (2 * eps)
    assert float(np.sum(gR.cpu().numpy() * w)) == pytest.approx(fd, rel=1e-5)


def test_recurrence_gradient_rejects_bad_arguments():
    p, F, rec, d = small_case(2, (20, 22), 1)
    sp = htd.Solver(p, precision="mixed", mode="project")
    with pytest.raises(htd.HtdError) as e:
        sp.grad_td(dev(F), rec, dev(d))
    assert e.value.status == 1
    s = htd.Solver(p, precision="mixed")
    with pytest.raises(htd.HtdError) as e:
        s.grad_td(dev(F), rec, dev(d), checkpoint_every=-1)
    assert e.value.status == 1
    bad = rec.copy()
    bad[0] = p.N
    with pytest.raises(htd.HtdError) as e:
        s.grad_td(dev(F), bad, dev(d))
    assert e.value.status == 1


def _config5_data(st, precision="fp64"):
    """Receiver data of the adjoint configuration for the recurrence misfit: the
    preconditioner's own output for the 'true' model (c with the 5 % blob),
    sampled at the receivers (computed with the library; the comparisons below
    use GPU misfits or the oracle on the same data)."""
    p = st.prob
    pt = W.Problem(p.name, 2, p.n, p.h, st.c_true, p.R_node, p.omega, p.F, p.T, p.rho)
    s = htd.Solver(pt, precision=precision)
    rec = torch.from_numpy(st.rec_idx).cuda()
    d = torch.stack([s.precond(dev(st.F[k])).reshape(-1)[rec] for k in range(st.F.shape[0])])
    s.close()
    return d.contiguous()


def test_recurrence_gradient_at_the_adjoint_configuration_size():
    """The checkpointed reverse-time adjoint on the full adjoint configuration:
    2-D 512^2, smooth random c, 8 seeded point sources, receivers on the first
    row inside the top absorbing layer.  FP64: the gradient along localized
    directions (which leave the recurrence parameters, chosen from min / max c,
    unchanged) against central differences of the GPU misfit, relative error
    < 1e-4.  Mixed precision against FP64: the misfit residual r = P F - d is a
    difference of O(1) quantities, so the FP32 state error (<= 2e-5 relative to
    P F, the full-grid kernel parity) is amplified by ||P F|| / ||r|| at the
    receivers in J and in the adjoint forcing; the tolerance is 2e-5 times that
    amplification times 10."""
    st = W.config_adjoint(512)
    p = st.prob
    F = dev(st.F)
    d = _config5_data(st)
    s = htd.Solver(p, precision="fp64")
    prm0 = s.params
    J, gm, gR = s.grad_td(F, st.rec_idx, d)
    rec = torch.from_numpy(st.rec_idx).cuda()
    PF = torch.stack([s.precond(F[k].contiguous()).reshape(-1)[rec] for k in range(F.shape[0])])
    amp = float(torch.linalg.norm(PF) / torch.linalg.norm(PF - d))
    s.close()
    gm, gR = gm.cpu().numpy(), gR.cpu().numpy()
    assert J > 0 and np.isfinite(gm).all() and np.isfinite(gR).all()
    mm = p.c_cell ** -2.0
    n1 = p.n[0] + 1
    xs = (np.arange(n1) - 0.5) * p.h
    X, Y = np.meshgrid(xs, xs, indexing="ij")

    def J_at(mv=None, Rv=None):
        q = W.Problem(p.name, p.ndim, p.n, p.h, (mm if mv is None else mv) ** -0.5,
                      p.R_node if Rv is None else Rv, p.omega, p.F, p.T, p.rho)
        sq = htd.Solver(q, precision="fp64")
        for k in ("nP", "dt", "omega_c"):
            assert sq.params[k] == prm0[k], k
        Jq = sq.grad_td(F, st.rec_idx, d, want_grad=False)[0]
        sq.close()
        return Jq

    eps = 1e-3
    for cen, wid in (((0.4, 0.6), 0.02), ((0.7, 0.3), 0.005)):
        v = np.exp(-((X - cen[0]) ** 2 + (Y - cen[1]) ** 2) / wid) * mm
        v[mm == mm.max()] = 0.0
        v[mm == mm.min()] = 0.0
        # relative changes of 1e-4 (eps v / m): large against the rounding of J,
        # small enough for central differences at 1e-4
        v *= 1e-1
        fd = (J_at(mv=mm + eps * v) - J_at(mv=mm - eps * v)) / (2 * eps)
        assert abs(np.sum(gm * v) - fd) <= 1e-4 * abs(fd), (np.sum(gm * v), fd)
    w = 1e-1 * p.R_node * np.exp(-((X[:-1, :-1] - 0.02) ** 2 + (Y[:-1, :-1] - 0.5) ** 2) / 0.01)
    fd = (J_at(Rv=p.R_node + eps * w) - J_at(Rv=p.R_node - eps * w)) / (2 * eps)
    assert abs(np.sum(gR * w) - fd) <= 1e-4 * abs(fd), (np.sum(gR * w), fd)
    # mixed precision against FP64
    tol = 10 * 2e-5 * amp
    sm = htd.Solver(p, precision="mixed")
    Jm, gmm, gRm = sm.grad_td(F, st.rec_idx, d)
    sm.close()
    print(f"\nconfig-5 recurrence adjoint: amplification {amp:.1f}, mixed-vs-FP64 "
          f"J {abs(Jm / J - 1):.2e}, grad_m {rel(gmm.cpu().numpy(), gm):.2e}, "
          f"grad_R {rel(gRm.cpu().numpy(), gR):.2e}, tolerance {tol:.2e}")
    assert abs(Jm / J - 1) <= tol
    assert rel(gmm.cpu().numpy(), gm) <= tol and rel(gRm.cpu().numpy(), gR) <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_recurrence_gradient_on_a_block_of_the_adjoint_configuration(precision):
    """Oracle parity on a 96 x 96 block cropped from the adjoint configuration's
    model (its top-left corner: part of the top absorbing layer with the
    receivers on its first row), three seeded sources inside the block, T by
    the block's size in wavelengths."""
    st = W.config_adjoint(512)
    p = st.prob
    b = 96
    c = np.ascontiguousarray(p.c_cell[: b + 1, : b + 1])
    R = np.ascontiguousarray(p.R_node[:b, :b])
    T = W.periods_for(b, p.h, float(c.min()), p.omega)
    F = W.seeded_sources(11, 2, (b, b), p.h, 3, 8)
    q = W.Problem("adjoint_block", 2, (b, b), p.h, c, R, p.omega, F[0], T, p.rho)
    rec = np.arange(1 * b, 2 * b, dtype=np.int64)          # the block's second row
    d = 1e-2 * (W.white_noise(21, (3, rec.size)) + 1j * W.white_noise(22, (3, rec.size)))
    s = htd.Solver(q, precision=precision)
    J, gm, gR = s.grad_td(dev(F), rec, dev(d))
    s.close()
    Jo, gmo, gRo = oracle.Oracle(q).grad_td(F, rec, d, "table1")
    fp64 = precision == "fp64"
    assert J == pytest.approx(Jo, rel=1e-10 if fp64 else 1e-5)
    assert rel(gm.cpu().numpy(), gmo) <= (1e-8 if fp64 else 2e-4)
    assert rel(gR.cpu().numpy(), gRo) <= (1e-8 if fp64 else 2e-4)
