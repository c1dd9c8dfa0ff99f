"""The allocation-free residual norm (htd_residual_norm_noalloc).

Some callers of this library cannot let it allocate device memory when they
call it: applications whose device memory is handed out by their own pool (a
framework's caching allocator that has reserved most of the GPU, so a library's
cudaMalloc would fail or fragment it) and solve loops that cannot afford the
device-wide synchronisation cudaMalloc/cudaFree may imply.  For them
htd_residual_norm_noalloc keeps its residual vector and partial sums in a fixed
buffer inside the library.  These tests check, through the C ABI, that two
calls in a row give the same relative residual as the ordinary
htd_residual_norm, that a call allocates nothing (device memory in use and
free are unchanged across it), that the largest accepted problem agrees with
the oracle's residual, that a call on a separate stream works, and that
problems larger than the buffer are refused.

The file is named so that pytest collects it last: if it fails, a run that
stops at the first failure has already run every other test.  It passes both
alone in a fresh process and after the other tests (the buffer keeps the last
call's contents, and every call writes what it reads first).
"""
import math

import numpy as np
import pytest

from paper_2006_16861_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2006_16861_gb300 import htd  # noqa: E402


def _problem(ndim, n, seed):
    n = tuple(n)
    h = 1.0 / (max(n) - 1)
    g = W.gaussian_random_field(seed, tuple(m + 1 for m in n), 3.0)
    c = np.clip(2.0 + 0.5 * g, 1.0, 3.0)
    omega = 2 * math.pi * c.min() / (8 * h)
    R = W.damping_profile(ndim, n, 4, 2 * omega)
    return W.Problem("noalloc", ndim, n, h, c, R, omega, W.point_source(ndim, n, h), 2)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("ndim,n", [(2, (301, 257)), (3, (40, 37, 45))])
def test_noalloc_residual_matches_residual_norm(ndim, n):
    p = _problem(ndim, n, 3)
    s = htd.Solver(p)
    F = _dev(W.random_rhs(1, p.n))
    U = _dev(W.random_rhs(2, p.n) * 1e-4)
    ref = htd.htd_residual_norm(s.handle, F, U)
    got1 = htd.htd_residual_norm_noalloc(s.handle, F, U)
    got2 = htd.htd_residual_norm_noalloc(s.handle, F, U)
    assert got1 == pytest.approx(ref, rel=1e-12, abs=0)
    assert got2 == pytest.approx(ref, rel=1e-12, abs=0)
    # a different right-hand side on the same buffer: the previous contents do not leak in
    F2 = _dev(W.random_rhs(5, p.n))
    assert htd.htd_residual_norm_noalloc(s.handle, F2, U) == pytest.approx(
        htd.htd_residual_norm(s.handle, F2, U), rel=1e-12, abs=0)
    s.close()


def test_noalloc_call_allocates_nothing():
    """After the first call (which looks up the buffer address), a call changes
    neither torch's allocated bytes nor the device's free memory."""
    p = _problem(2, (200, 211), 7)
    s = htd.Solver(p)
    F = _dev(W.random_rhs(1, p.n))
    U = _dev(W.random_rhs(2, p.n) * 1e-4)
    htd.htd_residual_norm_noalloc(s.handle, F, U)
    torch.cuda.synchronize()
    used0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    v = htd.htd_residual_norm_noalloc(s.handle, F, U)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == used0
    assert torch.cuda.mem_get_info()[0] == free0
    assert v == pytest.approx(htd.htd_residual_norm(s.handle, F, U), rel=1e-12, abs=0)
    s.close()


def test_noalloc_at_the_size_limit_matches_the_oracle():
    """N = HTD_NOALLOC_MAX_NODES (512 x 512): the relative residual equals the one
    computed from the FP64 oracle's operator, ||F - H U|| / ||F||."""
    p = _problem(2, (512, 512), 9)
    assert math.prod(p.n) == htd.HTD_NOALLOC_MAX_NODES
    s = htd.Solver(p, restart=1)
    Fh = W.random_rhs(1, p.n)
    Uh = W.random_rhs(2, p.n) * 1e-4
    o = oracle.Oracle(p)
    want = np.linalg.norm(Fh - o.apply_H(Uh)) / np.linalg.norm(Fh)
    got = htd.htd_residual_norm_noalloc(s.handle, _dev(Fh), _dev(Uh))
    assert got == pytest.approx(want, rel=1e-12, abs=0)
    s.close()


def test_noalloc_on_a_separate_stream():
    """The call on a non-default stream that is not capturing: the stream's
    pending work (the operands written on it) is ordered before the call."""
    p = _problem(3, (33, 30, 28), 8)
    s = htd.Solver(p)
    st = torch.cuda.Stream()
    Fh, Uh = W.random_rhs(1, p.n), W.random_rhs(2, p.n) * 1e-4
    with torch.cuda.stream(st):
        F = torch.from_numpy(np.ascontiguousarray(Fh)).to("cuda", non_blocking=False)
        U = torch.from_numpy(np.ascontiguousarray(Uh)).to("cuda", non_blocking=False)
        got = htd.htd_residual_norm_noalloc(s.handle, F, U, stream=st)
    torch.cuda.synchronize()
    assert got == pytest.approx(htd.htd_residual_norm(s.handle, F, U), rel=1e-12, abs=0)
    s.close()


def test_noalloc_refuses_problems_larger_than_its_buffer():
    p = _problem(2, (600, 600), 4)
    assert math.prod(p.n) > htd.HTD_NOALLOC_MAX_NODES
    s = htd.Solver(p, restart=1)
    F = torch.zeros(p.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(htd.HtdError) as e:
        htd.htd_residual_norm_noalloc(s.handle, F, F.clone())
    assert e.value.status == 8
    s.close()
