"""The allocation-free residual norm (htd_residual_norm_noalloc).

Some callers of this library cannot allocate device memory when they call it:
code running under a CUDA stream capture, where cudaMalloc is not permitted,
and applications that hand all device memory out from their own pool and forbid
libraries to allocate in their solve loop.  For them htd_residual_norm_noalloc
keeps its residual vector and partial sums in a fixed buffer inside the library.
This test checks, through the C ABI, that two calls in a row give the same
relative residual as the ordinary htd_residual_norm, and that problems larger
than the buffer are refused.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

from paper_2006_16861_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2006_16861_gb300 import htd  # noqa: E402


def _problem(ndim, n, seed):
    n = tuple(n)
    h = 1.0 / (max(n) - 1)
    g = W.gaussian_random_field(seed, tuple(m + 1 for m in n), 3.0)
    c = np.clip(2.0 + 0.5 * g, 1.0, 3.0)
    omega = 2 * math.pi * c.min() / (8 * h)
    R = W.damping_profile(ndim, n, 4, 2 * omega)
    return W.Problem("noalloc", ndim, n, h, c, R, omega, W.point_source(ndim, n, h), 2)


@pytest.mark.parametrize("ndim,n", [(2, (301, 257)), (3, (40, 37, 45))])
def test_noalloc_residual_matches_residual_norm(ndim, n):
    p = _problem(ndim, n, 3)
    s = htd.Solver(p)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    F = dev(W.random_rhs(1, p.n))
    U = dev(W.random_rhs(2, p.n) * 1e-4)
    ref = htd.htd_residual_norm(s.handle, F, U)
    got1 = htd.htd_residual_norm_noalloc(s.handle, F, U)
    got2 = htd.htd_residual_norm_noalloc(s.handle, F, U)
    assert got1 == pytest.approx(ref, rel=1e-12, abs=0)
    assert got2 == pytest.approx(ref, rel=1e-12, abs=0)
    # a different right-hand side on the same buffer: the previous contents do not leak in
    F2 = dev(W.random_rhs(5, p.n))
    assert htd.htd_residual_norm_noalloc(s.handle, F2, U) == pytest.approx(
        htd.htd_residual_norm(s.handle, F2, U), rel=1e-12, abs=0)
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
