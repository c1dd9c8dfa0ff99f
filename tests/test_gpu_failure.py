"""Failure paths on the GPU, made without a fault or a hang.

- A device-side wait that runs out: htd_set_wait_limit's stall test makes the
  first neighbour wait of every CTA of the blocked 2-D kernel wait on a barrier
  that nothing arrives on, bounded by a short limit.  The kernel records the
  timeout and finishes; the solve returns HTD_ERR_TIMEOUT; the same handle then
  solves normally once the limit and the stall are reset.
- A device allocation that fails: htd_test_fail_alloc makes allocation number k
  of htd_create fail (host-side injection).  Every k up to the last allocation
  gives HTD_ERR_OOM and releases all that create had taken; then a create
  without injection succeeds.
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

TIMEOUT, OOM = 7, 3


def _problem(n=(129, 161)):
    """A 2-D heterogeneous problem with T = its side length in wavelengths (the
    workloads' recipe), so that FGMRES(20) converges in a few dozen steps."""
    h = 1.0 / (max(n) - 1)
    g = W.gaussian_random_field(11, tuple(m + 1 for m in n), 0.05 / h)
    c = np.clip(3.0 + 0.75 * g, 1.5, 4.5)
    omega = 2 * math.pi * c.min() / (8 * h)
    R = W.damping_profile(2, n, 12, 2 * omega)
    T = W.periods_for(max(n), h, float(c.min()), omega)
    return W.Problem("failure", 2, tuple(n), h, c, R, omega, W.point_source(2, n, h), T)


def test_neighbour_wait_runs_out_then_the_handle_solves():
    p = _problem()
    s = htd.Solver(p, precision="mixed", tblock=8, tb_form=htd.TB_PAIR)
    assert s.params["step_kernel"] == 1 and s.params["tile"][2] == 2
    F = torch.from_numpy(np.ascontiguousarray(p.F)).cuda()
    htd.htd_set_wait_limit(s.handle, 1_000_000, stall_test=True)     # 1 ms, stalled
    U = s.zeros()
    with pytest.raises(htd.HtdError) as e:
        htd.htd_gmres_solve(s.handle, F, U, 1e-6, 2)
    assert e.value.status == TIMEOUT
    # the context is still usable and the handle solves once the stall is off
    htd.htd_set_wait_limit(s.handle, 0, stall_test=False)
    U.zero_()
    info = htd.htd_gmres_solve(s.handle, F, U, 1e-6, 200)
    assert info["converged"]
    Ug = U.cpu().numpy()
    rel = np.linalg.norm(p.F - oracle.Oracle(p).apply_H(Ug)) / np.linalg.norm(p.F)
    assert rel <= 1e-6
    # a short limit without the stall does not give up on healthy waits
    htd.htd_set_wait_limit(s.handle, 50_000_000, stall_test=False)
    U.zero_()
    assert htd.htd_gmres_solve(s.handle, F, U, 1e-6, 200)["converged"]
    s.close()


def test_wait_limit_option_is_checked():
    s = htd.Solver(_problem((65, 70)), precision="mixed", wait_limit_ns=2_000_000_000)
    with pytest.raises(htd.HtdError) as e:
        htd.htd_set_wait_limit(s.handle, -1)
    assert e.value.status == 1
    s.close()


@pytest.mark.parametrize("precision,ndim", [("mixed", 2), ("fp64", 2), ("mixed", 3)])
def test_every_failed_allocation_of_create_is_reported_and_released(precision, ndim):
    if ndim == 2:
        p = _problem((769, 801))
    else:
        p = W.config_3d_layered(64, layer=6, T=2)
    kw = dict(precision=precision, restart=8)
    htd.Solver(p, **kw).close()                       # kernels loaded, tuner warmed up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seen_ok = False
    try:
        for k in range(200):
            htd.htd_test_fail_alloc(k)
            try:
                s = htd.Solver(p, **kw)
            except htd.HtdError as e:
                assert e.status == OOM, (k, e)
                torch.cuda.synchronize()
                free = torch.cuda.mem_get_info()[0]
                assert abs(free - free0) <= (2 << 20), (k, free0 - free)
                continue
            # allocation k was never reached: create made fewer allocations
            s.close()
            seen_ok = True
            assert k > 10
            break
    finally:
        htd.htd_test_fail_alloc(-1)
    assert seen_ok
    s = htd.Solver(p, **kw)
    s.close()
