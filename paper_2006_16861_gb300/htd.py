"""Thin ctypes binding of libhtd (include/htd.h) -- argument marshalling only.

The functions carry the C names (``htd_create``, ``htd_apply_precond``,
``htd_gmres_solve`` ...).  Device buffers are torch CUDA tensors (complex128,
contiguous); streams are torch streams.  Every step of the computation runs in
libhtd's CUDA kernels; there is no CPU fallback: if the library is missing or
no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _native

HTD_OK = 0
STATUS = {0: "HTD_OK", 1: "HTD_ERR_ARG", 2: "HTD_ERR_CUDA", 3: "HTD_ERR_OOM",
          4: "HTD_ERR_UNSTABLE", 5: "HTD_ERR_NONFINITE", 6: "HTD_ERR_NOT_CONVERGED",
          7: "HTD_ERR_TIMEOUT", 8: "HTD_ERR_SIZE"}
HTD_NOALLOC_MAX_NODES = 262144
FP64, MIXED = 0, 1
MODE_TABLE1, MODE_EXACT, MODE_PROJECT = 0, 1, 2
ACD, ABD = 0, 1
DAMP_NODE, DAMP_CELL = 0, 1
FGMRES, LEFT_GMRES = 0, 1
STENCIL_Q1MIX, STENCIL_FD5, STENCIL_FAMILY = 0, 1, 2
BC_DIRICHLET = 0
TB_ANY, TB_COLUMN, TB_PAIR, TB_PAIR_SD, TB_RESIDENT = 0, 1, 2, 3, 4
S3_PAIR, S3_ZMARCH, S3_NODE_32x8, S3_NODE_64x4, S3_NODE_128x2 = 0, 1, 2, 3, 4
LAUNCH_NO_OVERLAP, LAUNCH_NO_GRAPH, LAUNCH_NO_GROUP = 1, 2, 4

#: every function include/htd.h declares (checked by the ABI test)
EXPORTS = ("htd_default_options", "htd_create", "htd_destroy", "htd_plan", "htd_get_params",
           "htd_apply_precond", "htd_apply_H", "htd_residual_norm", "htd_residual_norm_noalloc",
           "htd_gmres_solve", "htd_grad", "htd_grad_td",
           "htd_gmres_solve_host", "htd_batch_create", "htd_batch_destroy",
           "htd_batch_apply_precond", "htd_batch_gmres_solve", "htd_batch_describe",
           "htd_batch_set_form",
           "htd_set_wait_limit",
           "htd_test_fail_alloc", "htd_status_string")


class HtdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_msg(status)})")


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("mode", ctypes.c_int), ("krylov", ctypes.c_int),
                ("T", ctypes.c_int), ("rho", ctypes.c_double), ("nP", ctypes.c_int),
                ("stencil", ctypes.c_int), ("restart", ctypes.c_int), ("max_rhs", ctypes.c_int),
                ("proj_periods", ctypes.c_int), ("integrator", ctypes.c_int),
                ("damping", ctypes.c_int), ("stencil_a", ctypes.c_double),
                ("stencil_gamma", ctypes.c_double), ("tblock", ctypes.c_int),
                ("tb_rows", ctypes.c_int), ("tb_form", ctypes.c_int),
                ("s3_kernel", ctypes.c_int), ("s3_stages", ctypes.c_int),
                ("s3_zchunk", ctypes.c_int), ("s3_rhs_per_cta", ctypes.c_int),
                ("launch", ctypes.c_int), ("wait_limit_ns", ctypes.c_longlong)]


class Params(ctypes.Structure):
    _fields_ = [("k_min", ctypes.c_double), ("k_max", ctypes.c_double),
                ("omega_c", ctypes.c_double), ("lam_max_reH", ctypes.c_double),
                ("lam_max_A", ctypes.c_double), ("dt", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("rho", ctypes.c_double),
                ("nP", ctypes.c_int), ("T", ctypes.c_int), ("steps", ctypes.c_longlong),
                ("steps_per_launch", ctypes.c_int), ("tile", ctypes.c_int * 3),
                ("ctas_per_sm", ctypes.c_int), ("waves", ctypes.c_int),
                ("step_kernel", ctypes.c_int), ("rhs_per_cta", ctypes.c_int)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "tile"}
        d["tile"] = list(self.tile)
        return d



class BatchDesc(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int), ("systems", ctypes.c_int),
                ("grouped", ctypes.c_int), ("group_ctas", ctypes.c_int),
                ("group_tasks", ctypes.c_longlong), ("group_steps_per_task", ctypes.c_int),
                ("form", ctypes.c_int), ("ns_per_update_plain", ctypes.c_double),
                ("ns_per_update_group", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("precond_applies", ctypes.c_int), ("converged", ctypes.c_int),
                ("steps", ctypes.c_longlong), ("rel_res_true", ctypes.c_double),
                ("rel_res_est", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_precond", ctypes.c_double), ("launches", ctypes.c_longlong),
                ("reorth", ctypes.c_int), ("hist_len", ctypes.c_int),
                ("hist", ctypes.c_double * 256)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "hist"}
        d["hist"] = list(self.hist[: self.hist_len])
        return d


_lib = None


def library_path() -> str:
    return _native.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libhtd.so (building it first if needed).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _native.build() if build_if_missing else _native.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libhtd.so not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.htd_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.htd_default_options.restype = None
    lib.htd_create.argtypes = [ctypes.POINTER(Grid), vp, vp, d, i, ctypes.POINTER(Options),
                               ctypes.POINTER(vp)]
    lib.htd_destroy.argtypes = [vp]
    lib.htd_plan.argtypes = [ctypes.POINTER(Grid), vp, vp, d, i, ctypes.POINTER(Options),
                             ctypes.POINTER(Params)]
    lib.htd_get_params.argtypes = [vp, ctypes.POINTER(Params)]
    lib.htd_apply_precond.argtypes = [vp, vp, vp, vp]
    lib.htd_apply_H.argtypes = [vp, vp, vp, vp]
    lib.htd_residual_norm.argtypes = [vp, vp, vp, vp, ctypes.POINTER(d), vp]
    lib.htd_residual_norm_noalloc.argtypes = [vp, vp, vp, ctypes.POINTER(d), vp]
    lib.htd_gmres_solve.argtypes = [vp, vp, vp, d, i, vp, ctypes.POINTER(SolveInfo)]
    lib.htd_gmres_solve_host.argtypes = [vp, vp, vp, d, i, vp, ctypes.POINTER(SolveInfo)]
    lib.htd_grad.argtypes = [vp, i, vp, i, vp, vp, d, i, vp, vp, ctypes.POINTER(d), vp,
                             ctypes.POINTER(SolveInfo)]
    lib.htd_grad_td.argtypes = [vp, i, vp, i, vp, vp, i, vp, vp, ctypes.POINTER(d), vp]
    lib.htd_batch_create.argtypes = [i, vp, vp, ctypes.POINTER(vp)]
    lib.htd_batch_destroy.argtypes = [vp]
    lib.htd_batch_apply_precond.argtypes = [vp, vp, vp, vp]
    lib.htd_batch_gmres_solve.argtypes = [vp, vp, vp, d, i, vp, vp]
    lib.htd_batch_describe.argtypes = [vp, ctypes.POINTER(BatchDesc)]
    lib.htd_batch_set_form.argtypes = [vp, i]
    lib.htd_set_wait_limit.argtypes = [vp, ctypes.c_longlong, i]
    lib.htd_test_fail_alloc.argtypes = [ctypes.c_longlong]
    lib.htd_test_fail_alloc.restype = None
    lib.htd_status_string.argtypes = [i]
    lib.htd_status_string.restype = ctypes.c_char_p
    for f in EXPORTS:
        if f not in ("htd_default_options", "htd_status_string", "htd_test_fail_alloc"):
            getattr(lib, f).restype = i
    _lib = lib
    return lib


def _msg(status: int) -> str:
    try:
        return load(False).htd_status_string(status).decode()
    except Exception:  # noqa: BLE001 - only used to format an error message
        return "?"


def _check(st: int, where: str, allow=(HTD_OK,)) -> int:
    if st not in allow:
        raise HtdError(st, where)
    return st


def _dev_ptr(t) -> int:
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128
            and t.is_contiguous()):
        raise TypeError("expected a contiguous complex128 CUDA tensor")
    return t.data_ptr()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _host_ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---- the C entry points with the same names ---------------------------------

def htd_default_options() -> Options:
    o = Options()
    load().htd_default_options(ctypes.byref(o))
    return o


def _grid(ndim: int, n, h: float) -> Grid:
    g = Grid()
    g.ndim = ndim
    for a in range(3):
        g.n[a] = int(n[a]) if a < min(ndim, len(n)) else 1
    g.h = h
    return g


def htd_plan(ndim: int, n, h: float, c_cell: np.ndarray, R_node: np.ndarray,
             omega_phys: float, bc: int = BC_DIRICHLET, options: Options | None = None) -> dict:
    """Host-only parameter selection (no GPU needed)."""
    c = np.ascontiguousarray(c_cell, dtype=np.float64)
    R = np.ascontiguousarray(R_node, dtype=np.float64)
    out = Params()
    st = load().htd_plan(ctypes.byref(_grid(ndim, n, h)), _host_ptr(c), _host_ptr(R),
                         float(omega_phys), int(bc),
                         ctypes.byref(options) if options is not None else None, ctypes.byref(out))
    _check(st, "htd_plan")
    return out.as_dict()


def htd_create(ndim: int, n, h: float, c_cell: np.ndarray, R_node: np.ndarray,
               omega_phys: float, bc: int = BC_DIRICHLET, options: Options | None = None) -> int:
    lib = load()
    c = np.ascontiguousarray(c_cell, dtype=np.float64)
    R = np.ascontiguousarray(R_node, dtype=np.float64)
    handle = ctypes.c_void_p()
    st = lib.htd_create(ctypes.byref(_grid(ndim, n, h)), _host_ptr(c), _host_ptr(R),
                        float(omega_phys), int(bc),
                        ctypes.byref(options) if options is not None else None,
                        ctypes.byref(handle))
    _check(st, "htd_create")
    return handle.value


def htd_destroy(handle: int) -> None:
    _check(load().htd_destroy(handle), "htd_destroy")


def htd_get_params(handle: int) -> dict:
    out = Params()
    _check(load().htd_get_params(handle, ctypes.byref(out)), "htd_get_params")
    return out.as_dict()


def htd_apply_precond(handle: int, F, U, stream=None) -> None:
    _check(load().htd_apply_precond(handle, _dev_ptr(F), _dev_ptr(U), _stream_ptr(stream)),
           "htd_apply_precond")


def htd_apply_H(handle: int, X, Y, stream=None) -> None:
    _check(load().htd_apply_H(handle, _dev_ptr(X), _dev_ptr(Y), _stream_ptr(stream)),
           "htd_apply_H")


def htd_residual_norm(handle: int, F, U, r=None, stream=None) -> float:
    rel = ctypes.c_double()
    _check(load().htd_residual_norm(handle, _dev_ptr(F), _dev_ptr(U),
                                    None if r is None else _dev_ptr(r), ctypes.byref(rel),
                                    _stream_ptr(stream)), "htd_residual_norm")
    return rel.value


def htd_residual_norm_noalloc(handle: int, F, U, stream=None) -> float:
    """||F - H U|| / ||F|| without any device allocation by the call: the residual
    and the partial sums live in a fixed buffer inside the library (problems up
    to HTD_NOALLOC_MAX_NODES nodes).  For callers that must not allocate while
    they run, e.g. under CUDA stream capture or with an application-owned
    memory pool.  Calls whose GPU work overlaps race on that buffer."""
    rel = ctypes.c_double()
    _check(load().htd_residual_norm_noalloc(handle, _dev_ptr(F), _dev_ptr(U), ctypes.byref(rel),
                                            _stream_ptr(stream)), "htd_residual_norm_noalloc")
    return rel.value


def htd_gmres_solve(handle: int, F, U, tol: float, max_iters: int, stream=None,
                    allow_not_converged: bool = False) -> dict:
    info = SolveInfo()
    allow = (HTD_OK, 6) if allow_not_converged else (HTD_OK,)
    st = load().htd_gmres_solve(handle, _dev_ptr(F), _dev_ptr(U), float(tol), int(max_iters),
                                _stream_ptr(stream), ctypes.byref(info))
    _check(st, "htd_gmres_solve", allow)
    d = info.as_dict()
    d["status"] = STATUS[st]
    return d


def htd_gmres_solve_host(handle: int, F_host: np.ndarray, U_host: np.ndarray, tol: float,
                         max_iters: int, stream=None, allow_not_converged: bool = False) -> dict:
    if F_host.dtype != np.complex128 or U_host.dtype != np.complex128:
        raise TypeError("host vectors must be complex128")
    if not (F_host.flags.c_contiguous and U_host.flags.c_contiguous):
        raise TypeError("host vectors must be C-contiguous")
    info = SolveInfo()
    allow = (HTD_OK, 6) if allow_not_converged else (HTD_OK,)
    st = load().htd_gmres_solve_host(handle, F_host.ctypes.data, U_host.ctypes.data, float(tol),
                                     int(max_iters), _stream_ptr(stream), ctypes.byref(info))
    _check(st, "htd_gmres_solve_host", allow)
    d = info.as_dict()
    d["status"] = STATUS[st]
    return d


def htd_grad(handle: int, F, rec_idx: np.ndarray, d, tol: float, max_iters: int,
             grad_m=None, grad_R=None, stream=None) -> tuple:
    """Receiver misfit J = 1/2 sum_s ||P U_s - d_s||^2 and (if grad_m / grad_R, float64
    CUDA tensors of the cell / node shapes, are given) its gradient with respect to
    c^-2 per cell and R per node.  F: (nsrc, *n) complex128 CUDA tensor; rec_idx:
    int64 node indices (host); d: (nsrc, nrec) complex128 CUDA tensor."""
    import torch
    nsrc = int(F.shape[0])
    rec = np.ascontiguousarray(np.asarray(rec_idx, dtype=np.int64).reshape(-1))
    for g in (grad_m, grad_R):
        if g is not None and not (isinstance(g, torch.Tensor) and g.is_cuda and
                                  g.dtype == torch.float64 and g.is_contiguous()):
            raise TypeError("gradients must be contiguous float64 CUDA tensors")
    J = ctypes.c_double()
    info = SolveInfo()
    st = load().htd_grad(handle, nsrc, _dev_ptr(F), int(rec.size), rec.ctypes.data,
                         _dev_ptr(d) if rec.size else None, float(tol), int(max_iters),
                         None if grad_m is None else grad_m.data_ptr(),
                         None if grad_R is None else grad_R.data_ptr(), ctypes.byref(J),
                         _stream_ptr(stream), ctypes.byref(info))
    _check(st, "htd_grad")
    return J.value, info.as_dict()


def htd_batch_create(handles, nrhs) -> int:
    """A batch of instances (handles) carrying nrhs[i] right-hand sides each."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*handles)
    rs = (ctypes.c_int * n)(*[int(r) for r in nrhs])
    out = ctypes.c_void_p()
    _check(load().htd_batch_create(n, hs, rs, ctypes.byref(out)), "htd_batch_create")
    return out.value


def htd_batch_destroy(batch: int) -> None:
    _check(load().htd_batch_destroy(batch), "htd_batch_destroy")


def htd_batch_describe(batch: int) -> dict:
    """How the batch runs its applications (after the first one)."""
    out = BatchDesc()
    _check(load().htd_batch_describe(batch, ctypes.byref(out)), "htd_batch_describe")
    return out.as_dict()


def htd_batch_set_form(batch: int, form: int) -> None:
    """0 = decide by timing the first rounds of the next solve, 1 = every
    handle's own step sequence, 2 = the group's persistent launch."""
    _check(load().htd_batch_set_form(batch, int(form)), "htd_batch_set_form")


def _ptr_array(ts) -> ctypes.Array:
    return (ctypes.c_void_p * len(ts))(*[_dev_ptr(t) for t in ts])


def htd_batch_apply_precond(batch: int, Fs, Us, stream=None) -> None:
    """Fs[i], Us[i]: contiguous complex128 CUDA tensors of shape (nrhs[i], *n_i)."""
    _check(load().htd_batch_apply_precond(batch, _ptr_array(Fs), _ptr_array(Us),
                                          _stream_ptr(stream)), "htd_batch_apply_precond")


def htd_batch_gmres_solve(batch: int, Fs, Us, tol: float, max_iters: int, nsys: int,
                          stream=None, allow_not_converged: bool = False) -> list:
    """Lockstep FGMRES of every system; one info dict per system (instance-major)."""
    infos = (SolveInfo * nsys)()
    allow = (HTD_OK, 6) if allow_not_converged else (HTD_OK,)
    st = load().htd_batch_gmres_solve(batch, _ptr_array(Fs), _ptr_array(Us), float(tol),
                                      int(max_iters), _stream_ptr(stream), infos)
    _check(st, "htd_batch_gmres_solve", allow)
    out = [infos[k].as_dict() for k in range(nsys)]
    for d in out:
        d["status"] = STATUS[st]
    return out


def htd_grad_td(handle: int, F, rec_idx: np.ndarray, d, grad_m=None, grad_R=None,
                checkpoint_every: int = 0, stream=None) -> float:
    """Misfit J = 1/2 sum_s ||P(P F_s) - d_s||^2 of the preconditioner's own output and
    (into grad_m / grad_R, float64 CUDA tensors of the cell / node shapes, if given)
    its gradient through the recurrence.  F: (nsrc, *n) complex128 CUDA tensor;
    rec_idx: int64 node indices (host); d: (nsrc, nrec) complex128 CUDA tensor."""
    import torch
    nsrc = int(F.shape[0])
    rec = np.ascontiguousarray(np.asarray(rec_idx, dtype=np.int64).reshape(-1))
    for g in (grad_m, grad_R):
        if g is not None and not (isinstance(g, torch.Tensor) and g.is_cuda and
                                  g.dtype == torch.float64 and g.is_contiguous()):
            raise TypeError("gradients must be contiguous float64 CUDA tensors")
    J = ctypes.c_double()
    st = load().htd_grad_td(handle, nsrc, _dev_ptr(F), int(rec.size), rec.ctypes.data,
                            _dev_ptr(d) if rec.size else None, int(checkpoint_every),
                            None if grad_m is None else grad_m.data_ptr(),
                            None if grad_R is None else grad_R.data_ptr(), ctypes.byref(J),
                            _stream_ptr(stream))
    _check(st, "htd_grad_td")
    return J.value


def htd_set_wait_limit(handle: int, limit_ns: int, stall_test: bool = False) -> None:
    """Bound of the blocked 2-D kernel's neighbour waits (0 = 1 s); with
    stall_test the first such wait of every CTA runs out (test hook)."""
    _check(load().htd_set_wait_limit(handle, int(limit_ns), int(bool(stall_test))),
           "htd_set_wait_limit")


def htd_test_fail_alloc(after: int) -> None:
    """Test hook: the library's allocation number `after` (counted from now)
    fails as if the device were out of memory; negative switches it off."""
    load().htd_test_fail_alloc(int(after))


def htd_status_string(status: int) -> str:
    return load().htd_status_string(int(status)).decode()


# ---- convenience object ------------------------------------------------------

KERNEL_FIELDS = ("tb_rows", "tb_form", "s3_kernel", "s3_stages", "s3_zchunk", "launch",
                 "wait_limit_ns", "s3_rhs_per_cta")


def make_options(prob=None, precision: str = "fp64", mode: str = "table1",
                 krylov: str = "fgmres", stencil: str = "q1mix", restart: int = 20,
                 nP: int = 0, T: int | None = None, rho: float | None = None,
                 max_rhs: int = 1, proj_periods: int = 1, integrator: str = "acd",
                 damping: str = "node", stencil_a: float | None = None,
                 stencil_gamma: float | None = None, tblock: int = 0,
                 **kernel) -> Options:
    """htd_options from names; T and rho default to the problem's.  stencil
    "family" takes stencil_a (consistent-mass weight) and stencil_gamma (Q1
    stiffness weight).  Keyword arguments named like the kernel-selection
    fields (tb_rows, tb_form, s3_kernel, s3_stages, s3_zchunk, launch,
    wait_limit_ns) set those fields."""
    o = htd_default_options()
    for k, v in kernel.items():
        if k not in KERNEL_FIELDS:
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, int(v))
    if stencil_a is not None:
        o.stencil_a = float(stencil_a)
    if stencil_gamma is not None:
        o.stencil_gamma = float(stencil_gamma)
    o.tblock = int(tblock)
    o.integrator = {"acd": ACD, "abd": ABD}[integrator]
    o.damping = {"node": DAMP_NODE, "cell": DAMP_CELL}[damping]
    o.max_rhs = int(max_rhs)
    o.proj_periods = int(proj_periods)
    o.precision = {"fp64": FP64, "mixed": MIXED}[precision]
    o.mode = {"table1": MODE_TABLE1, "exact": MODE_EXACT, "project": MODE_PROJECT}[mode]
    o.krylov = {"fgmres": FGMRES, "left": LEFT_GMRES}[krylov]
    o.stencil = {"q1mix": STENCIL_Q1MIX, "fd5": STENCIL_FD5, "family": STENCIL_FAMILY}[stencil]
    o.restart = restart
    o.nP = nP
    if T is not None or prob is not None:
        o.T = int(prob.T if T is None else T)
    if rho is not None or prob is not None:
        o.rho = float(prob.rho if rho is None else rho)
    return o


def plan(prob, **kw) -> dict:
    """htd_plan for a workloads.Problem (host only)."""
    return htd_plan(prob.ndim, prob.n, prob.h, prob.c_cell, prob.R_node, prob.omega,
                    BC_DIRICHLET, make_options(prob, **kw))


class Solver:
    """One problem on the current CUDA device; owns an htd handle."""

    def __init__(self, prob, precision: str = "fp64", mode: str = "table1",
                 krylov: str = "fgmres", stencil: str = "q1mix", restart: int = 20,
                 nP: int = 0, T: int | None = None, rho: float | None = None,
                 max_rhs: int = 1, proj_periods: int = 1, integrator: str = "acd",
                 damping: str = "node", stencil_a: float | None = None,
                 stencil_gamma: float | None = None, tblock: int = 0, **kernel):
        o = make_options(prob, precision, mode, krylov, stencil, restart, nP, T, rho, max_rhs,
                         proj_periods, integrator, damping, stencil_a, stencil_gamma, tblock,
                         **kernel)
        self.max_rhs = int(max_rhs)
        self.prob = prob
        self.n = tuple(prob.n)
        self.handle = htd_create(prob.ndim, prob.n, prob.h, prob.c_cell, prob.R_node, prob.omega,
                                 BC_DIRICHLET, o)
        self.params = htd_get_params(self.handle)

    def close(self):
        if self.handle:
            htd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def zeros(self):
        import torch
        return torch.zeros(self.n, dtype=torch.complex128, device="cuda")

    def precond(self, F, U=None, stream=None):
        U = self.zeros() if U is None else U
        htd_apply_precond(self.handle, F, U, stream)
        return U

    def apply_H(self, X, Y=None, stream=None):
        Y = self.zeros() if Y is None else Y
        htd_apply_H(self.handle, X, Y, stream)
        return Y

    def grad(self, F, rec_idx, d, tol=1e-10, max_iters=400, stream=None, want_grad=True):
        """(J, grad_m, grad_R, info): misfit and gradient w.r.t. c^-2 per cell and R per node."""
        import torch
        gm = gR = None
        if want_grad:
            gm = torch.empty([m + 1 for m in self.n], dtype=torch.float64, device="cuda")
            gR = torch.empty(self.n, dtype=torch.float64, device="cuda")
        J, info = htd_grad(self.handle, F, rec_idx, d, tol, max_iters, gm, gR, stream)
        return J, gm, gR, info

    def grad_td(self, F, rec_idx, d, checkpoint_every=0, stream=None, want_grad=True):
        """(J, grad_m, grad_R): misfit of this preconditioner's own output and its
        gradient through the recurrence w.r.t. c^-2 per cell and R per node."""
        import torch
        gm = gR = None
        if want_grad:
            gm = torch.empty([m + 1 for m in self.n], dtype=torch.float64, device="cuda")
            gR = torch.empty(self.n, dtype=torch.float64, device="cuda")
        J = htd_grad_td(self.handle, F, rec_idx, d, gm, gR, checkpoint_every, stream)
        return J, gm, gR

    def solve(self, F, U=None, tol=1e-6, max_iters=400, stream=None, allow_not_converged=False):
        U = self.zeros() if U is None else U
        info = htd_gmres_solve(self.handle, F, U, tol, max_iters, stream, allow_not_converged)
        return U, info


class Batch:
    """Several Solvers, solver i carrying nrhs[i] right-hand sides, run together:
    one graph launch applies every preconditioner, FGMRES advances all systems
    in lockstep (htd_batch_*).  The solvers must outlive the batch."""

    def __init__(self, solvers, nrhs):
        self.solvers = list(solvers)
        self.nrhs = [int(r) for r in nrhs]
        self.handle = htd_batch_create([s.handle for s in self.solvers], self.nrhs)

    @property
    def nsys(self) -> int:
        return sum(self.nrhs)

    def close(self):
        if self.handle:
            htd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def zeros(self):
        import torch
        return [torch.zeros((r, *s.n), dtype=torch.complex128, device="cuda")
                for s, r in zip(self.solvers, self.nrhs)]

    def precond(self, Fs, Us=None, stream=None):
        Us = self.zeros() if Us is None else Us
        htd_batch_apply_precond(self.handle, Fs, Us, stream)
        return Us

    def describe(self) -> dict:
        return htd_batch_describe(self.handle)

    def set_form(self, form: int) -> None:
        htd_batch_set_form(self.handle, form)

    def solve(self, Fs, Us=None, tol=1e-6, max_iters=400, stream=None,
              allow_not_converged=False):
        Us = self.zeros() if Us is None else Us
        infos = htd_batch_gmres_solve(self.handle, Fs, Us, tol, max_iters, self.nsys, stream,
                                      allow_not_converged)
        return Us, infos
