"""FP64 CPU oracle for the time-domain Helmholtz preconditioner (test infrastructure).

This package is the checker, not the product.  Only the test suite, the smoke
check and the benchmark's CPU-baseline / reference leg may import it.  It wraps
``htd_oracle.c`` (plain C, double precision) with ctypes and shares no code with
the CUDA library.

Functions take a ``workloads.Problem`` (grid, c per cell, R per node, physical
omega, T, rho) and a stencil name ("q1mix", "fd5", or "family" with the mass
and stiffness weights stencil_a, stencil_gamma).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "htd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

STENCILS = {"q1mix": 0, "fd5": 1, "family": 2}
MODES = {"table1": 0, "exact": 1}
PRECONDS = {"identity": 0, "table1": 1, "exact": 2, "direct": 3}
KRYLOV = {"fgmres": 0, "left": 1}
DAMPING = {"node": 0, "cell": 1}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_longlong * 3), ("h", ctypes.c_double),
                ("stencil", ctypes.c_int), ("c_cell", ctypes.c_void_p),
                ("R_node", ctypes.c_void_p), ("omega_phys", ctypes.c_double),
                ("damping", ctypes.c_int), ("stencil_a", ctypes.c_double),
                ("stencil_gamma", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("k_min", ctypes.c_double), ("k_max", ctypes.c_double),
                ("omega", ctypes.c_double), ("lam_max_reH", ctypes.c_double),
                ("lam_max_A", ctypes.c_double), ("nP", ctypes.c_int),
                ("dt", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("T", ctypes.c_int), ("rho", ctypes.c_double), ("nsteps", ctypes.c_longlong),
                ("integrator", ctypes.c_int), ("lam_max_imH", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("precond_applies", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_res_true", ctypes.c_double), ("rel_res_est", ctypes.c_double),
                ("hist_len", ctypes.c_int), ("hist", ctypes.c_double * 4096)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    """Declare the argument types of the C entry points on a loaded library."""
    P = ctypes.POINTER(_Problem)
    Q = ctypes.POINTER(_Params)
    vp = ctypes.c_void_p
    lib.ora_tables.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp]
    lib.ora_tables_family.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, vp, vp]
    lib.ora_setup.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int, Q]
    lib.ora_setup_abd.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int, Q]
    lib.ora_abd_step.argtypes = [P, Q, vp, vp, vp, vp]
    lib.ora_apply_imH.argtypes = [P, vp, ctypes.c_longlong, vp]
    lib.ora_apply_reH.argtypes = [P, vp, ctypes.c_longlong, vp]
    lib.ora_apply_H.argtypes = [P, vp, vp]
    lib.ora_assemble_H.argtypes = [P, ctypes.c_longlong, vp, vp, vp, vp]
    lib.ora_assemble_H.restype = ctypes.c_longlong
    lib.ora_window.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.ora_window.restype = ctypes.c_double
    lib.ora_acd_step.argtypes = [P, Q, vp, vp, vp, vp]
    lib.ora_precond.argtypes = [P, Q, ctypes.c_int, vp, vp]
    lib.ora_precond_project.argtypes = [P, Q, ctypes.c_int, vp, vp]
    lib.ora_project_states.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_longlong,
                                       ctypes.c_longlong, vp, vp]
    lib.ora_direct_solve.argtypes = [P, vp, vp]
    lib.ora_grad.argtypes = [P, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.ora_grad_td.argtypes = [P, Q, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp,
                                vp, vp, vp]
    lib.ora_gmres.argtypes = [P, Q, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_double,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(_Info)]
    return lib


@contextlib.contextmanager
def use_library(path: str):
    """Run the oracle from another build of its source (tests that plant a
    mistake in a copy of htd_oracle.c and check that the pins catch it)."""
    global _lib
    saved = _load()
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield _lib
    finally:
        _lib = saved


def compile_library(src_path: str, out_path: str) -> str:
    """Compile a copy of the oracle source with the flags build() uses."""
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off", "-o", out_path, src_path, "-lm"])
    return out_path


def source_path() -> str:
    return _SRC


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Oracle:
    """One problem bound to the C oracle.  Keeps its input arrays alive."""

    def __init__(self, prob, stencil: str = "q1mix", nP: int = 0, T: int | None = None,
                 rho: float | None = None, integrator: str = "acd", damping: str = "node",
                 stencil_a: float = 0.5, stencil_gamma: float = 1.0):
        self.lib = _load()
        self.prob = prob
        self.ndim = prob.ndim
        self.n = tuple(int(m) for m in prob.n)
        self.N = int(np.prod(self.n))
        self.c = np.ascontiguousarray(prob.c_cell, dtype=np.float64)
        self.R = np.ascontiguousarray(prob.R_node, dtype=np.float64)
        assert self.c.size == int(np.prod([m + 1 for m in self.n]))
        assert self.R.size == self.N
        p = _Problem()
        p.ndim = prob.ndim
        for a in range(3):
            p.n[a] = self.n[a] if a < prob.ndim else 1
        p.h = prob.h
        p.stencil = STENCILS[stencil]
        p.c_cell = _ptr(self.c)
        p.R_node = _ptr(self.R)
        p.omega_phys = prob.omega
        p.damping = DAMPING[damping]
        p.stencil_a = float(stencil_a)
        p.stencil_gamma = float(stencil_gamma)
        self._p = p
        self.params = _Params()
        setup = self.lib.ora_setup_abd if integrator == "abd" else self.lib.ora_setup
        rc = setup(ctypes.byref(p), int(prob.T if T is None else T),
                   float(prob.rho if rho is None else rho), int(nP), ctypes.byref(self.params))
        if rc != 0:
            raise ValueError(f"oracle setup failed (rc={rc})")

    # ---- parameters -------------------------------------------------------
    def param_dict(self) -> dict:
        q = self.params
        return {f: getattr(q, f) for f, _ in _Params._fields_}

    # ---- operator ---------------------------------------------------------
    def _c(self, x) -> np.ndarray:
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128).reshape(-1))
        assert x.size == self.N
        return x

    def apply_H(self, U) -> np.ndarray:
        U = self._c(U)
        out = np.empty_like(U)
        self.lib.ora_apply_H(ctypes.byref(self._p), _ptr(U), _ptr(out))
        return out.reshape(self.n)

    def apply_reH(self, u) -> np.ndarray:
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
        out = np.empty_like(u)
        self.lib.ora_apply_reH(ctypes.byref(self._p), _ptr(u), 1, _ptr(out))
        return out.reshape(self.n)

    def assemble_H(self):
        """(rows, cols, values) triplets of H; duplicates are to be summed."""
        cnt = self.lib.ora_assemble_H(ctypes.byref(self._p), 0, None, None, None, None)
        rows = np.empty(cnt, np.int64)
        cols = np.empty(cnt, np.int64)
        re = np.empty(cnt)
        im = np.empty(cnt)
        self.lib.ora_assemble_H(ctypes.byref(self._p), cnt, _ptr(rows), _ptr(cols),
                                _ptr(re), _ptr(im))
        return rows, cols, re + 1j * im

    def H_sparse(self):
        import scipy.sparse as sp
        r, c, v = self.assemble_H()
        return sp.csr_matrix((v, (r, c)), shape=(self.N, self.N))

    # ---- method -----------------------------------------------------------
    def window(self, s: float, rho: float | None = None) -> float:
        return self.lib.ora_window(float(s), float(self.params.rho if rho is None else rho))

    def apply_imH(self, u) -> np.ndarray:
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
        out = np.empty_like(u)
        self.lib.ora_apply_imH(ctypes.byref(self._p), _ptr(u), 1, _ptr(out))
        return out.reshape(self.n)

    def abd_step(self, un, unm1, fn) -> np.ndarray:
        un, unm1, fn = self._c(un), self._c(unm1), self._c(fn)
        out = np.empty_like(un)
        self.lib.ora_abd_step(ctypes.byref(self._p), ctypes.byref(self.params),
                              _ptr(un), _ptr(unm1), _ptr(fn), _ptr(out))
        return out.reshape(self.n)

    def acd_step(self, un, unm1, fn) -> np.ndarray:
        un, unm1, fn = self._c(un), self._c(unm1), self._c(fn)
        out = np.empty_like(un)
        self.lib.ora_acd_step(ctypes.byref(self._p), ctypes.byref(self.params),
                              _ptr(un), _ptr(unm1), _ptr(fn), _ptr(out))
        return out.reshape(self.n)

    def precond(self, F, mode: str = "table1", periods: int = 1) -> np.ndarray:
        """Table 1 ("table1"), S_T ("exact"), or the Table 1 run read out by the
        e^{-i omega t} projection of its last `periods` periods ("project")."""
        F = self._c(F)
        out = np.empty_like(F)
        if mode == "project":
            rc = self.lib.ora_precond_project(ctypes.byref(self._p), ctypes.byref(self.params),
                                              int(periods), _ptr(F), _ptr(out))
        else:
            rc = self.lib.ora_precond(ctypes.byref(self._p), ctypes.byref(self.params),
                                      MODES[mode], _ptr(F), _ptr(out))
        if rc:
            raise ValueError("bad mode or periods")
        return out.reshape(self.n)

    def direct_solve(self, F) -> np.ndarray:
        F = self._c(F)
        out = np.empty_like(F)
        if self.lib.ora_direct_solve(ctypes.byref(self._p), _ptr(F), _ptr(out)):
            raise ArithmeticError("singular H")
        return out.reshape(self.n)

    def grad(self, F, rec_idx, d):
        """Misfit 1/2 sum_s ||P U_s - d_s||^2 and its gradient with respect to
        m = c^-2 per cell and R per node (direct solves).  F: (nsrc, *n), rec_idx:
        node linear indices, d: (nsrc, nrec).  Returns (J, grad_m, grad_R)."""
        F = np.ascontiguousarray(np.asarray(F, dtype=np.complex128).reshape(-1, self.N))
        nsrc = F.shape[0]
        rec = np.ascontiguousarray(np.asarray(rec_idx, dtype=np.int64).reshape(-1))
        d = np.ascontiguousarray(np.asarray(d, dtype=np.complex128).reshape(nsrc, rec.size))
        gm = np.zeros(self.c.shape)
        gR = np.zeros(self.n)
        J = ctypes.c_double()
        if self.lib.ora_grad(ctypes.byref(self._p), nsrc, _ptr(F), int(rec.size), _ptr(rec),
                             _ptr(d), _ptr(gm), _ptr(gR), ctypes.byref(J)):
            raise ArithmeticError("singular H")
        return J.value, gm, gR

    def grad_td(self, F, rec_idx, d, mode: str = "table1"):
        """Misfit 1/2 sum_s ||P(P F_s) - d_s||^2 of the preconditioner's own
        approximate solution (one application, mode "table1" or "exact") and its
        gradient through the recurrence with respect to m = c^-2 per cell and R
        per node, omega, dt and n_P held at this oracle's values.
        Returns (J, grad_m, grad_R)."""
        F = np.ascontiguousarray(np.asarray(F, dtype=np.complex128).reshape(-1, self.N))
        nsrc = F.shape[0]
        rec = np.ascontiguousarray(np.asarray(rec_idx, dtype=np.int64).reshape(-1))
        d = np.ascontiguousarray(np.asarray(d, dtype=np.complex128).reshape(nsrc, rec.size))
        gm = np.zeros(self.c.shape)
        gR = np.zeros(self.n)
        J = ctypes.c_double()
        if self.lib.ora_grad_td(ctypes.byref(self._p), ctypes.byref(self.params), MODES[mode],
                                nsrc, _ptr(F), int(rec.size), _ptr(rec), _ptr(d), _ptr(gm),
                                _ptr(gR), ctypes.byref(J)):
            raise ValueError("bad mode")
        return J.value, gm, gR

    def with_params(self, other: "Oracle") -> "Oracle":
        """Use another oracle's recurrence parameters (omega, dt, n_P, ...) for this
        problem: a perturbed model evaluated with the parameters held fixed."""
        ctypes.memmove(ctypes.byref(self.params), ctypes.byref(other.params),
                       ctypes.sizeof(_Params))
        return self

    def gmres(self, F, krylov: str = "fgmres", precond: str = "table1", tol: float = 1e-6,
              restart: int = 20, maxit: int = 200, fixed: bool = False, U0=None):
        F = self._c(F)
        U = np.zeros_like(F) if U0 is None else self._c(U0).copy()
        info = _Info()
        rc = self.lib.ora_gmres(ctypes.byref(self._p), ctypes.byref(self.params),
                                KRYLOV[krylov], PRECONDS[precond], _ptr(F), _ptr(U),
                                float(tol), int(restart), int(maxit), int(bool(fixed)),
                                ctypes.byref(info))
        if rc:
            raise ValueError("gmres failed")
        d = {f: getattr(info, f) for f, _ in _Info._fields_ if f != "hist"}
        d["hist"] = list(info.hist[: info.hist_len])
        return U.reshape(self.n), d


def project_states(states: np.ndarray, nP: int, j_first: int) -> np.ndarray:
    """(2 / n_acc) sum_k e^{-i 2 pi (j_first + k) / nP} states[k] for real states of
    shape (n_acc, ...)."""
    lib = _load()
    st = np.ascontiguousarray(states, dtype=np.float64)
    n_acc = st.shape[0]
    N = int(np.prod(st.shape[1:]))
    out = np.empty(N, dtype=np.complex128)
    lib.ora_project_states(N, int(nP), int(j_first), n_acc, _ptr(st), _ptr(out))
    return out.reshape(st.shape[1:])


def tables(ndim: int, stencil: str = "q1mix", stencil_a: float = 0.5,
           stencil_gamma: float = 1.0):
    """(S, M) Hamming-distance tables used by the oracle (length ndim + 1)."""
    lib = _load()
    S = np.zeros(4)
    M = np.zeros(4)
    if stencil == "family":
        rc = lib.ora_tables_family(ndim, float(stencil_a), float(stencil_gamma), _ptr(S), _ptr(M))
    else:
        rc = lib.ora_tables(ndim, STENCILS[stencil], _ptr(S), _ptr(M))
    if rc:
        raise ValueError("bad stencil")
    return S[: ndim + 1].copy(), M[: ndim + 1].copy()
