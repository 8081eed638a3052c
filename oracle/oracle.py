"""ctypes binding of the FP64 C oracle (test infrastructure only).

``build()`` compiles ``qc_oracle.c`` with gcc into ``oracle/_build/``; the
functions below marshal numpy arrays into the C structs and call it.  No
arithmetic of the method happens here.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

OC_DIAG, OC_FULL, OC_PHASE, OC_DELAY = 0, 1, 2, 3
_KIND = {"diag": OC_DIAG, "full": OC_FULL, "phase": OC_PHASE, "delay": OC_DELAY}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle (plain C99, -O2, no fast-math) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("n_row", C.c_int), ("n_chan", C.c_int), ("n_ant", C.c_int), ("n_time", C.c_int),
                ("data", C.c_void_p), ("model", C.c_void_p), ("weight", C.c_void_p),
                ("flag", C.c_void_p), ("ant1", C.c_void_p), ("ant2", C.c_void_p),
                ("time_idx", C.c_void_p)]


class _Term(C.Structure):
    _fields_ = [("type", C.c_int), ("n_tint", C.c_int), ("n_fint", C.c_int),
                ("t_map", C.c_void_p), ("f_map", C.c_void_p), ("params", C.c_void_p),
                ("gain_flags", C.c_void_p), ("solve", C.c_int), ("max_iter", C.c_int),
                ("tol", C.c_double), ("chan_freq", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("n_epochs", C.c_int), ("damping_mode", C.c_int), ("damping", C.c_double), ("div_flag", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            vp, i32 = C.c_void_p, C.c_int
            sig = {
                "oc_normal_equations": [vp, vp, i32, i32, vp, vp, vp],
                "oc_solve_term": [vp, vp, i32, i32, vp, vp],
                "oc_solve": [vp, vp, i32, vp, vp],
                "oc_residual": [vp, vp, i32, vp, vp],
                "oc_block_solve": [i32, vp, vp, vp],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.restype = C.c_int
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class OracleProblem:
    """Inputs in FP64: complex128 data/model, float64 weights (upcast from any input dtype)."""

    def __init__(self, data, model, weight, flag, ant1, ant2, time_idx, n_ant: int, n_time: int):
        self.data = np.ascontiguousarray(data, dtype=np.complex128)
        self.model = np.ascontiguousarray(model, dtype=np.complex128)
        self.weight = np.ascontiguousarray(weight, dtype=np.float64)
        self.flag = None if flag is None else np.ascontiguousarray(flag, dtype=np.uint8)
        self.ant1 = np.ascontiguousarray(ant1, dtype=np.int32)
        self.ant2 = np.ascontiguousarray(ant2, dtype=np.int32)
        self.time_idx = np.ascontiguousarray(time_idx, dtype=np.int32)
        self.n_row, self.n_chan = self.data.shape[0], self.data.shape[1]
        assert self.data.shape == (self.n_row, self.n_chan, 4)
        self.n_ant, self.n_time = int(n_ant), int(n_time)
        self._c = _Problem(self.n_row, self.n_chan, self.n_ant, self.n_time, _ptr(self.data),
                           _ptr(self.model), _ptr(self.weight), _ptr(self.flag), _ptr(self.ant1),
                           _ptr(self.ant2), _ptr(self.time_idx))

    @classmethod
    def from_obs(cls, obs) -> "OracleProblem":
        return cls(obs.data, obs.model, obs.weight, obs.flag, obs.ant1, obs.ant2, obs.time_idx,
                   obs.n_ant, obs.n_time)


class OracleTerm:
    """One chain term; ``params`` is complex128 [tint][fint][ant][4], float64 [..][2] (phase)
    or float64 [..][4] = (phi_X, tau_X, phi_Y, tau_Y) (delay, with ``chan_freq`` [n_chan])."""

    def __init__(self, kind: str, t_map, f_map, n_tint: int, n_fint: int, n_ant: int,
                 params=None, solve: bool = True, max_iter: int = 20, tol: float = 1e-6, chan_freq=None):
        self.kind = kind
        self.type = _KIND[kind]
        self.chan_freq = None
        if kind == "delay":
            if chan_freq is None:
                raise ValueError("a delay term needs chan_freq")
            self.chan_freq = np.ascontiguousarray(chan_freq, dtype=np.float64)
        self.t_map = np.ascontiguousarray(t_map, dtype=np.int32)
        self.f_map = np.ascontiguousarray(f_map, dtype=np.int32)
        self.n_tint, self.n_fint, self.n_ant = int(n_tint), int(n_fint), int(n_ant)
        if params is None:
            if kind == "phase":
                params = np.zeros((n_tint, n_fint, n_ant, 2))
            elif kind == "delay":
                params = np.zeros((n_tint, n_fint, n_ant, 4))
            else:
                params = np.zeros((n_tint, n_fint, n_ant, 4), dtype=np.complex128)
                params[..., 0] = 1.0
                params[..., 3] = 1.0
        if kind == "phase":
            self.params = np.ascontiguousarray(params, dtype=np.float64).copy()
            assert self.params.shape == (n_tint, n_fint, n_ant, 2)
        elif kind == "delay":
            self.params = np.ascontiguousarray(params, dtype=np.float64).copy()
            assert self.params.shape == (n_tint, n_fint, n_ant, 4)
        else:
            self.params = np.ascontiguousarray(params, dtype=np.complex128).copy()
            assert self.params.shape == (n_tint, n_fint, n_ant, 4)
            if kind == "diag":
                self.params[..., 1] = 0
                self.params[..., 2] = 0
        self.gain_flags = np.zeros((n_tint, n_fint, n_ant), dtype=np.int8)
        self.solve, self.max_iter, self.tol = bool(solve), int(max_iter), float(tol)

    @property
    def n_param(self) -> int:
        return 4 if self.kind in ("full", "delay") else 2

    def jones(self) -> np.ndarray:
        """The term's Jones matrices [tint][fint][ant][4] (complex128); for a delay term
        [tint][chan][ant][4], evaluated at every channel (its f_map then becomes the identity)."""
        if self.kind == "delay":
            nu = self.chan_freq[None, :, None]
            u = self.params[:, self.f_map]                          # [tint][chan][ant][4]
            out = np.zeros(u.shape[:-1] + (4,), dtype=np.complex128)
            out[..., 0] = np.exp(1j * (u[..., 0] + 2 * np.pi * u[..., 1] * nu))
            out[..., 3] = np.exp(1j * (u[..., 2] + 2 * np.pi * u[..., 3] * nu))
            return out
        if self.kind == "phase":
            out = np.zeros(self.params.shape[:-1] + (4,), dtype=np.complex128)
            out[..., 0] = np.exp(1j * self.params[..., 0])
            out[..., 3] = np.exp(1j * self.params[..., 1])
            return out
        return self.params

    def _c(self) -> _Term:
        return _Term(self.type, self.n_tint, self.n_fint, _ptr(self.t_map), _ptr(self.f_map),
                     _ptr(self.params), _ptr(self.gain_flags), int(self.solve), self.max_iter, self.tol,
                     _ptr(self.chan_freq))

    @classmethod
    def from_spec(cls, spec, n_ant: int, params=None, **kw) -> "OracleTerm":
        return cls(spec.kind, spec.t_map, spec.f_map, spec.n_tint, spec.n_fint, n_ant, params=params, **kw)


def _terms_array(terms: Sequence[OracleTerm]):
    arr = (_Term * len(terms))(*[t._c() for t in terms])
    return arr


def normal_equations(problem: OracleProblem, terms: Sequence[OracleTerm], n: int, active=None):
    """Per-(interval, antenna) JHJ and JHr blocks of term n
    (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified; Scenario 1 for phase terms,
    Scenario 2 for delay terms).

    Returns (jhj [n_tint, n_fint, n_ant, np, np], jhr [n_tint, n_fint, n_ant, np]) complex128.
    """
    lib = _load()
    T = terms[n]
    npar = T.n_param
    jhj = np.zeros((T.n_tint, T.n_fint, problem.n_ant, npar, npar), dtype=np.complex128)
    jhr = np.zeros((T.n_tint, T.n_fint, problem.n_ant, npar), dtype=np.complex128)
    act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
    arr = _terms_array(terms)
    rc = lib.oc_normal_equations(C.addressof(problem._c), C.addressof(arr), len(terms), n, _ptr(act), _ptr(jhj), _ptr(jhr))
    if rc:
        raise RuntimeError(f"oc_normal_equations failed: {rc}")
    return jhj, jhr


def solve_term(problem: OracleProblem, terms: Sequence[OracleTerm], n: int, damping: float = 1.0,
               damping_mode: int = 0, div_flag: bool = False) -> np.ndarray:
    """Algorithm 1 for term n; gains updated in place; returns iterations per interval.
    div_flag: flag (gain flag 2) and restore gains whose updates do not shrink (see oc_solve_term)."""
    lib = _load()
    T = terms[n]
    iters = np.zeros((T.n_tint, T.n_fint), dtype=np.int32)
    arr = _terms_array(terms)
    opts = _Opts(1, damping_mode, damping, int(div_flag))
    rc = lib.oc_solve_term(C.addressof(problem._c), C.addressof(arr), len(terms), n, C.addressof(opts), _ptr(iters))
    if rc:
        raise RuntimeError(f"oc_solve_term failed: {rc}")
    return iters


def solve(problem: OracleProblem, terms: Sequence[OracleTerm], n_epochs: int = 1, damping: float = 1.0,
          damping_mode: int = 0, div_flag: bool = False) -> List[np.ndarray]:
    """Chain schedule: epochs x terms x Algorithm 1.  Returns last-epoch iterations per term."""
    lib = _load()
    sizes = [t.n_tint * t.n_fint for t in terms]
    iters = np.zeros(sum(sizes), dtype=np.int32)
    arr = _terms_array(terms)
    opts = _Opts(n_epochs, damping_mode, damping, int(div_flag))
    rc = lib.oc_solve(C.addressof(problem._c), C.addressof(arr), len(terms), C.addressof(opts), _ptr(iters))
    if rc:
        raise RuntimeError(f"oc_solve failed: {rc}")
    out, off = [], 0
    for t, s in zip(terms, sizes):
        out.append(iters[off:off + s].reshape(t.n_tint, t.n_fint))
        off += s
    return out


def residual(problem: OracleProblem, terms: Sequence[OracleTerm], want_resid: bool = False):
    """chi^2 (Eq. min) and optionally the residual r = D - C_p M C_q^H [row][chan][4]."""
    lib = _load()
    res = np.zeros_like(problem.data) if want_resid else None
    chi2 = C.c_double(0.0)
    arr = _terms_array(terms)
    lib.oc_residual(C.addressof(problem._c), C.addressof(arr), len(terms), _ptr(res), C.addressof(chi2))
    return (chi2.value, res) if want_resid else chi2.value


def block_solve(A: np.ndarray, b: np.ndarray):
    """x = A^{-1} b for one small block; returns (x, singular)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    sing = lib.oc_block_solve(int(b.size), _ptr(A), _ptr(b), _ptr(x))
    return x, bool(sing)
