"""Python binding of libqc (ctypes): argument marshalling only.

Every step of the solve runs in the CUDA kernels behind the C ABI declared
in ``include/qc.h``; this module only builds the C structs from numpy
arrays (host memory) or CUDA tensors (device memory, anything exposing
``data_ptr()`` and ``is_cuda``).  There is no CPU fallback: if the library
cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

QC_OK, QC_EINVAL, QC_ENOMEM, QC_ECUDA, QC_ETIMEOUT, QC_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
QC_TERM_DIAG, QC_TERM_FULL, QC_TERM_PHASE, QC_TERM_DELAY = 0, 1, 2, 3
QC_MEM_HOST, QC_MEM_DEVICE = 0, 1
QC_DAMP_CONST, QC_DAMP_ALTERNATE = 0, 1
KINDS = {"diag": QC_TERM_DIAG, "full": QC_TERM_FULL, "phase": QC_TERM_PHASE, "delay": QC_TERM_DELAY}

_lib = None
_lock = threading.Lock()


class QCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libqc error {code}: {msg}")
        self.code = code


class _Problem(C.Structure):
    _fields_ = [("n_row", C.c_int32), ("n_chan", C.c_int32), ("n_corr", C.c_int32), ("n_ant", C.c_int32),
                ("n_dir", C.c_int32), ("n_time", C.c_int32), ("data", C.c_void_p), ("model", C.c_void_p),
                ("weight", C.c_void_p), ("flag", C.c_void_p), ("ant1", C.c_void_p), ("ant2", C.c_void_p),
                ("time_idx", C.c_void_p), ("memory", C.c_int32), ("model_fp16", C.c_int32)]


class _Term(C.Structure):
    _fields_ = [("type", C.c_int32), ("n_tint", C.c_int32), ("n_fint", C.c_int32), ("t_map", C.c_void_p),
                ("f_map", C.c_void_p), ("gains", C.c_void_p), ("gain_flags", C.c_void_p), ("iters", C.c_void_p),
                ("solve", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double), ("memory", C.c_int32),
                ("reduce", C.c_int32), ("chan_freq", C.c_void_p), ("dd", C.c_int32)]


ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p)


class _Opts(C.Structure):
    _fields_ = [("n_epochs", C.c_int32), ("damping_mode", C.c_int32), ("damping", C.c_double),
                ("stream", C.c_void_p), ("use_graph", C.c_int32), ("want_chi2", C.c_int32), ("order", C.c_int32),
                ("block_threads", C.c_int32), ("ctas_per_sm", C.c_int32), ("kernel", C.c_int32),
                ("allreduce", ALLREDUCE_FN),
                ("allreduce_user", C.c_void_p), ("div_flag", C.c_int32), ("robust", C.c_int32),
                ("robust_nu", C.c_double), ("moments", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("chi2_before", C.c_double), ("chi2_after", C.c_double), ("ms", C.c_double), ("acc_ms", C.c_double),
                ("vis_iters", C.c_int64), ("acc_bytes", C.c_int64), ("acc_launches", C.c_int64),
                ("launches", C.c_int64), ("n_iter_max", C.c_int32), ("pass_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqc.so (building it first when sources are newer); raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libqc.so not found at {_build.LIB}; run paper_2412_10072_gb300.build.build()")
        lib = C.CDLL(_build.LIB)
        vp, i32 = C.c_void_p, C.c_int32
        lib.qc_create.argtypes = [C.POINTER(_Problem), C.POINTER(vp)]
        lib.qc_create.restype = C.c_int
        lib.qc_solve.argtypes = [vp, C.POINTER(_Term), i32, C.POINTER(_Opts), C.POINTER(Stats)]
        lib.qc_solve.restype = C.c_int
        lib.qc_residual.argtypes = [vp, C.POINTER(_Term), i32, vp, i32, C.POINTER(C.c_double)]
        lib.qc_residual.restype = C.c_int
        lib.qc_delay_init.argtypes = [vp, C.POINTER(_Term), i32, i32]
        lib.qc_delay_init.restype = C.c_int
        lib.qc_mad_flag.argtypes = [vp, C.POINTER(_Term), i32, C.c_double, i32, vp, i32, C.POINTER(C.c_int64)]
        lib.qc_mad_flag.restype = C.c_int
        lib.qc_destroy.argtypes = [vp]
        lib.qc_destroy.restype = None
        lib.qc_last_error.argtypes = [vp]
        lib.qc_last_error.restype = C.c_char_p
        lib.qc_version.argtypes = []
        lib.qc_version.restype = C.c_char_p
        lib.qc_test_fail_alloc.argtypes = [C.c_int64]
        lib.qc_test_fail_alloc.restype = None
        lib.qc_test_live_allocs.argtypes = []
        lib.qc_test_live_allocs.restype = C.c_int64
        lib.qc_test_wait_limit.argtypes = [C.c_int64, i32]
        lib.qc_test_wait_limit.restype = None
        _lib = lib
        return lib


def _is_dev(a) -> bool:
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _addr(a) -> Optional[int]:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    return int(a.ctypes.data)


def _is_host_tensor(a) -> bool:
    return hasattr(a, "data_ptr") and not getattr(a, "is_cuda", False)


def _host(a, dtype):
    if _is_host_tensor(a):           # e.g. a pinned CPU tensor: passed without a copy
        if not a.is_contiguous() or a.element_size() != np.dtype(dtype).itemsize:
            raise ValueError("host tensors must be contiguous and of the documented dtype")
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def _complex64(a):
    """Host complex data as interleaved complex64 (upcast/downcast allowed)."""
    if _is_dev(a):
        return a
    return _host(a, np.complex64)


class Term:
    """One Jones term (see qc_term in include/qc.h).

    gains: numpy complex [n_tint][n_fint][n_ant][4] (diag/full), float [..][2] (phase) or float
    [..][4] = (phi_X, tau_X, phi_Y, tau_Y) (delay, with ``chan_freq`` [n_chan], the frequency of
    every channel), or a CUDA tensor of the same layout (complex64 / float32).  After a solve the
    solved values are in ``self.gains`` (host arrays are updated in place).
    A direction-dependent term (``dd`` with ``n_dir`` > 1) has gains [n_tint][n_fint][n_ant][n_dir][4]
    and gain flags [n_tint][n_fint][n_ant][n_dir].
    """

    def __init__(self, kind: str, t_map, f_map, n_tint: int, n_fint: int, n_ant: int, gains=None,
                 solve: bool = True, max_iter: int = 20, tol: float = 1e-6, reduce: bool = False,
                 chan_freq=None, dd: bool = False, n_dir: int = 1):
        self.kind = kind
        self.type = KINDS[kind]
        self.dd = bool(dd)
        nd = int(n_dir) if (dd and n_dir > 1) else 1
        ax = (n_ant, nd) if nd > 1 else (n_ant,)
        self.chan_freq = None
        if kind == "delay":
            if chan_freq is None:
                raise ValueError("a delay term needs chan_freq")
            self.chan_freq = np.ascontiguousarray(chan_freq, dtype=np.float64)
        self.t_map = _host(t_map, np.int32)
        self.f_map = _host(f_map, np.int32)
        self.n_tint, self.n_fint, self.n_ant = int(n_tint), int(n_fint), int(n_ant)
        if gains is None:
            if kind == "phase":
                gains = np.zeros((n_tint, n_fint, n_ant, 2), dtype=np.float32)
            elif kind == "delay":
                gains = np.zeros((n_tint, n_fint, n_ant, 4), dtype=np.float32)
            else:
                gains = np.zeros((n_tint, n_fint) + ax + (4,), dtype=np.complex64)
                gains[..., 0] = 1
                gains[..., 3] = 1
        if _is_dev(gains):
            self.gains = gains
            self.memory = QC_MEM_DEVICE
            dev = gains.device
            import torch
            self.gain_flags = torch.zeros((n_tint, n_fint) + ax, dtype=torch.int8, device=dev)
            self.iters = torch.zeros((n_tint, n_fint), dtype=torch.int32, device=dev)
        else:
            dt = np.float32 if kind in ("phase", "delay") else np.complex64
            self.gains = np.array(gains, dtype=dt, copy=True, order="C")
            self.memory = QC_MEM_HOST
            self.gain_flags = np.zeros((n_tint, n_fint) + ax, dtype=np.int8)
            self.iters = np.zeros((n_tint, n_fint), dtype=np.int32)
        self.solve, self.max_iter, self.tol, self.reduce = bool(solve), int(max_iter), float(tol), bool(reduce)

    @classmethod
    def from_spec(cls, spec, n_ant: int, gains=None, **kw) -> "Term":
        return cls(spec.kind, spec.t_map, spec.f_map, spec.n_tint, spec.n_fint, n_ant, gains=gains, **kw)

    def _c(self) -> _Term:
        return _Term(self.type, self.n_tint, self.n_fint, _addr(self.t_map), _addr(self.f_map), _addr(self.gains),
                     _addr(self.gain_flags), _addr(self.iters), int(self.solve), self.max_iter, self.tol,
                     self.memory, int(self.reduce), _addr(self.chan_freq), int(self.dd))


def _terms_array(terms: Sequence[Term]):
    return (_Term * len(terms))(*[t._c() for t in terms])


class Solver:
    """A staged calibration problem (qc_create / qc_solve / qc_residual / qc_destroy).

    The model is [n_row][n_chan][4], or [n_row][n_chan][n_dir][4] for a model with directions.
    """

    def __init__(self, data, model, weight, flag, ant1, ant2, time_idx, n_ant: int, n_time: int,
                 model_fp16: bool = False):
        self._lib = load()
        dev = _is_dev(data)
        if dev:
            for a in (model, weight) + ((flag,) if flag is not None else ()):
                if not _is_dev(a):
                    raise ValueError("data, model, weight and flag must all be host arrays or all CUDA tensors")
            self._keep = (data, model, weight, flag)
            n_row, n_chan = int(data.shape[0]), int(data.shape[1])
            memory = QC_MEM_DEVICE
        else:
            data = _complex64(data)
            model = _complex64(model)
            weight = _host(weight, np.float32)
            flag = None if flag is None else _host(flag, np.uint8)
            self._keep = (data, model, weight, flag)
            n_row, n_chan = data.shape[0], data.shape[1]
            memory = QC_MEM_HOST
        a1, a2, ti = _host(ant1, np.int32), _host(ant2, np.int32), _host(time_idx, np.int32)
        self._meta = (a1, a2, ti)
        self.n_row, self.n_chan, self.n_ant, self.n_time = n_row, n_chan, int(n_ant), int(n_time)
        self.n_dir = int(model.shape[2]) if len(model.shape) == 4 else 1
        p = _Problem(n_row, n_chan, 4, self.n_ant, self.n_dir, self.n_time, _addr(data), _addr(model), _addr(weight),
                     _addr(flag), _addr(a1), _addr(a2), _addr(ti), memory, int(bool(model_fp16)))
        h = C.c_void_p()
        rc = self._lib.qc_create(C.byref(p), C.byref(h))
        if rc != QC_OK:
            raise QCError(rc, self._lib.qc_last_error(None).decode())
        self._h = h
        if memory == QC_MEM_HOST:
            self._keep = None          # copied to the device at create

    @classmethod
    def from_obs(cls, obs, **kw) -> "Solver":
        return cls(obs.data, obs.model, obs.weight, obs.flag, obs.ant1, obs.ant2, obs.time_idx, obs.n_ant,
                   obs.n_time, **kw)

    def _err(self, rc):
        raise QCError(rc, self._lib.qc_last_error(self._h).decode())

    def solve(self, terms: List[Term], n_epochs: int = 1, damping_mode: int = QC_DAMP_ALTERNATE,
              damping: float = 1.0, use_graph: bool = True, want_chi2: bool = False, order: int = -1,
              block_threads: int = 0, ctas_per_sm: int = 0, stream=None, allreduce=None,
              kernel: int = 0, div_flag: bool = False, robust_nu: Optional[float] = None,
              moments: bool = False) -> Stats:
        """robust_nu: robust reweighting between epochs with nu degrees of freedom (None: off);
        div_flag: flag (gain flag 2) and restore diverging gains; moments: solve each term of a
        chain of one or two terms from per-(interval, antenna pair) sums (include/qc.h)."""
        arr = _terms_array(terms)
        cb = ALLREDUCE_FN(allreduce) if allreduce is not None else ALLREDUCE_FN()
        st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        o = _Opts(n_epochs, damping_mode, damping, st or None, int(use_graph), int(want_chi2), order,
                  block_threads, ctas_per_sm, kernel, cb, None, int(bool(div_flag)), int(robust_nu is not None),
                  float(robust_nu or 0.0), int(bool(moments)))
        s = Stats()
        rc = self._lib.qc_solve(self._h, arr, len(terms), C.byref(o), C.byref(s))
        if rc != QC_OK:
            self._err(rc)
        return s

    def delay_init(self, term: Term, ref: int = 0, oversample: int = 4) -> Term:
        """Overwrite a delay term's parameters with the initial estimate of qc_delay_init (the
        peak of the Fourier transform along frequency of the baselines with antenna ``ref``)."""
        arr = _terms_array([term])
        rc = self._lib.qc_delay_init(self._h, arr, int(ref), int(oversample))
        if rc != QC_OK:
            self._err(rc)
        return term

    def mad_flag(self, terms: List[Term], threshold: float = 5.0, out=None, per_baseline: bool = False):
        """Outlier flags of the residual after calibration (qc_mad_flag): uint8 [n_row][n_chan]
        (a new host array, or ``out``, a CUDA tensor) and the number of samples flagged; median and
        MAD over all baselines, or over each baseline with ``per_baseline``."""
        arr = _terms_array(terms)
        n = C.c_int64(0)
        if out is None:
            out = np.zeros((self.n_row, self.n_chan), dtype=np.uint8)
        mem = QC_MEM_DEVICE if _is_dev(out) else QC_MEM_HOST
        rc = self._lib.qc_mad_flag(self._h, arr, len(terms), float(threshold), int(bool(per_baseline)), _addr(out),
                                   mem, C.byref(n))
        if rc != QC_OK:
            self._err(rc)
        return out, int(n.value)

    def residual(self, terms: List[Term], want_resid: bool = False, resid_out=None):
        arr = _terms_array(terms)
        chi2 = C.c_double(0.0)
        res, mem = None, QC_MEM_HOST
        if resid_out is not None:
            res, mem = resid_out, (QC_MEM_DEVICE if _is_dev(resid_out) else QC_MEM_HOST)
        elif want_resid:
            res = np.zeros((self.n_row, self.n_chan, 4), dtype=np.complex64)
        rc = self._lib.qc_residual(self._h, arr, len(terms), _addr(res), mem, C.byref(chi2))
        if rc != QC_OK:
            self._err(rc)
        return (chi2.value, res) if (want_resid or resid_out is not None) else chi2.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.qc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return load().qc_version().decode()


# ---------------------------------------------------------------------------
# batched solves of independent solution intervals
# ---------------------------------------------------------------------------

QC_SCHED_AUTO, QC_SCHED_LPT, QC_SCHED_STATIC = 0, 1, 2
QC_BATCH_MAX_ANT = 256


class _BatchProblem(C.Structure):
    _fields_ = [("n_prob", C.c_int32), ("row_offset", C.c_void_p), ("vis_offset", C.c_void_p),
                ("n_chan", C.c_void_p), ("n_ant", C.c_void_p), ("data", C.c_void_p), ("model", C.c_void_p),
                ("weight", C.c_void_p), ("flag", C.c_void_p), ("ant1", C.c_void_p), ("ant2", C.c_void_p),
                ("memory", C.c_int32), ("model_fp16", C.c_int32)]


class _BatchOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("tol", C.c_double), ("damping_mode", C.c_int32), ("damping", C.c_double),
                ("stream", C.c_void_p), ("threads", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("schedule", C.c_int32), ("use_graph", C.c_int32), ("depth", C.c_int32),
                ("fallback_gains", C.c_void_p), ("fallback_chi2", C.c_void_p), ("split", C.c_int64),
                ("small_threads", C.c_int32), ("small_ctas_per_sm", C.c_int32)]


class BatchStats(C.Structure):
    _fields_ = [("ms", C.c_double), ("vis_iters", C.c_int64), ("bytes", C.c_int64), ("n_iter_max", C.c_int32),
                ("mean_iters", C.c_double), ("threads", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("schedule", C.c_int32), ("grid", C.c_int32), ("depth", C.c_int32), ("n_fallback", C.c_int32),
                ("split", C.c_int64), ("small_threads", C.c_int32), ("small_ctas_per_sm", C.c_int32),
                ("small_grid", C.c_int32), ("n_small", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load_batch(lib):
    if getattr(lib, "_batch_ready", False):
        return lib
    vp, i32 = C.c_void_p, C.c_int32
    lib.qc_batch_create.argtypes = [C.POINTER(_BatchProblem), C.POINTER(vp)]
    lib.qc_batch_create.restype = C.c_int
    lib.qc_batch_solve.argtypes = [vp, vp, vp, vp, i32, C.POINTER(_BatchOpts), C.POINTER(BatchStats)]
    lib.qc_batch_solve_moments.argtypes = [vp, vp, vp, vp, i32, C.POINTER(_BatchOpts), C.POINTER(BatchStats)]
    lib.qc_batch_solve_moments.restype = C.c_int
    lib.qc_batch_solve.restype = C.c_int
    lib.qc_batch_autotune.argtypes = [vp, C.POINTER(_BatchOpts), C.POINTER(BatchStats), C.POINTER(C.c_int32)]
    lib.qc_batch_autotune.restype = C.c_int
    lib.qc_batch_residual.argtypes = [vp, vp, i32, vp]
    lib.qc_batch_residual.restype = C.c_int
    lib.qc_batch_destroy.argtypes = [vp]
    lib.qc_batch_destroy.restype = None
    lib.qc_batch_last_error.argtypes = [vp]
    lib.qc_batch_last_error.restype = C.c_char_p
    lib._batch_ready = True
    return lib


class BatchSolver:
    """Many independent one-interval diagonal-gain problems (qc_batch_* of include/qc.h).

    Arrays are the problems' [row][chan][4] blocks concatenated; ``row_offset`` and
    ``vis_offset`` (length n_prob + 1), ``n_chan``, ``n_ant`` and ``ant1``/``ant2`` are host
    arrays.  Gains are [sum n_ant][2] complex64 (g_XX, g_YY).
    """

    def __init__(self, data, model, weight, flag, ant1, ant2, row_offset, vis_offset, n_chan, n_ant,
                 model_fp16: bool = False):
        self._lib = _load_batch(load())
        dev = _is_dev(data)
        if not dev:
            data = _complex64(data)
            model = _complex64(model)
            weight = _host(weight, np.float32)
            flag = None if flag is None else _host(flag, np.uint8)
        self._keep = (data, model, weight, flag) if dev else None
        self.row_offset = _host(row_offset, np.int64)
        self.vis_offset = _host(vis_offset, np.int64)
        self.n_chan = _host(n_chan, np.int32)
        self.n_ant = _host(n_ant, np.int32)
        self.ant1 = _host(ant1, np.int32)
        self.ant2 = _host(ant2, np.int32)
        self.n_prob = int(self.n_chan.size)
        self.gain_offset = np.concatenate([[0], np.cumsum(self.n_ant)]).astype(np.int64)
        p = _BatchProblem(self.n_prob, _addr(self.row_offset), _addr(self.vis_offset), _addr(self.n_chan),
                          _addr(self.n_ant), _addr(data), _addr(model), _addr(weight), _addr(flag), _addr(self.ant1),
                          _addr(self.ant2), QC_MEM_DEVICE if dev else QC_MEM_HOST, int(bool(model_fp16)))
        h = C.c_void_p()
        rc = self._lib.qc_batch_create(C.byref(p), C.byref(h))
        if rc != QC_OK:
            raise QCError(rc, self._lib.qc_batch_last_error(None).decode())
        self._h = h

    @property
    def total_ant(self) -> int:
        return int(self.gain_offset[-1])

    def unit_gains(self):
        g = np.zeros((self.total_ant, 2), dtype=np.complex64)
        g[:] = 1
        return g

    def _opts(self, max_iter, tol, damping_mode, damping, stream, threads, ctas_per_sm, schedule, use_graph,
              depth=0, fallback=None, split=0, small_threads=0, small_ctas_per_sm=0):
        st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        fb_g, fb_c = (None, None) if fallback is None else (fallback[0].data_ptr(), fallback[1].data_ptr())
        return _BatchOpts(max_iter, tol, damping_mode, damping, st or None, threads, ctas_per_sm, schedule,
                          int(use_graph), depth, fb_g, fb_c, int(split), int(small_threads), int(small_ctas_per_sm))

    def _err(self, rc):
        raise QCError(rc, self._lib.qc_batch_last_error(self._h).decode())

    def solve(self, gains=None, max_iter: int = 20, tol: float = 1e-6, damping_mode: int = QC_DAMP_ALTERNATE,
              damping: float = 1.0, stream=None, threads: int = 0, ctas_per_sm: int = 0,
              schedule: int = QC_SCHED_AUTO, use_graph: bool = True, want_flags: bool = True, depth: int = 0,
              fallback=None, moments: bool = False, split: int = 0, small_threads: int = 0,
              small_ctas_per_sm: int = 0):
        """Solve in place; returns (gains, gain_flags, iters, BatchStats).  fallback: optional
        (device gains [sum n_ant][2] complex64, device chi^2 [n_prob] float64) -- a problem whose
        starting gains fit worse than its fallback chi^2 restarts from the fallback gains.
        moments: one pass forms per-baseline sums and the iterations use them
        (qc_batch_solve_moments; at most 64 antennas; with a fallback, chi^2 at both starts comes
        from the sums and the fallback chi^2 array is not read)."""
        if gains is None:
            gains = self.unit_gains()
        dev = _is_dev(gains)
        if dev:
            import torch
            flags = torch.zeros(self.total_ant, dtype=torch.int8, device=gains.device) if want_flags else None
            iters = torch.zeros(self.n_prob, dtype=torch.int32, device=gains.device)
        else:
            gains = np.ascontiguousarray(gains, dtype=np.complex64)
            flags = np.zeros(self.total_ant, dtype=np.int8) if want_flags else None
            iters = np.zeros(self.n_prob, dtype=np.int32)
        o = self._opts(max_iter, tol, damping_mode, damping, stream, threads, ctas_per_sm, schedule, use_graph, depth,
                       fallback, split, small_threads, small_ctas_per_sm)
        s = BatchStats()
        fn = self._lib.qc_batch_solve_moments if moments else self._lib.qc_batch_solve
        rc = fn(self._h, _addr(gains), _addr(flags), _addr(iters), QC_MEM_DEVICE if dev else QC_MEM_HOST, C.byref(o),
                C.byref(s))
        if rc != QC_OK:
            self._err(rc)
        return gains, flags, iters, s

    def autotune(self, max_iter: int = 20, tol: float = 1e-6, damping_mode: int = QC_DAMP_ALTERNATE, stream=None):
        o = self._opts(max_iter, tol, damping_mode, 1.0, stream, 0, 0, QC_SCHED_AUTO, False)
        s = BatchStats()
        n = C.c_int32(0)
        rc = self._lib.qc_batch_autotune(self._h, C.byref(o), C.byref(s), C.byref(n))
        if rc != QC_OK:
            self._err(rc)
        return s, n.value

    def residual(self, gains):
        dev = _is_dev(gains)
        if dev:
            import torch
            chi2 = torch.zeros(self.n_prob, dtype=torch.float64, device=gains.device)
        else:
            gains = np.ascontiguousarray(gains, dtype=np.complex64)
            chi2 = np.zeros(self.n_prob, dtype=np.float64)
        rc = self._lib.qc_batch_residual(self._h, _addr(gains), QC_MEM_DEVICE if dev else QC_MEM_HOST, _addr(chi2))
        if rc != QC_OK:
            self._err(rc)
        return chi2

    def close(self):
        if getattr(self, "_h", None):
            self._lib.qc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
