"""The allocation-free chi^2 entry point against the context-based one.

qc_residual_noalloc exists for callers that must not allocate device memory
(real-time pipelines with a fixed device-memory plan, host frameworks that own
every buffer); it keeps its scratch in a static device array.  This file is
collected last so that a failure here does not hide the other tests, and it
passes on its own in a fresh process as well as after them.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CHI2_TOL = 1e-5          # the relative chi^2 tolerance of the parity tests


def _lib():
    lib = qc.load()
    vp, i32 = C.c_void_p, C.c_int32
    lib.qc_residual_noalloc.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, vp, vp]
    lib.qc_residual_noalloc.restype = C.c_int
    return lib


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _noalloc_chi2(lib, obs, term, gains, ant1=None, time_idx=None):
    d = dict(data=_dev(obs.data, np.complex64), model=_dev(obs.model, np.complex64),
             weight=_dev(obs.weight, np.float32), flag=_dev(obs.flag, np.uint8),
             a1=_dev(obs.ant1 if ant1 is None else ant1, np.int32), a2=_dev(obs.ant2, np.int32),
             t=_dev(obs.time_idx if time_idx is None else time_idx, np.int32), tm=_dev(term.t_map, np.int32),
             fm=_dev(term.f_map, np.int32),
             g=_dev(gains, np.float32 if term.kind == "phase" else np.complex64))
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    rc = lib.qc_residual_noalloc(obs.n_row, obs.n_chan, obs.n_ant, obs.n_time, d["data"].data_ptr(),
                                 d["model"].data_ptr(),
                                 d["weight"].data_ptr(), d["flag"].data_ptr(), d["a1"].data_ptr(), d["a2"].data_ptr(),
                                 d["t"].data_ptr(), qc.KINDS[term.kind], term.n_tint, term.n_fint,
                                 d["tm"].data_ptr(), d["fm"].data_ptr(), d["g"].data_ptr(), out.data_ptr(), None)
    assert rc == qc.QC_OK, lib.qc_last_error(None)
    torch.cuda.synchronize()
    return float(out.item())


def _ctx_chi2(obs, term, gains):
    S = qc.Solver.from_obs(obs)
    t = qc.Term.from_spec(term, obs.n_ant, gains=gains, solve=False)
    chi2 = S.residual([t])
    S.close()
    return chi2


def test_noalloc_chi2_matches_qc_residual_twice_in_a_row():
    lib = _lib()
    obs = synth.plain_small(seed=2, noise=0.01)
    obs.flag[::7, 3] = 1
    spec = obs.terms[0]
    rng = np.random.default_rng(0)
    g1 = spec.truth.astype(np.complex64)
    g2 = (spec.truth * (1 + 0.1 * rng.standard_normal(spec.truth.shape))).astype(np.complex64)
    g2[..., 1:3] = 0
    for g in (g1, g2):                                   # two calls in a row reuse the same scratch
        want = _ctx_chi2(obs, spec, g)
        got = _noalloc_chi2(lib, obs, spec, g)
        assert abs(got - want) <= CHI2_TOL * want, (got, want)


def test_noalloc_full_jones_and_phase_terms():
    lib = _lib()
    rng = np.random.default_rng(3)
    n_ant, n_time, n_chan = 6, 4, 40
    freqs = synth.meerkat_band(n_chan)
    for kind in ("full", "phase"):
        spec = synth.TermSpec(kind, synth.interval_map(n_time, 2), synth.interval_map(n_chan, 8), 2, 5)
        spec.truth = (0.5 * rng.standard_normal((2, 5, n_ant, 2)) if kind == "phase"
                      else synth.full_truth(n_ant, 2, 5, rng))
        obs = synth.make_observation(n_ant, n_time, freqs, [spec], n_src=4, seed=3, noise=0.05, rng=rng)
        g = (spec.truth if kind == "phase" else spec.truth).astype(np.float32 if kind == "phase" else np.complex64)
        want = _ctx_chi2(obs, spec, g)
        got = _noalloc_chi2(lib, obs, spec, g)
        assert abs(got - want) <= CHI2_TOL * want, (kind, got, want)


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = _lib()
    big = np.zeros(16, np.int32)
    rc = lib.qc_residual_noalloc(4, 4, 64, 4, big.ctypes.data, big.ctypes.data, big.ctypes.data, None, big.ctypes.data,
                                 big.ctypes.data, big.ctypes.data, qc.QC_TERM_DIAG, 1024, 1024, big.ctypes.data,
                                 big.ctypes.data, big.ctypes.data, big.ctypes.data, None)
    assert rc == qc.QC_EINVAL
    assert b"QC_NOALLOC_MAX_GAINS" in lib.qc_last_error(None)


def test_noalloc_index_out_of_range_gives_nan_then_recovers():
    """Indices in device memory are checked by the kernel before use: an antenna index equal
    to n_ant, or a time index past n_time, is never used to read anything; the result is NaN.
    The next call with valid indices clears the check and gives the right chi^2 again."""
    lib = _lib()
    obs = synth.plain_small(seed=4, noise=0.01)
    spec = obs.terms[0]
    g = spec.truth.astype(np.complex64)
    bad_ant = np.array(obs.ant1, np.int32)
    bad_ant[5] = obs.n_ant
    assert np.isnan(_noalloc_chi2(lib, obs, spec, g, ant1=bad_ant))
    bad_t = np.array(obs.time_idx, np.int32)
    bad_t[-1] = obs.n_time
    assert np.isnan(_noalloc_chi2(lib, obs, spec, g, time_idx=bad_t))
    want = _ctx_chi2(obs, spec, g)
    got = _noalloc_chi2(lib, obs, spec, g)
    assert abs(got - want) <= CHI2_TOL * want, (got, want)
