"""Gain flagging on divergence and robust reweighting on the GPU, against the oracle.

- Divergence (Section 4.3, "Gain flagging"): the planted oscillating interval of
  tests/test_oracle_divergence.py (one usable baseline, undamped step) gets gain flag 2 and its
  start gains back, bit for bit as the oracle's flags; nothing else is flagged, and the damped
  solve flags nothing.
- Robust reweighting (Section 4.3, after Sob et al. 2020): three epochs with planted RFI give the
  oracle's gains (1e-4 after referencing) and chi^2 (1e-5, the caller's weights), and leave the
  context's weights as they were.
"""
import numpy as np
import pytest

import oracle as O
from oracle import robust
from oracle.gauge import reference_diag, rel_err
from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu

GAIN_TOL = 1e-4
CHI2_TOL = 1e-5
PLANT_T = (4, 8)


def _planted(seed=1):
    obs = synth.plain_small(seed=seed, noise=0.0)
    spec = obs.terms[0]
    rows = np.nonzero((obs.time_idx >= PLANT_T[0]) & (obs.time_idx < PLANT_T[1]))[0]
    keep = (obs.ant1[rows] == 0) & (obs.ant2[rows] == 1)
    obs.flag[np.ix_(rows[~keep], np.arange(4))] = 1
    start = spec.truth.astype(np.complex64).copy()
    rng = np.random.default_rng(seed)
    start[1, 0, :2, 0] *= 1.3 * np.exp(0.7j * rng.standard_normal(2)).astype(np.complex64)
    start[1, 0, :2, 3] *= 0.8 * np.exp(0.5j * rng.standard_normal(2)).astype(np.complex64)
    return obs, spec, start


@pytest.mark.parametrize("kernel", [0, 2])
@pytest.mark.parametrize("damping_mode", [0, 1])
def test_planted_divergence_flags_match_oracle(kernel, damping_mode):
    obs, spec, start = _planted()
    tol = 1e-5                         # truth-started intervals converge at once in FP32 and FP64
    P = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(spec, obs.n_ant, params=start.astype(np.complex128), max_iter=20, tol=tol)
    O.solve(P, [T], damping_mode=damping_mode, damping=1.0, div_flag=True)
    S = qc.Solver.from_obs(obs)
    g = qc.Term.from_spec(spec, obs.n_ant, gains=start, max_iter=20, tol=tol)
    S.solve([g], damping_mode=damping_mode, damping=1.0, div_flag=True, kernel=kernel)
    S.close()
    diff = np.argwhere(g.gain_flags != T.gain_flags)
    assert diff.size == 0, [(tuple(i), int(g.gain_flags[tuple(i)]), int(T.gain_flags[tuple(i)])) for i in diff[:8]]
    if damping_mode == 0:
        assert np.array_equal(g.gain_flags[1, 0, :2], [2, 2])
        assert np.array_equal(np.asarray(g.gains)[1, 0, :2], start[1, 0, :2])     # restored exactly
    else:
        assert not np.any(g.gain_flags == 2)
    other = np.ones(g.gain_flags.shape[:2], bool)
    other[1, 0] = False
    err = rel_err(reference_diag(np.asarray(g.gains, np.complex128)[other][None]),
                  reference_diag(T.params[other][None]))
    assert err < GAIN_TOL, err


def _rfi_obs(seed=7):
    obs = synth.plain_small(seed=seed, noise=0.01)
    rng = np.random.default_rng(3)
    bad = rng.random(obs.flag.shape) < 0.01
    obs.data[bad] += 5.0 * (rng.standard_normal((bad.sum(), 4)) + 1j * rng.standard_normal((bad.sum(), 4)))
    return obs


@pytest.mark.parametrize("kernel", [0, 2, 4])
def test_robust_reweighting_matches_oracle(kernel):
    obs = _rfi_obs()
    nu = 3.0
    P = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    robust.solve_robust(P, [T], 3, nu)
    ochi2 = O.residual(P, [T])
    S = qc.Solver.from_obs(obs)
    g = qc.Term.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    st = S.solve([g], n_epochs=3, robust_nu=nu, want_chi2=True, kernel=kernel)
    err = rel_err(reference_diag(np.asarray(g.gains, np.complex128)), reference_diag(T.params))
    assert err < GAIN_TOL, err
    assert abs(st.chi2_after - ochi2) <= CHI2_TOL * ochi2, (st.chi2_after, ochi2)
    # the reweighting helped against the planted RFI, as it does in the oracle
    truth = reference_diag(obs.terms[0].truth.astype(np.complex128))
    plain = qc.Term.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    S.solve([plain], n_epochs=3, kernel=kernel)
    assert rel_err(reference_diag(np.asarray(g.gains, np.complex128)), truth) < \
        0.5 * rel_err(reference_diag(np.asarray(plain.gains, np.complex128)), truth)
    # the context's weights are the caller's again: the plain solve equals one on a fresh context
    S2 = qc.Solver.from_obs(obs)
    fresh = qc.Term.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    S2.solve([fresh], n_epochs=3, kernel=kernel)
    S2.close()
    S.close()
    assert np.array_equal(np.asarray(plain.gains), np.asarray(fresh.gains))


def test_robust_reweighting_in_a_two_term_chain():
    obs = synth.plain_large(seed=3, n_ant=10, n_time=12, n_chan=40, noise=0.05, flag_row_frac=0.1, n_src=8)
    rng = np.random.default_rng(9)
    bad = rng.random(obs.flag.shape) < 0.01
    obs.data[bad] += 3.0 * (rng.standard_normal((bad.sum(), 4)) + 1j * rng.standard_normal((bad.sum(), 4)))
    P = O.OracleProblem.from_obs(obs)
    ot = [O.OracleTerm.from_spec(s, obs.n_ant, max_iter=20, tol=1e-6) for s in obs.terms]
    robust.solve_robust(P, ot, 3, 4.0)
    ochi2 = O.residual(P, ot)
    S = qc.Solver.from_obs(obs)
    gt = [qc.Term.from_spec(s, obs.n_ant, max_iter=20, tol=1e-6) for s in obs.terms]
    st = S.solve(gt, n_epochs=3, robust_nu=4.0, want_chi2=True)
    S.close()
    from oracle.gauge import chain_products, reference_chain
    Cg = reference_chain(chain_products([np.asarray(t.gains, np.complex128) for t in gt], [t.t_map for t in gt],
                                        [t.f_map for t in gt], obs.n_time, obs.n_chan))
    Co = reference_chain(chain_products([t.jones() for t in ot], [t.t_map for t in ot], [t.f_map for t in ot],
                                        obs.n_time, obs.n_chan))
    assert rel_err(Cg, Co) < GAIN_TOL
    assert abs(st.chi2_after - ochi2) <= CHI2_TOL * ochi2
