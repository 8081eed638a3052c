"""Pins of gain flagging on divergence (Section 4.3, "Gain flagging": gains whose updates do not
tend to zero), as the oracle reads it: an interval that ends at max_iter = K >= 4 without
converging flags (gain flag 2) and restores every antenna with
max(d(K-1), d(K)) >= 0.9 max(d(1), d(2)) > 0, d(k) its relative update at iteration k.

The planted divergence is an interval left with a single usable baseline (p, q), solved with
the undamped step of Algorithm 1 (alpha = 1): the product g_p conj(g_q) is fixed by the data
but not the two gains, and the per-antenna step maps (g_p, g_q) -> (c / conj(g_q), conj(c) /
conj(g_p)), c the baseline's least-squares ratio, so the gains return to their start every two
iterations (a closed form, checked first)."""
import numpy as np

import oracle as O
from paper_2412_10072_gb300 import synth

PLANT_T = (4, 8)            # times of the planted interval (interval index 1 along time)


def _noise_free_truth_start(seed=1):
    obs = synth.plain_small(seed=seed, noise=0.0)
    spec = obs.terms[0]
    rows = np.nonzero((obs.time_idx >= PLANT_T[0]) & (obs.time_idx < PLANT_T[1]))[0]
    keep = (obs.ant1[rows] == 0) & (obs.ant2[rows] == 1)
    obs.flag[np.ix_(rows[~keep], np.arange(4))] = 1
    start = spec.truth.astype(np.complex128).copy()
    rng = np.random.default_rng(seed)
    start[1, 0, :2, 0] *= 1.3 * np.exp(0.7j * rng.standard_normal(2))     # only the planted interval is off
    start[1, 0, :2, 3] *= 0.8 * np.exp(0.5j * rng.standard_normal(2))
    return obs, spec, start


def _solve(obs, spec, start, max_iter, damping_mode, div_flag, tol=1e-9):
    P = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(spec, obs.n_ant, params=start.copy(), max_iter=max_iter, tol=tol)
    O.solve(P, [T], damping_mode=damping_mode, damping=1.0, div_flag=div_flag)
    return T


def test_single_baseline_undamped_step_has_period_two():
    obs, spec, start = _noise_free_truth_start()
    one = _solve(obs, spec, start, 1, 0, False, tol=0.0).params
    two = _solve(obs, spec, start, 2, 0, False, tol=0.0).params
    # the two antennas move away from their start, then come back exactly
    assert np.max(np.abs(one[1, 0, :2] - start[1, 0, :2])) > 0.1
    np.testing.assert_allclose(two[1, 0, :2], start[1, 0, :2], rtol=0, atol=1e-12)
    # the step's closed form: g_p <- c / conj(g_q), g_q <- conj(c) / conj(g_p) per correlation
    rows = np.nonzero((obs.time_idx >= PLANT_T[0]) & (obs.time_idx < PLANT_T[1]) & (obs.ant1 == 0) &
                      (obs.ant2 == 1))[0]
    for k in (0, 3):
        m, d = obs.model[rows, :4, k], obs.data[rows, :4, k]
        c = np.sum(np.conj(m) * d) / np.sum(np.abs(m) ** 2)
        np.testing.assert_allclose(one[1, 0, 0, k], c / np.conj(start[1, 0, 1, k]), rtol=1e-12)
        np.testing.assert_allclose(one[1, 0, 1, k], np.conj(c) / np.conj(start[1, 0, 0, k]), rtol=1e-12)


def test_planted_oscillation_is_flagged_and_restored_and_nothing_else():
    obs, spec, start = _noise_free_truth_start()
    T = _solve(obs, spec, start, 20, 0, True)
    ref = _solve(obs, spec, start, 20, 0, False)
    flags = T.gain_flags
    assert np.array_equal(flags[1, 0, :2], [2, 2])                 # the oscillating pair
    assert np.all(flags[1, 0, 2:] == 1)                             # no usable data: singular blocks
    other = np.ones(flags.shape[:2], bool)
    other[1, 0] = False
    assert np.all(flags[other] == 0)
    np.testing.assert_array_equal(T.params[1, 0, :2], start[1, 0, :2])        # restored
    np.testing.assert_array_equal(T.params[other], ref.params[other])         # untouched elsewhere


def test_damped_solve_of_the_same_interval_is_not_flagged():
    obs, spec, start = _noise_free_truth_start()
    T = _solve(obs, spec, start, 20, 1, True)
    assert not np.any(T.gain_flags == 2)


def test_converging_problem_flags_nothing():
    obs = synth.plain_small(seed=3, noise=0.01)
    P = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    O.solve(P, [T], damping_mode=1, div_flag=True)
    assert not np.any(T.gain_flags == 2)
