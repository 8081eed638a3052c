"""Pins of the oracle's delay initial estimate (peak of the Fourier transform along frequency of
the baselines with the reference antenna, Section 4.3 "Initial estimates").

- A delay on the transform's grid is recovered exactly: at the true bin every channel's term
  has the same phase, so |X| reaches the triangle-inequality bound sum |x_c| that no other
  bin reaches; the phase follows exactly.  Checked with the reference antenna first and last
  on its baselines (both orientations).
- A delay off the grid is recovered within half a grid step.
- The purpose of the estimate: delays large enough that a Gauss-Newton solve started from zero
  stops in a local minimum are solved exactly when it starts from the estimate.
"""
import numpy as np
import pytest

import oracle as O
from oracle.delay_init import delay_init, next_pow2
from paper_2412_10072_gb300 import synth


def _obs(truth, nu, seed, n_time=1, flag_frac=0.0, noise=0.0):
    """Noise-free (or noisy) data of the chain [K] with parameters truth [n_time][1][ant][4]."""
    rng = np.random.default_rng(seed)
    n_ant = truth.shape[2]
    p, q = synth.baselines(n_ant)
    ant1, ant2 = np.tile(p, n_time), np.tile(q, n_time)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    n_chan = nu.size
    shp = (ant1.size, n_chan, 4)
    model = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(2)
    weight = rng.uniform(0.5, 2.0, size=shp)
    flag = (rng.random(shp[:2]) < flag_frac).astype(np.uint8)
    w2 = 2 * np.pi * nu
    g = np.zeros((n_time, n_chan, n_ant, 2), dtype=np.complex128)
    g[..., 0] = np.exp(1j * (truth[:, 0, None, :, 0] + truth[:, 0, None, :, 1] * w2[None, :, None]))
    g[..., 1] = np.exp(1j * (truth[:, 0, None, :, 2] + truth[:, 0, None, :, 3] * w2[None, :, None]))
    gp = g[tidx[:, None], np.arange(n_chan)[None, :], ant1[:, None]]      # [row][chan][2]
    gq = g[tidx[:, None], np.arange(n_chan)[None, :], ant2[:, None]]
    data = model.copy()
    data[..., 0] *= gp[..., 0] * np.conj(gq[..., 0])
    data[..., 1] *= gp[..., 0] * np.conj(gq[..., 1])
    data[..., 2] *= gp[..., 1] * np.conj(gq[..., 0])
    data[..., 3] *= gp[..., 1] * np.conj(gq[..., 1])
    data = data + noise * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    return O.OracleProblem(data, model, weight, flag, ant1, ant2, tidx, n_ant, n_time)


def _wrap(a):
    return np.angle(np.exp(1j * a))


@pytest.mark.parametrize("ref", [0, 2, 4])
def test_on_grid_delays_are_recovered_exactly(ref):
    n_ant, n_chan, over = 5, 16, 4
    nu = 1.0 + 0.05 * np.arange(n_chan)
    N = next_pow2(over * n_chan)
    step = 1.0 / (N * 0.05)
    rng = np.random.default_rng(1)
    truth = np.zeros((1, 1, n_ant, 4))
    truth[..., 0::2] = rng.uniform(-3, 3, (1, 1, n_ant, 2))
    truth[..., 1::2] = step * rng.integers(-N // 2 + 1, N // 2, (1, 1, n_ant, 2))
    truth[:, :, ref, :] = 0.0                      # the gauge: the reference antenna's gains are 1
    P = _obs(truth, nu, seed=2)
    est = delay_init(P, np.zeros(1, np.int32), np.zeros(n_chan, np.int32), 1, 1, nu, ref=ref, oversample=over)
    np.testing.assert_allclose(est[..., 1::2], truth[..., 1::2], rtol=0, atol=1e-12)
    assert np.abs(_wrap(est[..., 0::2] - truth[..., 0::2])).max() <= 1e-9
    assert np.all(est[:, :, ref] == 0)


def test_off_grid_delays_within_half_a_step():
    n_ant, n_chan, over = 6, 40, 4
    nu = np.linspace(0.9, 1.7, n_chan)
    dnu = nu[1] - nu[0]
    N = next_pow2(over * n_chan)
    rng = np.random.default_rng(3)
    truth = np.zeros((2, 1, n_ant, 4))
    truth[..., 0::2] = rng.uniform(-3, 3, (2, 1, n_ant, 2))
    truth[..., 1::2] = rng.uniform(-10, 10, (2, 1, n_ant, 2))
    truth[:, :, 0, :] = 0.0
    P = _obs(truth, nu, seed=4, n_time=2, flag_frac=0.2)
    est = delay_init(P, np.arange(2, dtype=np.int32), np.zeros(n_chan, np.int32), 2, 1, nu, ref=0, oversample=over)
    assert np.abs(est[..., 1::2] - truth[..., 1::2]).max() <= 0.5 / (N * dnu) + 1e-12


def test_flagged_cells_do_not_enter():
    n_ant, n_chan = 4, 24
    nu = np.linspace(1.0, 1.5, n_chan)
    truth = np.zeros((1, 1, n_ant, 4))
    truth[0, 0, 1:, 1] = [0.5, -1.0, 2.0]
    P = _obs(truth, nu, seed=5, flag_frac=0.3)
    est = delay_init(P, np.zeros(1, np.int32), np.zeros(n_chan, np.int32), 1, 1, nu)
    bad = P.data.copy()
    bad[P.flag.astype(bool)] = np.nan
    P2 = O.OracleProblem(bad, P.model, P.weight, P.flag, P.ant1, P.ant2, P.time_idx, P.n_ant, P.n_time)
    est2 = delay_init(P2, np.zeros(1, np.int32), np.zeros(n_chan, np.int32), 1, 1, nu)
    np.testing.assert_array_equal(est, est2)


def test_estimate_reaches_delays_a_zero_start_cannot():
    """Delays of up to 3 ns over a 0.8 GHz band wind the phase by up to 15 rad: from zero the
    solve stops in a local minimum; from the estimate it recovers the generating parameters."""
    n_ant, n_chan = 6, 64
    nu = np.linspace(0.9, 1.7, n_chan)
    rng = np.random.default_rng(6)
    truth = np.zeros((1, 1, n_ant, 4))
    truth[..., 0::2] = rng.uniform(-2, 2, (1, 1, n_ant, 2))
    truth[..., 1::2] = rng.uniform(-3, 3, (1, 1, n_ant, 2))
    truth[:, :, 0, :] = 0.0
    P = _obs(truth, nu, seed=7)
    t_map, f_map = np.zeros(1, np.int32), np.zeros(n_chan, np.int32)
    K0 = O.OracleTerm("delay", t_map, f_map, 1, 1, n_ant, chan_freq=nu, max_iter=100, tol=1e-12)
    O.solve(P, [K0])
    chi_zero = O.residual(P, [K0])
    est = delay_init(P, t_map, f_map, 1, 1, nu)
    K1 = O.OracleTerm("delay", t_map, f_map, 1, 1, n_ant, params=est, chan_freq=nu, max_iter=100, tol=1e-12)
    O.solve(P, [K1])
    chi_est = O.residual(P, [K1])
    total = float(np.sum(P.weight * np.abs(P.data) ** 2))
    assert chi_zero > 1e-2 * total                      # a local minimum far from the data
    assert chi_est < 1e-20 * total
    got = K1.params - K1.params[:, :, :1, :]
    np.testing.assert_allclose(got[..., 1::2], truth[..., 1::2], rtol=0, atol=1e-9)
    assert np.abs(_wrap(got[..., 0::2] - truth[..., 0::2])).max() <= 1e-9
