"""Pins of the oracle's MAD residual flagger (Section 4, "Additional features").

- Order statistics against a sort written out here on tiny inputs.
- Gaussian residuals with planted outliers far outside the Gaussian tail: exactly the
  planted samples are flagged.
- The MAD of Gaussian whitened residuals scaled by 1.4826 estimates their spread.
- Flagged samples and autocorrelations neither enter the statistics nor get flagged.
"""
import numpy as np

from oracle.mad_flag import mad_flag, order_statistic, whitened_norm


def test_order_statistic_is_the_lower_middle_element():
    for vals in ([3.0], [2.0, 1.0], [5.0, 1.0, 4.0, 2.0], [7.0, 7.0, 1.0, 9.0, 3.0]):
        s = sorted(vals)
        assert order_statistic(np.array(vals, np.float32)) == np.float32(s[(len(s) - 1) // 2])


def _residuals(seed, n_row=400, n_chan=16, sigma=1.0):
    rng = np.random.default_rng(seed)
    r = (sigma * (rng.standard_normal((n_row, n_chan, 4)) + 1j * rng.standard_normal((n_row, n_chan, 4)))
         ).astype(np.complex64)
    w = np.ones((n_row, n_chan, 4), np.float32)
    ant1 = np.zeros(n_row, np.int32)
    ant2 = np.ones(n_row, np.int32)
    return rng, r, w, ant1, ant2


def test_planted_outliers_are_exactly_the_flagged_samples():
    rng, r, w, a1, a2 = _residuals(1)
    idx = rng.choice(r.shape[0] * r.shape[1], size=25, replace=False)
    rows, chans = np.unravel_index(idx, r.shape[:2])
    r[rows, chans, 0] += np.complex64(60.0)            # ~40 sigma of the whitened norm's spread
    out, (med, mad, n) = mad_flag(r, w, None, a1, a2, threshold=10.0)
    want = np.zeros(r.shape[:2], np.uint8)
    want[rows, chans] = 1
    np.testing.assert_array_equal(out, want)
    assert n == 25


def test_mad_estimates_the_spread_of_gaussian_norms():
    _, r, w, a1, a2 = _residuals(2, n_row=2000)
    z = whitened_norm(r, w).astype(np.float64).ravel()
    _, (med, mad, _) = mad_flag(r, w, None, a1, a2)
    assert abs(med - np.median(z)) <= 1e-3 * np.median(z)
    assert abs(1.4826 * mad - np.std(z)) <= 0.05 * np.std(z)


def test_flagged_samples_and_autocorrelations_are_left_out():
    rng, r, w, a1, a2 = _residuals(3)
    flag = (rng.random(r.shape[:2]) < 0.2).astype(np.uint8)
    r_big = r.copy()
    r_big[flag.astype(bool)] = np.complex64(1e6)       # would be outliers and would move the median
    a2 = a2.copy()
    a2[:10] = 0                                         # autocorrelation rows
    r_big[:10] = np.complex64(1e6)
    out1, s1 = mad_flag(r, w, flag, a1, a2)
    out2, s2 = mad_flag(r_big, w, flag, a1, a2)
    np.testing.assert_array_equal(out1, out2)
    assert s1[:2] == s2[:2]
    assert not out2[flag.astype(bool)].any() and not out2[:10].any()


def test_per_baseline_mode_follows_each_baseline_spread():
    """Two baselines whose residuals differ in scale by 100, the loud one a quarter of the rows:
    with global statistics most of the loud baseline's samples are outliers; per baseline, only
    the outliers planted in each baseline are."""
    from oracle.mad_flag import mad_flag_per_baseline
    rng = np.random.default_rng(4)
    n_row, n_chan = 40, 16
    ant1 = np.zeros(n_row, np.int32)
    ant2 = np.where(np.isin(np.arange(n_row) % 8, (3, 4)), 2, 1).astype(np.int32)
    ant1[::4], ant2[::4] = ant2[::4], 0                      # some rows in the other orientation
    scale = np.where(np.maximum(ant1, ant2) == 2, 100.0, 1.0)[:, None, None]
    r = (scale * (rng.standard_normal((n_row, n_chan, 4)) + 1j * rng.standard_normal((n_row, n_chan, 4)))
         ).astype(np.complex64)
    w = np.ones((n_row, n_chan, 4), np.float32)
    planted = [(2, 3), (5, 7), (3, 1), (12, 12)]          # quiet, quiet, loud, loud (swapped row)
    for row, ch in planted:
        r[row, ch, 0] += np.complex64(60.0 * scale[row, 0, 0])
    out, n = mad_flag_per_baseline(r, w, None, ant1, ant2, threshold=10.0)
    want = np.zeros((n_row, n_chan), np.uint8)
    for row, ch in planted:
        want[row, ch] = 1
    np.testing.assert_array_equal(out, want)
    glob, _ = mad_flag(r, w, None, ant1, ant2, threshold=10.0)
    assert glob[np.maximum(ant1, ant2) == 2].mean() > 0.5      # the global mode flags the loud baseline


def test_per_baseline_mode_equals_global_mode_on_one_baseline():
    from oracle.mad_flag import mad_flag_per_baseline
    rng, r, w, a1, a2 = _residuals(8)
    flag = (rng.random(r.shape[:2]) < 0.1).astype(np.uint8)
    a, n_a = mad_flag_per_baseline(r, w, flag, a1, a2)
    b, (_, _, n_b) = mad_flag(r, w, flag, a1, a2)
    np.testing.assert_array_equal(a, b)
    assert n_a == n_b
