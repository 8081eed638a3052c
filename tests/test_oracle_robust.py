"""Pins of the robust reweighting oracle (Section 4.3, "Robust reweighting", after Sob et al.
2020; the Student's t scale-mixture reading stated in oracle/robust.py).

- The E step's factor equals the posterior mean of the mixing variable, computed by numerical
  integration over its Gamma prior times the complex Gaussian likelihood.
- The M step's scale maximises the expected complete-data log-likelihood (brute force on a grid).
- The Gaussian limit (nu -> inf) leaves the weights unchanged; a sample at the expected power
  k sigma^2 keeps factor 1; residuals scaled by c scale sigma^2 by c^2 and leave the factors.
- Planted outliers get factors far below those of the Gaussian samples; flagged samples and
  autocorrelations keep factor 1 and do not enter the scale.
- With planted RFI, the robust chain solve lands closer to the true gains than the plain one.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import robust
from oracle.gauge import reference_diag, rel_err
from paper_2412_10072_gb300 import synth

scipy_integrate = pytest.importorskip("scipy.integrate")
scipy_special = pytest.importorskip("scipy.special")


def _lam(z, k, sigma2, nu):
    return (nu + 2.0 * k) / (nu + 2.0 * z / sigma2)


@pytest.mark.parametrize("z,k,sigma2,nu", [(0.3, 4, 1.0, 5.0), (8.0, 4, 2.0, 3.0), (150.0, 2, 0.7, 10.0),
                                           (1.0, 1, 1.0, 0.5)])
def test_factor_is_the_posterior_mean_of_the_mixing_variable(z, k, sigma2, nu):
    # p(lambda | r) propto Gamma(lambda; nu/2, rate nu/2) * (lambda / sigma2)^k exp(-lambda z / sigma2)
    def log_post(lam):
        log_prior = (nu / 2) * math.log(nu / 2) - scipy_special.gammaln(nu / 2) + (nu / 2 - 1) * math.log(lam) - nu / 2 * lam
        return log_prior + k * math.log(lam / sigma2) - lam * z / sigma2
    grid = np.logspace(-8, 4, 2000)
    lp = np.array([log_post(g) for g in grid])
    top, peak = lp.max(), grid[int(np.argmax(lp))]           # numerical conditioning only

    def post(lam, moment):
        return lam ** moment * math.exp(log_post(lam) - top)
    hi = peak * 200.0
    num = scipy_integrate.quad(post, 0, hi, args=(1,), points=[peak], limit=800, epsrel=1e-12)[0]
    den = scipy_integrate.quad(post, 0, hi, args=(0,), points=[peak], limit=800, epsrel=1e-12)[0]
    assert abs(num / den - _lam(z, k, sigma2, nu)) <= 1e-7 * (num / den)


def test_scale_maximises_the_expected_log_likelihood():
    rng = np.random.default_rng(0)
    n_row, n_chan = 40, 8
    r = rng.standard_normal((n_row, n_chan, 4)) + 1j * rng.standard_normal((n_row, n_chan, 4))
    w = rng.uniform(0.5, 2, (n_row, n_chan, 4))
    a1, a2 = np.zeros(n_row, np.int32), np.ones(n_row, np.int32)
    lam_prev = rng.uniform(0.2, 1.5, (n_row, n_chan))
    _, s2 = robust.reweight(r, w, None, a1, a2, 4.0, lam_prev)
    z, k = robust.whitened_power(r, w, None, a1, a2)
    grid = s2 * np.linspace(0.8, 1.2, 4001)
    q = [-np.sum(k) * math.log(g) - np.sum(lam_prev * z) / g for g in grid]
    assert abs(grid[int(np.argmax(q))] - s2) <= 1.5e-4 * s2


def test_gaussian_limit_expected_power_and_scale_invariance():
    rng = np.random.default_rng(1)
    r = rng.standard_normal((30, 6, 4)) + 1j * rng.standard_normal((30, 6, 4))
    w = np.ones((30, 6, 4))
    a1, a2 = np.zeros(30, np.int32), np.ones(30, np.int32)
    lam, _ = robust.reweight(r, w, None, a1, a2, 1e12)
    assert np.max(np.abs(lam - 1)) < 1e-9
    lam, s2 = robust.reweight(r, w, None, a1, a2, 3.0)
    r2 = r.copy()
    z0 = 4 * s2                                    # a sample at the expected power k sigma^2
    r2[0, 0] = np.sqrt(z0 / 4)
    lam2, s2b = robust.reweight(r2, w, None, a1, a2, 3.0)
    z, _ = robust.whitened_power(r2, w, None, a1, a2)
    np.testing.assert_allclose(lam2[0, 0], (3 + 8) / (3 + 2 * z[0, 0] / s2b), rtol=1e-14)
    lam3, s23 = robust.reweight(7.0 * r, w, None, a1, a2, 3.0)
    np.testing.assert_allclose(s23, 49.0 * s2, rtol=1e-12)
    np.testing.assert_allclose(lam3, lam, rtol=1e-12)
    rr = np.full((1, 1, 4), np.sqrt(2.0))
    lam1, s21 = robust.reweight(rr, np.ones((1, 1, 4)), None, np.zeros(1, np.int32), np.ones(1, np.int32), 5.0)
    assert abs(s21 - 2.0) <= 1e-15 and abs(lam1[0, 0] - 1.0) <= 1e-15   # z = k sigma^2: factor 1


def test_planted_outliers_flags_and_autocorrelations():
    rng = np.random.default_rng(2)
    n_row, n_chan = 500, 16
    r = (rng.standard_normal((n_row, n_chan, 4)) + 1j * rng.standard_normal((n_row, n_chan, 4))) / np.sqrt(2)
    out = rng.choice(n_row * n_chan, 40, replace=False)
    rf = r.reshape(-1, 4)
    rf[out] *= 40.0
    w = np.ones_like(r.real)
    a1 = np.zeros(n_row, np.int32)
    a2 = np.ones(n_row, np.int32)
    a2[:5] = 0                                      # autocorrelations
    flag = np.zeros((n_row, n_chan), np.uint8)
    flag[10, :] = 1
    r[10] = 1e6                                     # a flagged row with huge residuals
    lam1, s21 = robust.reweight(r, w, flag, a1, a2, 5.0)
    lam, s2 = robust.reweight(r, w, flag, a1, a2, 5.0, lam1)    # a second EM step
    lf = lam.reshape(-1)
    mask = np.zeros(lf.size, bool)
    mask[out] = True
    usable = (np.arange(n_row)[:, None] >= 5) & (flag == 0)
    usable = usable.reshape(-1)
    assert np.all(lam[:5] == 1) and np.all(lam[10] == 1)
    assert np.max(lf[mask & usable]) < 0.01 * np.median(lf[~mask & usable])
    # the outliers inflate the first scale estimate; the second step, with them down-weighted, shrinks it
    z, k = robust.whitened_power(r, w, flag, a1, a2)
    assert s21 > 2.0 and s2 < 0.6 * s21
    np.testing.assert_allclose(s21, z.sum() / k.sum(), rtol=1e-12)


def test_robust_solve_resists_planted_rfi():
    obs = synth.plain_small(seed=7, noise=0.01)
    rng = np.random.default_rng(3)
    bad = rng.random(obs.flag.shape) < 0.01
    obs.data[bad] += 5.0 * (rng.standard_normal((bad.sum(), 4)) + 1j * rng.standard_normal((bad.sum(), 4)))
    truth = reference_diag(obs.terms[0].truth.astype(np.complex128))
    errs = []
    for nu in (None, 3.0):
        P = O.OracleProblem.from_obs(obs)
        T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
        if nu is None:
            O.solve(P, [T], n_epochs=3, damping_mode=1)
        else:
            robust.solve_robust(P, [T], 3, nu)
        errs.append(rel_err(reference_diag(T.params), truth))
    assert errs[1] < 0.5 * errs[0], errs
