"""Robust reweighting between solver epochs (test infrastructure only).

Section 4.3 ("Robust reweighting") reweights the data between solver epochs after Sob et al.
(2020), to limit the pull of RFI and unmodelled emission on the gains; it gives no formulas.
The reading used here is the complex Student's t noise model written as a scale mixture of
complex Gaussians, with one step of expectation-maximisation between epochs:

  - a usable sample s (unflagged cross-correlation) has k_s correlations with w_c > 0 and
    whitened residual power z_s = sum_c w_c |r_c|^2 (w_c the caller's weights);
  - given a mixing variable lambda_s ~ Gamma(shape nu/2, rate nu/2), its residuals are
    independent complex Gaussians CN(0, sigma^2 / (lambda_s w_c));
  - M step (scale, given the previous factors, 1 at the first reweighting):
        sigma^2 = sum_s lambda_s z_s / sum_s k_s;
  - E step (the posterior mean of the mixing variable):
        lambda_s = (nu + 2 k_s) / (nu + 2 z_s / sigma^2);
  - the next epoch solves with weights w_c lambda_s.

nu is fixed by the caller (large nu: the Gaussian limit, lambda -> 1).  FP64 numpy.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def whitened_power(resid, weight, flag, ant1, ant2):
    """z [row][chan] = sum_c w_c |r_c|^2 and k [row][chan] = #(w_c > 0), both zero where the
    sample is flagged or an autocorrelation."""
    resid = np.asarray(resid, dtype=np.complex128)
    w = np.asarray(weight, dtype=np.float64)
    use = np.asarray(ant1)[:, None] != np.asarray(ant2)[:, None]
    use = np.broadcast_to(use, w.shape[:2]).copy()
    if flag is not None:
        use &= np.asarray(flag) == 0
    z = np.where(use, np.sum(w * np.abs(resid) ** 2, axis=-1), 0.0)
    k = np.where(use, np.sum(w > 0, axis=-1), 0)
    return z, k


def reweight(resid, weight, flag, ant1, ant2, nu, lam_prev=None):
    """One EM step: (lambda [row][chan], sigma^2).  lambda is 1 where the sample is unusable."""
    z, k = whitened_power(resid, weight, flag, ant1, ant2)
    lp = np.ones_like(z) if lam_prev is None else np.asarray(lam_prev, dtype=np.float64)
    n_comp = float(np.sum(k))
    sigma2 = float(np.sum(lp * z) / n_comp) if n_comp > 0 else 1.0
    lam = np.where(k > 0, (nu + 2.0 * k) / (nu + 2.0 * z / sigma2), 1.0) if sigma2 > 0 else np.ones_like(z)
    return lam, sigma2


def solve_robust(problem: O.OracleProblem, terms, n_epochs: int, nu: float, damping_mode: int = 1):
    """The chain schedule with robust reweighting between epochs: after every epoch but the
    last, one EM step on the residual of the current gains (whitened by the caller's weights)
    sets the weights of the next epoch.  Returns (iterations of the last epoch, the factors of
    the last reweighting or None, sigma^2 of the last reweighting or None).  The problem's
    weights are restored before returning."""
    w0 = problem.weight.copy()
    lam, sigma2, its = None, None, None
    try:
        for e in range(n_epochs):
            its = O.solve(problem, terms, n_epochs=1, damping_mode=damping_mode)
            if e == n_epochs - 1:
                break
            np.copyto(problem.weight, w0)
            _, r = O.residual(problem, terms, want_resid=True)
            lam, sigma2 = reweight(r, w0, problem.flag, problem.ant1, problem.ant2, nu, lam)
            np.copyto(problem.weight, w0 * lam[:, :, None])
    finally:
        np.copyto(problem.weight, w0)
    return its, lam, sigma2
