"""FP64 oracle of the delay term's initial estimate (test infrastructure only).

Section 4.3 ("Initial estimates"): a delay can be estimated from the peak of the Fourier
transform along frequency of the baselines that include the reference antenna.  Readings
(also listed in the design notes):

- the spectrum of antenna a, correlation c in {XX, YY}, over the channels of a parameter
  interval is x(nu) = sum over the interval's rows on baselines (a, ref) or (ref, a) of
  w d conj(m) for that correlation (unflagged samples only), conjugated for rows (ref, a),
  so that x ~ g_a conj(g_ref) |m|^2 with phase phi_a + 2 pi tau_a nu in the gauge of ref;
- the channels of an interval are uniformly spaced (dnu); the spectrum is zero-padded to
  N = the next power of two >= oversample x (its channels), and X_k = FFT(x)_k is its
  transform at the delays tau_k = k / (N dnu), k = -N/2 .. N/2 - 1;
- the peak is the largest |X_k| (the lowest k among equal values), tau = tau_k and
  phi = arg X_k - 2 pi tau nu_0 with nu_0 the interval's first channel, wrapped to (-pi, pi];
- the reference antenna, antennas without data, and intervals of one channel keep tau = 0
  (one channel: phi = arg x).

numpy's FFT is the transform step; nothing else here is more than the definition.
"""
from __future__ import annotations

import numpy as np


def next_pow2(n: int) -> int:
    p = 1
    while p < n:
        p *= 2
    return p


def delay_spectra(problem, t_map, n_tint: int, ref: int) -> np.ndarray:
    """x [n_tint][n_ant][2][n_chan] complex128, as in the module docstring."""
    n_chan = problem.data.shape[1]
    x = np.zeros((n_tint, problem.n_ant, 2, n_chan), dtype=np.complex128)
    for row in range(problem.data.shape[0]):
        p, q, t = int(problem.ant1[row]), int(problem.ant2[row]), int(problem.time_idx[row])
        if p == q or ref not in (p, q):
            continue
        a = q if p == ref else p
        ti = int(t_map[t])
        for c in range(n_chan):
            if problem.flag is not None and problem.flag[row, c]:
                continue
            for k, corr in ((0, 0), (1, 3)):
                z = problem.weight[row, c, corr] * problem.data[row, c, corr] * np.conj(problem.model[row, c, corr])
                x[ti, a, k, c] += np.conj(z) if p == ref else z
    return x


def delay_init(problem, t_map, f_map, n_tint: int, n_fint: int, chan_freq, ref: int = 0,
               oversample: int = 4) -> np.ndarray:
    """Initial parameters [n_tint][n_fint][n_ant][4] = (phi_X, tau_X, phi_Y, tau_Y)."""
    nu = np.asarray(chan_freq, dtype=np.float64)
    f_map = np.asarray(f_map)
    x = delay_spectra(problem, t_map, n_tint, ref)
    out = np.zeros((n_tint, n_fint, problem.n_ant, 4))
    for fi in range(n_fint):
        chans = np.nonzero(f_map == fi)[0]
        if chans.size == 0:
            continue
        c0, n_c = int(chans[0]), int(chans.size)
        N = next_pow2(oversample * n_c)
        dnu = (nu[chans[-1]] - nu[c0]) / (n_c - 1) if n_c > 1 else 0.0
        ks = np.arange(N)
        ks = np.where(ks < N // 2, ks, ks - N)                # signed delay index of each FFT bin
        order = np.argsort(ks, kind="stable")                 # bins in increasing k
        for ti in range(n_tint):
            for a in range(problem.n_ant):
                if a == ref:
                    continue
                for k in range(2):
                    xs = x[ti, a, k, chans]
                    if not np.any(xs != 0):
                        continue
                    if n_c == 1:
                        out[ti, fi, a, 2 * k] = np.angle(xs[0])
                        continue
                    X = np.fft.fft(xs, n=N)
                    mag = np.abs(X[order]) ** 2
                    best = order[int(np.argmax(mag))]          # first maximum in increasing k
                    tau = ks[best] / (N * dnu)
                    phi = np.angle(X[best]) - 2 * np.pi * tau * nu[c0]
                    out[ti, fi, a, 2 * k] = np.angle(np.exp(1j * phi))
                    out[ti, fi, a, 2 * k + 1] = tau
    return out
