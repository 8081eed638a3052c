"""Oracle of the MAD residual flagger (test infrastructure only).

Section 4 ("Additional features"): outliers in the residual visibilities after calibration
are found with the Median Absolute Deviation, over all baselines at once.  Readings (also
listed in the design notes):

- the statistic of an unflagged cross-correlation sample is its whitened residual norm
  z = sqrt(sum over the four correlations of w |r|^2), in float32 with every operation
  rounded (no fused multiply-add): t_c = re*re + im*im, acc = ((w_0 t_0 + w_1 t_1) + w_2 t_2)
  + w_3 t_3, z = sqrt(acc);
- median and MAD are exact order statistics: the floor((n - 1) / 2)-th smallest value
  (0-based) of the n samples' z, then of their deviations |z - median|;
- a sample is flagged when |z - median| > fl32(threshold * 1.4826) * MAD, the product and
  the comparison in float32 (1.4826 makes the MAD a standard deviation for Gaussian data).

These decide bytes, so they are taken in float32 on both sides, in the same order.
"""
from __future__ import annotations

import numpy as np


def whitened_norm(resid: np.ndarray, weight: np.ndarray) -> np.ndarray:
    """z [n_row][n_chan] float32 from resid complex64 [..][4] and weight float32 [..][4]."""
    r = np.asarray(resid, dtype=np.complex64)
    w = np.asarray(weight, dtype=np.float32)
    re, im = r.real.astype(np.float32), r.imag.astype(np.float32)
    acc = np.zeros(r.shape[:-1], dtype=np.float32)
    for c in range(4):
        t = re[..., c] * re[..., c] + im[..., c] * im[..., c]
        acc = acc + w[..., c] * t
    return np.sqrt(acc)


def order_statistic(values: np.ndarray) -> np.float32:
    """The floor((n - 1) / 2)-th smallest element of a non-empty float32 array."""
    v = np.sort(np.asarray(values, dtype=np.float32), kind="stable")
    return v[(v.size - 1) // 2]


def mad_flag_per_baseline(resid, weight, flag, ant1, ant2, threshold: float = 5.0):
    """The per-baseline mode: median and MAD of z over the samples of each baseline (all its
    rows and channels, whatever the row orientation) instead of over all baselines; the rest as
    mad_flag.  Returns the new flags and the number flagged."""
    flag = np.zeros(np.shape(resid)[:2], np.uint8) if flag is None else np.asarray(flag)
    a1, a2 = np.asarray(ant1), np.asarray(ant2)
    z = whitened_norm(resid, weight)
    out = np.zeros(flag.shape, dtype=np.uint8)
    key = np.minimum(a1, a2).astype(np.int64) * (int(max(a1.max(), a2.max())) + 1) + np.maximum(a1, a2)
    factor = np.float32(threshold * 1.4826)
    for k in np.unique(key[a1 != a2]):
        rows = np.nonzero(key == k)[0]
        use = flag[rows] == 0
        if not use.any():
            continue
        zb = z[rows]
        med = order_statistic(zb[use])
        dev = np.abs(zb - med)
        mad = order_statistic(dev[use])
        out[rows] = (use & (dev > factor * mad)).astype(np.uint8)
    return out, int(out.sum())


def mad_flag(resid, weight, flag, ant1, ant2, threshold: float = 5.0):
    """New flags uint8 [n_row][n_chan] (1 = outlier) and (median, MAD, number flagged)."""
    flag = np.zeros(np.shape(resid)[:2], np.uint8) if flag is None else np.asarray(flag)
    cross = (np.asarray(ant1) != np.asarray(ant2))[:, None]
    use = (flag == 0) & cross
    out = np.zeros(flag.shape, dtype=np.uint8)
    if not use.any():
        return out, (np.float32(0), np.float32(0), 0)
    z = whitened_norm(resid, weight)
    med = order_statistic(z[use])
    dev = np.abs(z - med)
    mad = order_statistic(dev[use])
    thr = np.float32(threshold * 1.4826) * mad
    out[use & (dev > thr)] = 1
    return out, (med, mad, int(out.sum()))
