"""Gauge referencing for comparing gain solutions (test infrastructure only).

With an unpolarised sky (M proportional to the identity) the model
V = C_p M C_q^H is unchanged by C_a -> C_a U for any unitary U common to all
antennas, and in a chain G.B a per-antenna diagonal factor can move between
the terms.  Solutions are therefore compared on the product chain C_a of
every (time, channel) sample after removing the unitary factor of a
reference antenna: C_ref = P U (left polar decomposition, P Hermitian
positive semidefinite), C_a <- C_a U^H.  For diagonal gains this reduces to
g_a * conj(g_ref) / |g_ref| per correlation.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def reference_diag(g: np.ndarray, ref: int = 0) -> np.ndarray:
    """Diagonal gains [..., n_ant, 4]: multiply every antenna by the conjugate unit phase of ``ref``."""
    g = np.asarray(g, dtype=np.complex128)
    out = g.copy()
    for k in (0, 3):
        r = g[..., ref:ref + 1, k]
        mag = np.abs(r)
        ph = np.where(mag > 0, np.conj(r) / np.where(mag > 0, mag, 1.0), 1.0)
        out[..., k] = g[..., k] * ph
    return out


def reference_chain(Cj: np.ndarray, ref: int = 0) -> np.ndarray:
    """Full 2x2 products [..., n_ant, 4]: right-multiply by U_ref^H where C_ref = P_ref U_ref."""
    C = np.asarray(Cj, dtype=np.complex128).reshape(Cj.shape[:-1] + (2, 2))
    W, _, Vh = np.linalg.svd(C[..., ref, :, :])
    U = W @ Vh                                        # unitary polar factor of C_ref
    out = C @ np.conj(np.swapaxes(U, -1, -2))[..., None, :, :]
    return out.reshape(Cj.shape)


def chain_products(jones: Sequence[np.ndarray], t_maps, f_maps, n_time: int, n_chan: int) -> np.ndarray:
    """Product chain C_a = prod_j G_{j,a} on the full (time, channel) grid: [n_time, n_chan, n_ant, 4]."""
    n_ant = jones[0].shape[2]
    C = np.zeros((n_time, n_chan, n_ant, 2, 2), dtype=np.complex128)
    C[...] = np.eye(2)
    t = np.arange(n_time)
    c = np.arange(n_chan)
    for J, tm, fm in zip(jones, t_maps, f_maps):
        G = J[np.asarray(tm)[t][:, None], np.asarray(fm)[c][None, :]].reshape(n_time, n_chan, n_ant, 2, 2)
        C = C @ G
    return C.reshape(n_time, n_chan, n_ant, 4)


def rel_err(a: np.ndarray, b: np.ndarray) -> float:
    """max |a - b| / max |b| over all entries."""
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
