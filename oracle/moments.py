"""Oracle of the sufficient-statistics pre-reduction (test infrastructure only).

Not in the paper: when the solved term is the only term of the chain and diagonal, every
sample of a baseline (p, q) in a solution interval enters JHJ and JHr (Eq. jhj_entry_simplified,
Eq. jhr_entry_simplified) through three weighted sums of that baseline and interval, per
correlation c:
    S_c = sum w_c |m_c|^2,   T_c = sum w_c conj(m_c) d_c,   U_c = sum w_c |d_c|^2.
With the gains g_a = diag(g_a0, g_a1) constant over the interval, and correlations ordered
(XX, XY, YX, YY) = (0, 1, 2, 3), antenna p of baseline (p, q) receives
    JHJ[0][0] += S_0 |g_q0|^2 + S_1 |g_q1|^2           JHJ[1][1] += S_2 |g_q0|^2 + S_3 |g_q1|^2
    JHr[0]    += g_q0 T_0 + g_q1 T_1 - g_p0 JHJ-term   JHr[1]    += g_q0 T_2 + g_q1 T_3 - g_p1 JHJ-term
and antenna q the same through the conjugate baseline (S_1 <-> S_2, T -> conj(T) with T_1 <-> T_2,
p <-> q).  With G_c = g_p,i conj(g_q,j) the gain product of correlation c = (i, j),
chi^2 = sum over baselines and correlations of U_c - 2 Re(conj(G_c) T_c) + |G_c|^2 S_c.
Each iteration then costs one pass over the baselines instead of one over the samples.
"""
from __future__ import annotations

import numpy as np


def moments(problem, t_map, n_tint: int):
    """S [n_tint][n_ant][n_ant][4] (real), T (complex), U (real), keyed by (p, q) with p < q:
    rows with p > q enter through their conjugate orientation."""
    na = problem.n_ant
    S = np.zeros((n_tint, na, na, 4))
    T = np.zeros((n_tint, na, na, 4), dtype=np.complex128)
    U = np.zeros((n_tint, na, na, 4))
    perm = [0, 2, 1, 3]
    for row in range(problem.data.shape[0]):
        p, q, t = int(problem.ant1[row]), int(problem.ant2[row]), int(problem.time_idx[row])
        if p == q:
            continue
        ti = int(t_map[t])
        for ch in range(problem.data.shape[1]):
            if problem.flag is not None and problem.flag[row, ch]:
                continue
            d, m, w = problem.data[row, ch], problem.model[row, ch], problem.weight[row, ch]
            if p > q:        # the conjugate baseline: D, M -> D^H, M^H, weights permuted
                d, m, w = np.conj(d[perm]), np.conj(m[perm]), w[perm]
            a, b = min(p, q), max(p, q)
            S[ti, a, b] += w * np.abs(m) ** 2
            T[ti, a, b] += w * np.conj(m) * d
            U[ti, a, b] += w * np.abs(d) ** 2
    return S, T, U


def normal_equations_from_moments(S, T, gains):
    """JHJ [n_tint][n_ant][2][2] and JHr [n_tint][n_ant][2] of a single diagonal term with gains
    [n_tint][n_ant][2] (the XX and YY entries), from the baseline sums."""
    n_tint, na = S.shape[:2]
    jhj = np.zeros((n_tint, na, 2, 2), dtype=np.complex128)
    jhr = np.zeros((n_tint, na, 2), dtype=np.complex128)
    for ti in range(n_tint):
        g = gains[ti]
        for p in range(na):
            for q in range(p + 1, na):
                s, t = S[ti, p, q], T[ti, p, q]
                # antenna p through baseline (p, q)
                h0 = s[0] * abs(g[q, 0]) ** 2 + s[1] * abs(g[q, 1]) ** 2
                h1 = s[2] * abs(g[q, 0]) ** 2 + s[3] * abs(g[q, 1]) ** 2
                jhj[ti, p, 0, 0] += h0
                jhj[ti, p, 1, 1] += h1
                jhr[ti, p, 0] += g[q, 0] * t[0] + g[q, 1] * t[1] - g[p, 0] * h0
                jhr[ti, p, 1] += g[q, 0] * t[2] + g[q, 1] * t[3] - g[p, 1] * h1
                # antenna q through the conjugate baseline (q, p)
                k0 = s[0] * abs(g[p, 0]) ** 2 + s[2] * abs(g[p, 1]) ** 2
                k1 = s[1] * abs(g[p, 0]) ** 2 + s[3] * abs(g[p, 1]) ** 2
                jhj[ti, q, 0, 0] += k0
                jhj[ti, q, 1, 1] += k1
                jhr[ti, q, 0] += g[p, 0] * np.conj(t[0]) + g[p, 1] * np.conj(t[2]) - g[q, 0] * k0
                jhr[ti, q, 1] += g[p, 0] * np.conj(t[1]) + g[p, 1] * np.conj(t[3]) - g[q, 1] * k1
    return jhj, jhr


def chi2_from_moments(S, T, U, gains):
    """chi^2 = sum over baselines and correlations of U - 2 Re(conj(G) T) + |G|^2 S, where
    G = g_p,i conj(g_q,j) is the gain product of correlation (i, j)."""
    n_tint, na = S.shape[:2]
    idx = [(0, 0), (0, 1), (1, 0), (1, 1)]
    tot = 0.0
    for ti in range(n_tint):
        g = gains[ti]
        for p in range(na):
            for q in range(p + 1, na):
                for c, (i, j) in enumerate(idx):
                    G = g[p, i] * np.conj(g[q, j])
                    tot += U[ti, p, q, c] - 2 * np.real(np.conj(G) * T[ti, p, q, c]) + abs(G) ** 2 * S[ti, p, q, c]
    return tot
