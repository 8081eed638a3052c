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


# ---------------------------------------------------------------------------
# the 4x4 full-Jones form (any single term: diagonal, full or phase-only)
# ---------------------------------------------------------------------------
#
# A single term G with gains constant over each solution interval (bin).  Per bin and
# baseline (p, q), p < q (rows with p > q through their conjugate orientation), with the
# weight index kj = 2k + j of correlation (k, j) and the row-major index u = 2l + m of the
# 2x2 model entry M_lm:
#     S[kj][u][v] = sum w_kj conj(M_u) M_v        (Hermitian in u, v)
#     T[kj][u]    = sum w_kj conj(M_u) D_kj
#     U[kj]       = sum w_kj |D_kj|^2
# Antenna p: X = M G_q^H and E = I (x) X^T (Eq. vectrick with L = I), so with the parameter
# index 2k + l of G_p,kl
#     JHJ_p[(k,l),(k,l')] += sum_j sum_m sum_m' G_q,jm conj(G_q,jm') S[kj][(l,m)][(l',m')]
#     b_p[(k,l)]          += sum_j sum_m G_q,jm T[kj][(l,m)]
# and antenna q, through the conjugate baseline (D -> D^H, M -> M^H, w -> P w),
#     JHJ_q[(k,l),(k,l')] += sum_j sum_m sum_m' G_p,jm conj(G_p,jm') conj(S[jk][(m,l)][(m',l')])
#     b_q[(k,l)]          += sum_j sum_m G_p,jm conj(T[jk][(m,l)]).
# Summed over an antenna's baselines, JHr = b - JHJ vec(G) (V = E vec(G_p) for every sample),
# and chi^2 = sum U - 2 Re sum_{k,j,l,m} conj(G_p,kl) G_q,jm T[kj][(l,m)] + vec(G_p)^H JHJ_p vec(G_p)
# per baseline.  A diagonal term takes the (0, 3) rows and columns; a phase-only term applies
# its chain rule to those.

def moments_full(problem, t_map, f_map, n_tint: int, n_fint: int):
    """S [bin][n_ant][n_ant][4][4][4] complex, T [bin][n_ant][n_ant][4][4] complex, U [..][4] real,
    bin = t_int * n_fint + f_int, keyed by (p, q) with p < q."""
    na = problem.n_ant
    nb = n_tint * n_fint
    S = np.zeros((nb, na, na, 4, 4, 4), dtype=np.complex128)
    T = np.zeros((nb, na, na, 4, 4), dtype=np.complex128)
    U = np.zeros((nb, na, na, 4))
    perm = [0, 2, 1, 3]
    for row in range(problem.data.shape[0]):
        p, q, t = int(problem.ant1[row]), int(problem.ant2[row]), int(problem.time_idx[row])
        if p == q:
            continue
        for ch in range(problem.data.shape[1]):
            if problem.flag is not None and problem.flag[row, ch]:
                continue
            b = int(t_map[t]) * n_fint + int(f_map[ch])
            d, m, w = problem.data[row, ch], problem.model[row, ch], problem.weight[row, ch]
            if p > q:
                d, m, w = np.conj(d[perm]), np.conj(m[perm]), w[perm]
            a, c = min(p, q), max(p, q)
            S[b, a, c] += w[:, None, None] * np.conj(m)[None, :, None] * m[None, None, :]
            T[b, a, c] += w[:, None] * np.conj(m)[None, :] * d[:, None]
            U[b, a, c] += w * np.abs(d) ** 2
    return S, T, U


def normal_equations_full(S, T, gains):
    """JHJ [bin][n_ant][4][4] and JHr [bin][n_ant][4] of a single full 2x2 term with gains
    [bin][n_ant][4] (row-major G), from the baseline sums."""
    nb, na = S.shape[:2]
    jhj = np.zeros((nb, na, 4, 4), dtype=np.complex128)
    bvec = np.zeros((nb, na, 4), dtype=np.complex128)
    for b in range(nb):
        G = gains[b].reshape(na, 2, 2)
        for p in range(na):
            for q in range(p + 1, na):
                for k in range(2):
                    for j in range(2):
                        kj, jk = 2 * k + j, 2 * j + k
                        for l in range(2):
                            for l2 in range(2):
                                for m in range(2):
                                    for m2 in range(2):
                                        u, v = 2 * l + m, 2 * l2 + m2
                                        jhj[b, p, 2 * k + l, 2 * k + l2] += \
                                            G[q, j, m] * np.conj(G[q, j, m2]) * S[b, p, q, kj, u, v]
                                        uq, vq = 2 * m + l, 2 * m2 + l2
                                        jhj[b, q, 2 * k + l, 2 * k + l2] += \
                                            G[p, j, m] * np.conj(G[p, j, m2]) * np.conj(S[b, p, q, jk, uq, vq])
                            for m in range(2):
                                bvec[b, p, 2 * k + l] += G[q, j, m] * T[b, p, q, kj, 2 * l + m]
                                bvec[b, q, 2 * k + l] += G[p, j, m] * np.conj(T[b, p, q, jk, 2 * m + l])
    jhr = bvec - np.einsum("bauv,bav->bau", jhj, gains.reshape(nb, na, 4))
    return jhj, jhr


def chi2_from_moments_full(S, T, U, gains):
    nb, na = S.shape[:2]
    tot = 0.0
    for b in range(nb):
        G = gains[b].reshape(na, 2, 2)
        for p in range(na):
            for q in range(p + 1, na):
                tot += float(np.sum(U[b, p, q]))
                gp = G[p].reshape(4)
                H = np.zeros((4, 4), dtype=np.complex128)
                cross = 0.0 + 0.0j
                for k in range(2):
                    for j in range(2):
                        kj = 2 * k + j
                        for l in range(2):
                            for m in range(2):
                                cross += np.conj(G[p, k, l]) * G[q, j, m] * T[b, p, q, kj, 2 * l + m]
                                for l2 in range(2):
                                    for m2 in range(2):
                                        H[2 * k + l, 2 * k + l2] += (G[q, j, m] * np.conj(G[q, j, m2]) *
                                                                     S[b, p, q, kj, 2 * l + m, 2 * l2 + m2])
                tot += -2.0 * cross.real + float(np.real(np.conj(gp) @ H @ gp))
    return tot
