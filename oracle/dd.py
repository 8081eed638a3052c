"""Oracle of direction-dependent chains, N_D >= 1 (test infrastructure only).

The model of Eq. baselinemodel with directions: V_pq = sum_d C_{p,d} M_{pq,d} C_{q,d}^H, where
C_{p,d} = prod_j G_{j,p,d} (Eq. joneschain) and each term is either direction-dependent (its
own gains per direction) or direction-independent (the same gains in every direction).  The
derivatives with respect to the solved term n (Eq. chain_trick):
  direction-dependent, per direction d:  dv/dg_{n,p,d} = L_{p,d} (x) (R_{p,d} M_d C_{q,d}^H)^T
                                         (Eq. g_derivative_dd);
  direction-independent: the sum of the same over d (Eq. g_derivative_di);
and for antenna q the conjugate baseline, as in the one-direction oracle.  The AllJones
approximation keeps one block per (interval, antenna) and, for a direction-dependent term,
per direction (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified); the update is Algorithm 1.

Plain numpy with explicit loops over rows, channels and directions: slow, small cases only.
Term kinds: "diag" (free XX, YY), "full" (all four entries) and "delay" (direction-independent
only): four real parameters u = (phi_X, tau_X, phi_Y, tau_Y) per interval and antenna, and the
diagonal gain g_c(nu) = exp(i (phi_c + 2 pi tau_c nu)) at the frequency nu of every channel
(Scenario 2, the residual delay and phase term K).  Its derivatives follow the chain rule
dg_c/dphi_c = i g_c, dg_c/dtau_c = 2 pi nu i g_c, and its blocks are 2 Re(.) of the sums
(Eq. jhj_case2, Eq. jhwr_case2); it converges on the relative change of its gains over the
interval's channels.
"""
from __future__ import annotations

import dataclasses

import numpy as np

PERM = [0, 2, 1, 3]


@dataclasses.dataclass
class DDTerm:
    kind: str                 # "diag", "full" or "delay"
    dd: bool                  # direction-dependent
    t_map: np.ndarray         # [n_time] -> interval
    f_map: np.ndarray         # [n_chan] -> interval
    params: np.ndarray        # complex [n_tint][n_fint][n_ant][n_dir if dd else 1][4]; delay: real [..][1][4]
    solve: bool = True
    max_iter: int = 20
    tol: float = 1e-6
    chan_freq: np.ndarray = None   # delay: [n_chan] frequency of every channel

    @property
    def free(self):
        return [0, 3] if self.kind == "diag" else [0, 1, 2, 3]

    def delay_gains(self, u, c):
        nu = self.chan_freq[c]
        return np.exp(1j * (u[0] + 2 * np.pi * u[1] * nu)), np.exp(1j * (u[2] + 2 * np.pi * u[3] * nu))

    def jones(self, t, c, a, d):
        g = self.params[self.t_map[t], self.f_map[c], a, d if self.dd else 0]
        if self.kind == "delay":
            gx, gy = self.delay_gains(g, c)
            return np.array([[gx, 0], [0, gy]], dtype=np.complex128)
        J = g.reshape(2, 2).copy()
        if self.kind == "diag":
            J[0, 1] = J[1, 0] = 0
        return J

    def columns(self, E, t, c, a):
        """The Jacobian columns of the term's free parameters from E = dv/dvec(G) (4x4)."""
        if self.kind != "delay":
            return E[:, self.free]
        nu = self.chan_freq[c]
        gx, gy = self.delay_gains(self.params[self.t_map[t], self.f_map[c], a, 0], c)
        Ex, Ey = E[:, 0] * 1j * gx, E[:, 3] * 1j * gy
        return np.stack([Ex, 2 * np.pi * nu * Ex, Ey, 2 * np.pi * nu * Ey], axis=1)


@dataclasses.dataclass
class DDProblem:
    data: np.ndarray          # complex [row][chan][4]
    model: np.ndarray         # complex [row][chan][dir][4]
    weight: np.ndarray        # [row][chan][4]
    flag: np.ndarray          # uint8 [row][chan]
    ant1: np.ndarray
    ant2: np.ndarray
    time_idx: np.ndarray
    n_ant: int

    @property
    def n_dir(self):
        return self.model.shape[2]


def _chain(terms, t, c, a, d):
    C = np.eye(2, dtype=np.complex128)
    for T in terms:
        C = C @ T.jones(t, c, a, d)
    return C


def _factors(terms, n, t, c, a, d):
    L = np.eye(2, dtype=np.complex128)
    R = np.eye(2, dtype=np.complex128)
    for j, T in enumerate(terms):
        J = T.jones(t, c, a, d)
        if j < n:
            L = L @ J
        elif j > n:
            R = R @ J
    return L, R


def model_vis(P: DDProblem, terms, row, c, orient=0):
    """V of one sample (orient 1: of the conjugate baseline) as a 2x2 matrix."""
    p, q, t = int(P.ant1[row]), int(P.ant2[row]), int(P.time_idx[row])
    if orient:
        p, q = q, p
    V = np.zeros((2, 2), dtype=np.complex128)
    for d in range(P.n_dir):
        M = P.model[row, c, d].reshape(2, 2)
        if orient:
            M = M.conj().T
        V += _chain(terms, t, c, p, d) @ M @ _chain(terms, t, c, q, d).conj().T
    return V


def residual(P: DDProblem, terms):
    """chi^2 (Eq. min) and r = D - V [row][chan][4] (zero where flagged or autocorrelation)."""
    r = np.zeros_like(P.data)
    chi = 0.0
    for row in range(P.data.shape[0]):
        if P.ant1[row] == P.ant2[row]:
            continue
        for c in range(P.data.shape[1]):
            if P.flag[row, c]:
                continue
            rr = P.data[row, c] - model_vis(P, terms, row, c).reshape(4)
            r[row, c] = rr
            chi += float(np.sum(P.weight[row, c] * np.abs(rr) ** 2))
    return chi, r


def normal_equations(P: DDProblem, terms, n):
    """JHJ [n_tint][n_fint][n_ant][n_blk][np][np] and JHr [..][np] of term n, n_blk = n_dir for a
    direction-dependent term, else 1; np = 2 (diag) or 4 (full)."""
    T = terms[n]
    free = T.free
    npar = len(free)
    nt, nf = T.params.shape[:2]
    nblk = P.n_dir if T.dd else 1
    jhj = np.zeros((nt, nf, P.n_ant, nblk, npar, npar), dtype=np.complex128)
    jhr = np.zeros((nt, nf, P.n_ant, nblk, npar), dtype=np.complex128)
    for row in range(P.data.shape[0]):
        p0, q0, t = int(P.ant1[row]), int(P.ant2[row]), int(P.time_idx[row])
        if p0 == q0:
            continue
        for c in range(P.data.shape[1]):
            if P.flag[row, c]:
                continue
            ti, fi = T.t_map[t], T.f_map[c]
            for orient in (0, 1):
                a, b = (p0, q0) if orient == 0 else (q0, p0)
                D = P.data[row, c].reshape(2, 2)
                w = P.weight[row, c] if orient == 0 else P.weight[row, c][PERM]
                if orient:
                    D = D.conj().T
                r = (D - model_vis(P, terms, row, c, orient)).reshape(4)
                Es = []
                for d in range(P.n_dir):
                    M = P.model[row, c, d].reshape(2, 2)
                    if orient:
                        M = M.conj().T
                    L, R = _factors(terms, n, t, c, a, d)
                    X = R @ M @ _chain(terms, t, c, b, d).conj().T
                    E = T.columns(np.kron(L, X.T), t, c, a)  # Eq. vectrick, restricted to the free parameters
                    Es.append(E)
                blocks = [(d, Es[d]) for d in range(P.n_dir)] if T.dd else [(0, sum(Es))]
                for k, E in blocks:
                    jhj[ti, fi, a, k] += E.conj().T @ (w[:, None] * E)
                    jhr[ti, fi, a, k] += E.conj().T @ (w * r)
    if T.kind == "delay":                            # real parameters: 2 Re(.) (Eq. jhj_case2, Eq. jhwr_case2)
        jhj, jhr = 2 * jhj.real + 0j, 2 * jhr.real + 0j
    return jhj, jhr


def solve_term(P: DDProblem, terms, n, damping_mode: int = 1):
    """Algorithm 1 for term n (per interval; blocks per antenna and, if dd, direction);
    returns iterations per interval.  Singular blocks (zero trace, rcond < 1e-12) keep their gains."""
    T = terms[n]
    free = T.free
    nt, nf = T.params.shape[:2]
    active = np.ones((nt, nf), bool)
    iters = np.zeros((nt, nf), np.int32)
    for k in range(1, T.max_iter + 1):
        if not active.any():
            break
        jhj, jhr = normal_equations(P, terms, n)
        alpha = (0.5 if k % 2 == 0 else 1.0) if damping_mode == 1 else 1.0
        for ti in range(nt):
            for fi in range(nf):
                if not active[ti, fi]:
                    continue
                old = T.params[ti, fi].copy()
                for a in range(P.n_ant):
                    for blk in range(jhj.shape[3]):
                        A, bvec = jhj[ti, fi, a, blk], jhr[ti, fi, a, blk]
                        tr = np.real(np.trace(A))
                        if not tr > 0 or 1.0 / np.linalg.cond(A, 1) < 1e-12:
                            continue
                        x = np.linalg.solve(A, bvec)
                        if T.kind == "delay":
                            T.params[ti, fi, a, blk] += alpha * x.real
                        else:
                            T.params[ti, fi, a, blk, free] += alpha * x
                iters[ti, fi] = k
                if T.kind == "delay":
                    # relative change of the gains over the interval's channels
                    num = den = 0.0
                    for c in np.nonzero(T.f_map == fi)[0]:
                        for a in range(P.n_ant):
                            go = np.array(T.delay_gains(old[a, 0], c))
                            gn = np.array(T.delay_gains(T.params[ti, fi, a, 0], c))
                            num += np.sum(np.abs(gn - go) ** 2)
                            den += np.sum(np.abs(gn) ** 2)
                else:
                    num = np.sum(np.abs(T.params[ti, fi] - old) ** 2)
                    den = np.sum(np.abs(T.params[ti, fi]) ** 2)
                if den == 0 or np.sqrt(num / den) < T.tol:
                    active[ti, fi] = False
    return iters
