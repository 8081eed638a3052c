"""Pins of the oracle's delay term (Scenario 2 of Section 2.4: gains evaluated per channel
from per-interval parameters, g_c(nu) = exp(i (phi_c + 2 pi tau_c nu)), parameters
(phi_X, tau_X, phi_Y, tau_Y) per antenna and interval).

The forward model here is written independently of the oracle (numpy, per sample), and
the normal equations are pinned against central differences of it in the real
parameters: JHJ = 2 Re(J^H W J), JHr = -2 Re(J^H W r) with J = dr/du
(Eq. jhj_entry_param, Eq. jhwr_entry_param; Eq. jhj_case2, Eq. jhwr_case2 restrict
them to one antenna's block).  Exact recovery of the generating parameters and the
singular case with one frequency close the set."""
import numpy as np
import pytest

import oracle as O
from paper_2412_10072_gb300 import synth


def _problem(seed, n_ant=4, n_time=3, n_chan=6, flag_frac=0.15):
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(n_ant)
    ant1 = np.tile(p, n_time)
    ant2 = np.tile(q, n_time)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    shp = (ant1.size, n_chan, 4)
    data = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    model = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    weight = rng.uniform(0.5, 2.0, size=shp)
    flag = (rng.random(shp[:2]) < flag_frac).astype(np.uint8)
    prob = O.OracleProblem(data, model, weight, flag, ant1, ant2, tidx, n_ant, n_time)
    nu = np.linspace(0.9, 1.7, n_chan)                 # GHz; delays in ns
    return prob, nu, rng


def _term(kind, prob, nu, rng, nt=1, nf=1):
    n_time, n_chan, n_ant = prob.n_time, prob.data.shape[1], prob.n_ant
    tm = (np.arange(n_time) * nt // n_time).astype(np.int32)
    fm = (np.arange(n_chan) * nf // n_chan).astype(np.int32)
    if kind == "delay":
        par = np.zeros((nt, nf, n_ant, 4))
        par[..., 0::2] = rng.uniform(-np.pi, np.pi, size=(nt, nf, n_ant, 2))
        par[..., 1::2] = rng.uniform(-0.4, 0.4, size=(nt, nf, n_ant, 2))
        return O.OracleTerm("delay", tm, fm, nt, nf, n_ant, params=par, chan_freq=nu)
    if kind == "phase":
        return O.OracleTerm("phase", tm, fm, nt, nf, n_ant, params=rng.uniform(-np.pi, np.pi, (nt, nf, n_ant, 2)))
    par = 1.0 + 0.3 * (rng.standard_normal((nt, nf, n_ant, 4)) + 1j * rng.standard_normal((nt, nf, n_ant, 4)))
    return O.OracleTerm(kind, tm, fm, nt, nf, n_ant, params=par)


def _jones(term, t, c, a):
    """2x2 Jones matrix of one term at data time t, channel c, antenna a (written out here)."""
    u = term.params[term.t_map[t], term.f_map[c], a]
    J = np.zeros((2, 2), dtype=np.complex128)
    if term.kind == "delay":
        nu = term.chan_freq[c]
        J[0, 0] = np.exp(1j * (u[0] + 2 * np.pi * u[1] * nu))
        J[1, 1] = np.exp(1j * (u[2] + 2 * np.pi * u[3] * nu))
    elif term.kind == "phase":
        J[0, 0], J[1, 1] = np.exp(1j * u[0]), np.exp(1j * u[1])
    elif term.kind == "diag":
        J[0, 0], J[1, 1] = u[0], u[3]
    else:
        J[:] = u.reshape(2, 2)
    return J


def _residual(prob, terms):
    """r = D - C_p M C_q^H per sample (zero where flagged or autocorrelation), [row][chan][4]."""
    n_row, n_chan = prob.data.shape[:2]
    r = np.zeros_like(prob.data)
    for row in range(n_row):
        p, q, t = prob.ant1[row], prob.ant2[row], prob.time_idx[row]
        if p == q:
            continue
        for c in range(n_chan):
            if prob.flag[row, c]:
                continue
            Cp = np.eye(2, dtype=np.complex128)
            Cq = np.eye(2, dtype=np.complex128)
            for T in terms:
                Cp = Cp @ _jones(T, t, c, p)
                Cq = Cq @ _jones(T, t, c, q)
            V = Cp @ prob.model[row, c].reshape(2, 2) @ Cq.conj().T
            r[row, c] = prob.data[row, c] - V.reshape(4)
    return r


def _weights(prob):
    w = prob.weight.copy()
    w[prob.flag.astype(bool)] = 0.0
    w[prob.ant1 == prob.ant2] = 0.0
    return w.reshape(-1)


CHAINS = [(("delay",), 0), (("delay", "diag"), 0), (("full", "delay"), 1), (("phase", "delay", "full"), 1)]


@pytest.mark.parametrize("kinds,n", CHAINS)
def test_residual_with_delay_term_matches_forward_model(kinds, n):
    prob, nu, rng = _problem(3)
    terms = [_term(k, prob, nu, rng, nt=2, nf=2) for k in kinds]
    chi2, r = O.residual(prob, terms, want_resid=True)
    want = _residual(prob, terms)
    np.testing.assert_allclose(r, want, rtol=0, atol=1e-12 * np.abs(want).max())
    assert abs(chi2 - np.sum(_weights(prob) * np.abs(want.reshape(-1)) ** 2)) <= 1e-11 * chi2


@pytest.mark.parametrize("kinds,n", CHAINS)
def test_delay_normal_equations_match_finite_differences(kinds, n):
    prob, nu, rng = _problem(7 + n)
    terms = [_term(k, prob, nu, rng, nt=2, nf=2) for k in kinds]
    T = terms[n]
    jhj, jhr = O.normal_equations(prob, terms, n)
    w = _weights(prob)
    r0 = _residual(prob, terms).reshape(-1)
    h = 1e-6
    for it in range(T.n_tint):
        for jf in range(T.n_fint):
            for a in range(prob.n_ant):
                cols = []
                for k in range(4):
                    base = T.params[it, jf, a, k]
                    T.params[it, jf, a, k] = base + h
                    rp = _residual(prob, terms).reshape(-1)
                    T.params[it, jf, a, k] = base - h
                    rm = _residual(prob, terms).reshape(-1)
                    T.params[it, jf, a, k] = base
                    cols.append((rp - rm) / (2 * h))
                J = np.stack(cols, axis=1)
                fj = 2 * np.real(J.conj().T @ (w[:, None] * J))
                fr = -2 * np.real(J.conj().T @ (w * r0))
                sj, sr = max(1.0, np.abs(fj).max()), max(1.0, np.abs(fr).max())
                assert np.abs(jhj[it, jf, a] - fj).max() <= 1e-7 * sj, (it, jf, a)
                assert np.abs(jhr[it, jf, a] - fr).max() <= 1e-7 * sr, (it, jf, a)
                assert np.abs(jhj[it, jf, a].imag).max() == 0 and np.abs(jhr[it, jf, a].imag).max() == 0


def test_delay_solve_recovers_generating_parameters():
    """Noise-free data from known phases and delays: the solve from zero recovers them up to
    the gauge (a common phase and a common delay per correlation, fixed by antenna 0)."""
    rng = np.random.default_rng(17)
    n_ant, n_time, n_chan = 6, 2, 16
    p, q = synth.baselines(n_ant)
    ant1, ant2 = np.tile(p, n_time), np.tile(q, n_time)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    nu = np.linspace(0.9, 1.7, n_chan)
    shp = (ant1.size, n_chan, 4)
    model = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    truth = np.zeros((n_time, 1, n_ant, 4))
    truth[..., 0::2] = rng.uniform(-0.8, 0.8, size=(n_time, 1, n_ant, 2))
    truth[..., 1::2] = rng.uniform(-0.15, 0.15, size=(n_time, 1, n_ant, 2))
    true_term = O.OracleTerm("delay", np.arange(n_time, dtype=np.int32), np.zeros(n_chan, np.int32), n_time, 1,
                             n_ant, params=truth, chan_freq=nu)
    zero = np.zeros(shp, dtype=np.complex128)
    prob0 = O.OracleProblem(zero, model, np.ones(shp), np.zeros(shp[:2], np.uint8), ant1, ant2, tidx, n_ant, n_time)
    data = -_residual(prob0, [true_term])                  # D = C_p M C_q^H (written out here)
    prob = O.OracleProblem(data, model, np.ones(shp), np.zeros(shp[:2], np.uint8), ant1, ant2, tidx, n_ant, n_time)
    K = O.OracleTerm("delay", np.arange(n_time, dtype=np.int32), np.zeros(n_chan, np.int32), n_time, 1, n_ant,
                     chan_freq=nu, max_iter=50, tol=1e-12)
    iters = O.solve(prob, [K])[0]
    assert np.all(iters < 50)
    got = K.params - K.params[:, :, :1, :]
    want = truth - truth[:, :, :1, :]
    got[..., 0::2] = np.angle(np.exp(1j * got[..., 0::2]))
    want[..., 0::2] = np.angle(np.exp(1j * want[..., 0::2]))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)
    assert O.residual(prob, [K]) <= 1e-18 * np.sum(np.abs(data) ** 2)


def test_delay_jhr_is_minus_chi2_gradient():
    prob, nu, rng = _problem(23)
    terms = [_term("full", prob, nu, rng), _term("delay", prob, nu, rng)]
    _, jhr = O.normal_equations(prob, terms, 1)
    T = terms[1]
    h = 1e-6
    chi0 = O.residual(prob, terms)
    # a central difference of chi^2 carries a rounding error of order eps * chi^2 / h
    fd_noise = 10 * np.finfo(float).eps * chi0 / h
    for a in range(prob.n_ant):
        for k in range(4):
            base = T.params[0, 0, a, k]
            T.params[0, 0, a, k] = base + h
            cp = O.residual(prob, terms)
            T.params[0, 0, a, k] = base - h
            cm = O.residual(prob, terms)
            T.params[0, 0, a, k] = base
            grad = (cp - cm) / (2 * h)
            assert abs(jhr[0, 0, a, k].real + grad) <= 1e-6 * max(1.0, abs(grad)) + fd_noise


def test_one_frequency_makes_the_block_singular():
    """With every channel at the same frequency the phase and delay columns are proportional:
    the 4x4 block is singular, the gain flag is set and the parameters stay as they were."""
    prob, _, rng = _problem(29, n_chan=4)
    nu = np.full(4, 1.3)
    K = _term("delay", prob, nu, rng)
    before = K.params.copy()
    jhj, _ = O.normal_equations(prob, [K], 0)
    for a in range(prob.n_ant):
        B = jhj[0, 0, a].real
        np.testing.assert_allclose(B[1], 2 * np.pi * 1.3 * B[0], rtol=1e-12, atol=1e-12 * np.abs(B).max())
    O.solve_term(prob, [K], 0)
    assert np.all(K.gain_flags == 1)
    np.testing.assert_array_equal(K.params, before)
