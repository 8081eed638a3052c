"""Pins of the direction-dependent oracle (oracle/dd.py; Eq. baselinemodel with N_D directions,
Eq. g_derivative_dd / Eq. g_derivative_di).

- With one direction it reproduces the one-direction C oracle (itself pinned in
  test_oracle_pins.py), for diagonal and full terms at every chain position.
- With two directions its normal-equation blocks equal central Wirtinger differences of the
  residual, for a direction-dependent and for a direction-independent solved term in chains
  mixing both kinds.
- Noise-free data from known direction-dependent gains: the solve recovers them up to each
  direction's gauge, and chi^2 vanishes.
"""
import numpy as np
import pytest

import oracle as O
from oracle import dd
from paper_2412_10072_gb300 import synth


def _problem(seed, n_ant=3, n_time=2, n_chan=2, n_dir=2, flag_frac=0.15):
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(n_ant)
    a1, a2 = np.tile(p, n_time).astype(np.int32), np.tile(q, n_time).astype(np.int32)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    shp = (a1.size, n_chan)
    data = rng.standard_normal(shp + (4,)) + 1j * rng.standard_normal(shp + (4,))
    model = rng.standard_normal(shp + (n_dir, 4)) + 1j * rng.standard_normal(shp + (n_dir, 4))
    weight = rng.uniform(0.5, 2.0, shp + (4,))
    flag = (rng.random(shp) < flag_frac).astype(np.uint8)
    return dd.DDProblem(data, model, weight, flag, a1, a2, tidx, n_ant), rng


def _term(rng, kind, is_dd, n_ant, n_time, n_chan, n_dir, nt=1, nf=1):
    nd = n_dir if is_dd else 1
    par = np.eye(2).reshape(4) + 0.3 * (rng.standard_normal((nt, nf, n_ant, nd, 4)) +
                                        1j * rng.standard_normal((nt, nf, n_ant, nd, 4)))
    if kind == "diag":
        par[..., 1] = par[..., 2] = 0
    tm = (np.arange(n_time) * nt // n_time).astype(np.int32)
    fm = (np.arange(n_chan) * nf // n_chan).astype(np.int32)
    return dd.DDTerm(kind, is_dd, tm, fm, par)


@pytest.mark.parametrize("kinds,n", [(("diag",), 0), (("full",), 0), (("diag", "full"), 0), (("diag", "full"), 1),
                                     (("full", "diag", "full"), 1)])
def test_one_direction_reproduces_the_c_oracle(kinds, n):
    P, rng = _problem(1, n_dir=1)
    terms = [_term(rng, k, True, P.n_ant, 2, 2, 1, nt=2) for k in kinds]
    jhj, jhr = dd.normal_equations(P, terms, n)
    CP = O.OracleProblem(P.data, P.model[:, :, 0], P.weight, P.flag, P.ant1, P.ant2, P.time_idx, P.n_ant, 2)
    ct = [O.OracleTerm(T.kind, T.t_map, T.f_map, T.params.shape[0], T.params.shape[1], P.n_ant,
                       params=T.params[:, :, :, 0].copy()) for T in terms]
    cj, cr = O.normal_equations(CP, ct, n)
    np.testing.assert_allclose(jhj[:, :, :, 0], cj, rtol=1e-12, atol=1e-12 * np.abs(cj).max())
    np.testing.assert_allclose(jhr[:, :, :, 0], cr, rtol=1e-12, atol=1e-12 * np.abs(cr).max())
    chi_dd, _ = dd.residual(P, terms)
    assert abs(chi_dd - O.residual(CP, ct)) <= 1e-12 * chi_dd


def _fd_blocks(P, terms, n, h=1e-6):
    """Wirtinger finite differences of the stacked residual for every (interval, antenna, block)."""
    T = terms[n]
    w = P.weight.copy()
    w[P.flag.astype(bool)] = 0
    w = w.reshape(-1)
    r0 = dd.residual(P, terms)[1].reshape(-1)
    nt, nf = T.params.shape[:2]
    nblk = T.params.shape[3]
    free = T.free
    out_j = np.zeros((nt, nf, P.n_ant, nblk, len(free), len(free)), dtype=np.complex128)
    out_r = np.zeros((nt, nf, P.n_ant, nblk, len(free)), dtype=np.complex128)
    for ti in range(nt):
        for fi in range(nf):
            for a in range(P.n_ant):
                for k in range(nblk):
                    Jul, Jll = [], []
                    for e in free:
                        base = T.params[ti, fi, a, k, e]
                        dv = []
                        for step in (h, 1j * h):
                            T.params[ti, fi, a, k, e] = base + step
                            rp = dd.residual(P, terms)[1].reshape(-1)
                            T.params[ti, fi, a, k, e] = base - step
                            rm = dd.residual(P, terms)[1].reshape(-1)
                            T.params[ti, fi, a, k, e] = base
                            dv.append((rp - rm) / (2 * h))
                        dx, dy = dv
                        Jul.append(0.5 * (dx - 1j * dy))
                        Jll.append(np.conj(0.5 * (dx + 1j * dy)))
                    Jul, Jll = np.stack(Jul, 1), np.stack(Jll, 1)
                    out_j[ti, fi, a, k] = Jul.conj().T @ (w[:, None] * Jul) + Jll.conj().T @ (w[:, None] * Jll)
                    out_r[ti, fi, a, k] = -(Jul.conj().T @ (w * r0) + Jll.conj().T @ (w * np.conj(r0)))
    return out_j, out_r


@pytest.mark.parametrize("solved_dd", [True, False])
@pytest.mark.parametrize("kinds,dds,n", [(("diag",), (None,), 0), (("full", "diag"), (False, None), 1),
                                         (("diag", "full"), (None, True), 0)])
def test_two_directions_match_finite_differences(solved_dd, kinds, dds, n):
    P, rng = _problem(3 + int(solved_dd))
    terms = [_term(rng, k, solved_dd if f is None else f, P.n_ant, 2, 2, 2) for k, f in zip(kinds, dds)]
    jhj, jhr = dd.normal_equations(P, terms, n)
    fj, fr = _fd_blocks(P, terms, n)
    assert np.abs(jhj - fj).max() <= 1e-7 * np.abs(fj).max()
    assert np.abs(jhr - fr).max() <= 1e-7 * np.abs(fr).max()


def test_direction_dependent_gains_are_recovered():
    P, rng = _problem(7, n_ant=5, n_time=2, n_chan=3, flag_frac=0.0)
    truth = _term(rng, "diag", True, P.n_ant, 2, 3, 2)
    V = np.zeros_like(P.data)
    for row in range(P.data.shape[0]):
        for c in range(P.data.shape[1]):
            V[row, c] = dd.model_vis(P, [truth], row, c).reshape(4)
    P.data = V
    start = dd.DDTerm("diag", True, truth.t_map, truth.f_map, truth.params.copy(), max_iter=60, tol=1e-12)
    start.params[..., [0, 3]] *= np.exp(0.2j) * 1.1
    dd.solve_term(P, [start], 0)
    chi, _ = dd.residual(P, [start])
    assert chi <= 1e-20 * float(np.sum(np.abs(V) ** 2))
    got = start.params[0, 0][:, :, [0, 3]]
    want = truth.params[0, 0][:, :, [0, 3]]
    ref = lambda g: g * np.conj(g[:1]) / np.abs(g[:1])         # each direction's phase gauge
    np.testing.assert_allclose(ref(got), ref(want), rtol=0, atol=1e-8)


# ---------------------------------------------------------------------------
# the delay kind (Scenario 2) in chains with directions
# ---------------------------------------------------------------------------

def _delay_term(rng, n_time, n_chan, n_ant, nt=1, nf=1, scale=1.0):
    """K: (phi_X, tau_X, phi_Y, tau_Y) per interval and antenna; frequencies in GHz, delays in ns."""
    par = scale * np.stack([rng.uniform(-1, 1, (nt, nf, n_ant)), rng.uniform(-0.5, 0.5, (nt, nf, n_ant)),
                            rng.uniform(-1, 1, (nt, nf, n_ant)), rng.uniform(-0.5, 0.5, (nt, nf, n_ant))], -1)
    tm = (np.arange(n_time) * nt // n_time).astype(np.int32)
    fm = (np.arange(n_chan) * nf // n_chan).astype(np.int32)
    freq = np.linspace(1.0, 1.4, n_chan)
    return dd.DDTerm("delay", False, tm, fm, par[:, :, :, None, :].copy(), chan_freq=freq)


def _c_terms(terms, n_ant):
    out = []
    for T in terms:
        nt, nf = T.params.shape[:2]
        par = T.params[:, :, :, 0].copy()
        out.append(O.OracleTerm(T.kind, T.t_map, T.f_map, nt, nf, n_ant, params=par,
                                chan_freq=T.chan_freq if T.kind == "delay" else None))
    return out


@pytest.mark.parametrize("kinds,n", [(("delay",), 0), (("delay", "diag"), 0), (("delay", "diag"), 1),
                                     (("full", "delay"), 1)])
def test_delay_with_one_direction_reproduces_the_c_oracle(kinds, n):
    """Normal equations, chi^2 and the whole Algorithm 1 solve of a delay term, and of a term
    beside it, equal the one-direction C oracle (itself pinned by finite differences)."""
    P, rng = _problem(9, n_chan=4, n_dir=1)
    terms = []
    for k in kinds:
        terms.append(_delay_term(rng, 2, 4, P.n_ant, nt=2) if k == "delay" else
                     _term(rng, k, False, P.n_ant, 2, 4, 1, nt=2))
    jhj, jhr = dd.normal_equations(P, terms, n)
    CP = O.OracleProblem(P.data, P.model[:, :, 0], P.weight, P.flag, P.ant1, P.ant2, P.time_idx, P.n_ant, 2)
    ct = _c_terms(terms, P.n_ant)
    cj, cr = O.normal_equations(CP, ct, n)
    np.testing.assert_allclose(jhj[:, :, :, 0], cj, rtol=1e-12, atol=1e-12 * np.abs(cj).max())
    np.testing.assert_allclose(jhr[:, :, :, 0], cr, rtol=1e-12, atol=1e-12 * np.abs(cr).max())
    assert abs(dd.residual(P, terms)[0] - O.residual(CP, ct)) <= 1e-12 * O.residual(CP, ct)
    terms[n].max_iter, terms[n].tol = 6, 1e-9
    ct[n].max_iter, ct[n].tol = 6, 1e-9
    it_dd = dd.solve_term(P, terms, n, damping_mode=1)
    it_c = O.solve_term(CP, ct, n, damping_mode=1)
    np.testing.assert_array_equal(it_dd, it_c)
    np.testing.assert_allclose(terms[n].params[:, :, :, 0], ct[n].params, rtol=0, atol=1e-9)


@pytest.mark.parametrize("kinds,dds,n", [(("delay", "diag"), (False, True), 0), (("delay", "full"), (False, True), 0)])
def test_delay_blocks_with_two_directions_match_finite_differences(kinds, dds, n):
    """With two directions and a direction-dependent term to its right, the delay term's real
    4x4 block is 2 Re(J^H W J) and its right-hand side 2 Re(J^H W r), J = dv/du by central
    differences in the four real parameters (Eq. jhj_case2, Eq. jhwr_case2)."""
    P, rng = _problem(12, n_chan=4)
    terms = [_delay_term(rng, 2, 4, P.n_ant), _term(rng, kinds[1], True, P.n_ant, 2, 4, 2)]
    jhj, jhr = dd.normal_equations(P, terms, n)
    T = terms[n]
    w = P.weight.copy()
    w[P.flag.astype(bool)] = 0
    w = w.reshape(-1)
    r0 = dd.residual(P, terms)[1].reshape(-1)
    h = 1e-6
    for a in range(P.n_ant):
        J = []
        for e in range(4):
            base = T.params[0, 0, a, 0, e]
            T.params[0, 0, a, 0, e] = base + h
            rp = dd.residual(P, terms)[1].reshape(-1)
            T.params[0, 0, a, 0, e] = base - h
            rm = dd.residual(P, terms)[1].reshape(-1)
            T.params[0, 0, a, 0, e] = base
            J.append(-(rp - rm) / (2 * h))                    # dv/du = -dr/du
        J = np.stack(J, 1)
        fj = 2 * (J.conj().T @ (w[:, None] * J)).real
        fr = 2 * (J.conj().T @ (w * r0)).real
        assert np.abs(jhj[0, 0, a, 0] - fj).max() <= 1e-6 * np.abs(fj).max()
        assert np.abs(jhr[0, 0, a, 0] - fr).max() <= 1e-6 * max(np.abs(fr).max(), 1e-30)
