"""Direction-dependent chains on the GPU against the direction-dependent oracle (oracle/dd.py).

Eq. baselinemodel with N_D directions: V_pq = sum_d C_{p,d} M_{pq,d} C_{q,d}^H, each chain term
direction-dependent (blocks per (interval, antenna, direction), Eq. g_derivative_dd) or
direction-independent (the derivative summed over directions, Eq. g_derivative_di).

- One Gauss-Newton step, element by element, for direction-dependent and direction-independent
  solved terms, diagonal and full, alone and in two-term chains, with flags, random weights,
  ragged channel counts and intervals that straddle the 32-channel tiles.
- The residual and chi^2 element by element.
- Converged solves: gains within 1e-4 after referencing, chi^2 within 1e-5.
- What the path rejects.
"""
import numpy as np
import pytest

from oracle import dd
from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu

GAIN_TOL = 1e-4
CHI2_TOL = 1e-5


def _problem(seed, n_ant=5, n_time=4, n_chan=45, n_dir=2, flag_frac=0.15, noise=0.0, terms=None):
    """Random polarised model per direction; data from the given terms (or random) plus noise."""
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(n_ant)
    swap = rng.random(p.size) < 0.3
    p, q = np.where(swap, q, p), np.where(swap, p, q)
    a1, a2 = np.tile(p, n_time).astype(np.int32), np.tile(q, n_time).astype(np.int32)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    shp = (a1.size, n_chan)
    model = rng.standard_normal(shp + (n_dir, 4)) + 1j * rng.standard_normal(shp + (n_dir, 4))
    data = rng.standard_normal(shp + (4,)) + 1j * rng.standard_normal(shp + (4,))
    weight = rng.uniform(0.5, 2.0, shp + (4,))
    flag = (rng.random(shp) < flag_frac).astype(np.uint8)
    P = dd.DDProblem(data, model, weight, flag, a1, a2, tidx, n_ant)
    if terms is not None:
        clean = np.zeros_like(data)
        for r in range(a1.size):
            for c in range(n_chan):
                clean[r, c] = dd.model_vis(P, terms, r, c).reshape(4)
        P.data = clean + noise * (rng.standard_normal(data.shape) + 1j * rng.standard_normal(data.shape))
    return P, rng


def _params(rng, kind, is_dd, n_ant, n_dir, nt, nf, spread=0.3):
    nd = n_dir if is_dd else 1
    par = np.eye(2).reshape(4) + spread * (rng.standard_normal((nt, nf, n_ant, nd, 4)) +
                                           1j * rng.standard_normal((nt, nf, n_ant, nd, 4)))
    if kind == "diag":
        par[..., 1] = par[..., 2] = 0
    return par


def _maps(n_time, n_chan, nt, nf):
    return (np.arange(n_time) * nt // n_time).astype(np.int32), (np.arange(n_chan) * nf // n_chan).astype(np.int32)


def _oterm(kind, is_dd, tm, fm, par, solve, max_iter=1, tol=0.0):
    return dd.DDTerm(kind, is_dd, tm, fm, par.copy(), solve=solve, max_iter=max_iter, tol=tol)


def _gterm(kind, is_dd, tm, fm, par, n_ant, n_dir, solve, max_iter=1, tol=0.0):
    nt, nf = par.shape[:2]
    g = par if (is_dd and n_dir > 1) else par[:, :, :, 0]
    return qc.Term(kind, tm, fm, nt, nf, n_ant, gains=g.astype(np.complex64), solve=solve, max_iter=max_iter,
                   tol=tol, dd=is_dd, n_dir=n_dir)


def _solver(P):
    return qc.Solver(P.data.astype(np.complex64), P.model.astype(np.complex64), P.weight.astype(np.float32),
                     P.flag, P.ant1, P.ant2, P.time_idx, P.n_ant, int(P.time_idx.max()) + 1)


def _gpu_params(t, n_dir):
    g = np.asarray(t.gains, dtype=np.complex128)
    return g if g.ndim == 5 else g[:, :, :, None, :]


# chains: (kind, direction-dependent, n_tint, n_fint) per term, leftmost first
CHAINS = [
    [("full", True, 2, 3)],
    [("diag", True, 4, 7)],
    [("diag", False, 2, 45), ("full", True, 1, 3)],
    [("full", False, 4, 1), ("diag", True, 2, 9)],
    [("diag", True, 1, 5), ("full", True, 2, 2)],
    [("full", False, 2, 1), ("diag", True, 2, 5), ("diag", False, 1, 45)],   # three terms: general kernel
]


# n_dir 2 and 3: the streaming kernel (chains of one or two terms, at most 4 directions; a
# diagonal direction-dependent solved term forms two directions per CTA, so 3 leaves one CTA
# row with a single direction); 5: the general kernel.  kernel 2 forces the general kernel.
@pytest.mark.parametrize("chain", CHAINS)
@pytest.mark.parametrize("n_dir,kernel", [(2, 0), (3, 0), (4, 0), (5, 0), (2, 2)])
def test_single_step_matches_oracle(chain, n_dir, kernel):
    n_ant, n_time, n_chan = 5, 4, 45
    P, rng = _problem(3 + n_dir, n_ant=n_ant, n_time=n_time, n_chan=n_chan, n_dir=n_dir)
    pars = [_params(rng, k, isdd, n_ant, n_dir, nt, nf) for (k, isdd, nt, nf) in chain]
    maps = [_maps(n_time, n_chan, nt, nf) for (_, _, nt, nf) in chain]
    pars32 = [p.astype(np.complex64).astype(np.complex128) for p in pars]
    for n in range(len(chain)):
        if n > 0 and not chain[n][1] and any(c[1] for c in chain[:n]):
            continue                      # a direction-independent term right of a direction-dependent one
        ot = [_oterm(k, isdd, tm, fm, p, i == n) for i, ((k, isdd, _, _), (tm, fm), p) in enumerate(zip(chain, maps, pars32))]
        dd.solve_term(P, ot, n, damping_mode=0)
        S = _solver(P)
        gt = [_gterm(k, isdd, tm, fm, p, n_ant, n_dir, i == n)
              for i, ((k, isdd, _, _), (tm, fm), p) in enumerate(zip(chain, maps, pars32))]
        S.solve(gt, damping_mode=qc.QC_DAMP_CONST, damping=1.0, kernel=kernel)
        S.close()
        want = ot[n].params
        got = _gpu_params(gt[n], n_dir)
        step = want - pars32[n]
        err = np.max(np.abs(got - want)) / max(np.max(np.abs(step)), 1e-30)
        assert err < 2e-3, (chain, n, err)


@pytest.mark.parametrize("n_dir", [1, 2, 4])
def test_residual_and_chi2_match_oracle(n_dir):
    n_ant, n_time, n_chan = 5, 3, 40
    P, rng = _problem(11, n_ant=n_ant, n_time=n_time, n_chan=n_chan, n_dir=n_dir)
    chain = [("full", False, 3, 1), ("diag", True, 1, 4)]
    pars = [_params(rng, k, isdd, n_ant, n_dir, nt, nf) for (k, isdd, nt, nf) in chain]
    maps = [_maps(n_time, n_chan, nt, nf) for (_, _, nt, nf) in chain]
    ot = [_oterm(k, isdd, tm, fm, p, False) for (k, isdd, _, _), (tm, fm), p in zip(chain, maps, pars)]
    ochi2, ores = dd.residual(P, ot)
    S = _solver(P)
    gt = [_gterm(k, isdd, tm, fm, p, n_ant, n_dir, False) for (k, isdd, _, _), (tm, fm), p in zip(chain, maps, pars)]
    gchi2, gres = S.residual(gt, want_resid=True)
    S.close()
    scale = np.max(np.abs(P.data))
    assert np.max(np.abs(gres - ores)) < 2e-5 * scale
    assert abs(gchi2 - ochi2) <= CHI2_TOL * ochi2


def _ref_dd(g):
    """Per-direction reference of diagonal gains [..][n_ant][nd][4] to antenna 0 (Eq. update is
    invariant under g_{a,d} -> g_{a,d} u_d with |u_d| = 1 per direction and correlation)."""
    g = np.asarray(g, dtype=np.complex128)
    out = g.copy()
    for k in (0, 3):
        g0 = g[:, :, 0:1, :, k]
        out[..., k] = g[..., k] * np.conj(g0) / np.abs(g0)
    return out


@pytest.mark.parametrize("n_dir", [2, 3])
def test_converged_direction_dependent_gains_match_oracle(n_dir):
    """Noise-free data from known gains of a chain G (direction-independent, full) x dE
    (direction-dependent, diagonal); G held at its truth, dE solved from a perturbed start."""
    n_ant, n_time, n_chan = 5, 2, 24
    rng = np.random.default_rng(21)
    chain = [("full", False, 2, 1), ("diag", True, 1, 4)]
    maps = [_maps(n_time, n_chan, nt, nf) for (_, _, nt, nf) in chain]
    truth = [_params(rng, k, isdd, n_ant, n_dir, nt, nf, spread=0.2) for (k, isdd, nt, nf) in chain]
    tterms = [_oterm(k, isdd, tm, fm, p, False) for (k, isdd, _, _), (tm, fm), p in zip(chain, maps, truth)]
    P, _ = _problem(22, n_ant=n_ant, n_time=n_time, n_chan=n_chan, n_dir=n_dir, terms=tterms, noise=0.01,
                    flag_frac=0.05)
    start = truth[1] + 0.05 * (rng.standard_normal(truth[1].shape) + 1j * rng.standard_normal(truth[1].shape))
    start[..., 1] = start[..., 2] = 0
    start32 = start.astype(np.complex64).astype(np.complex128)
    ot = [_oterm("full", False, *maps[0], truth[0], False),
          _oterm("diag", True, *maps[1], start32, True, max_iter=30, tol=1e-7)]
    dd.solve_term(P, ot, 1, damping_mode=1)
    ochi2, _ = dd.residual(P, ot)
    S = _solver(P)
    gt = [_gterm("full", False, *maps[0], truth[0], n_ant, n_dir, False),
          _gterm("diag", True, *maps[1], start32, n_ant, n_dir, True, max_iter=30, tol=1e-7)]
    S.solve(gt)
    gchi2 = S.residual(gt)
    S.close()
    got, want = _ref_dd(_gpu_params(gt[1], n_dir)), _ref_dd(ot[1].params)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < GAIN_TOL, err
    assert abs(gchi2 - ochi2) <= CHI2_TOL * ochi2
    assert gt[1].gain_flags.shape == (1, 4, n_ant, n_dir) and np.all(gt[1].gain_flags == 0)


def _delay(rng, n_ant, n_time, n_chan, nt=1, spread=1.0):
    par = spread * np.stack([rng.uniform(-1, 1, (nt, 1, n_ant)), rng.uniform(-0.5, 0.5, (nt, 1, n_ant)),
                             rng.uniform(-1, 1, (nt, 1, n_ant)), rng.uniform(-0.5, 0.5, (nt, 1, n_ant))], -1)
    tm, fm = _maps(n_time, n_chan, nt, 1)
    return par[:, :, :, None, :], tm, fm, np.linspace(1.0, 1.4, n_chan)


def _ok_delay(par, tm, fm, freq, solve, max_iter=1, tol=0.0):
    return dd.DDTerm("delay", False, tm, fm, par.copy(), solve=solve, max_iter=max_iter, tol=tol, chan_freq=freq)


def _gk_delay(par, tm, fm, freq, n_ant, solve, max_iter=1, tol=0.0):
    nt, nf = par.shape[:2]
    return qc.Term("delay", tm, fm, nt, nf, n_ant, gains=par[:, :, :, 0].astype(np.float32), solve=solve,
                   max_iter=max_iter, tol=tol, chan_freq=freq)


@pytest.mark.parametrize("n", [0, 1])
@pytest.mark.parametrize("dekind", ["diag", "full"])
@pytest.mark.parametrize("kernel", [0, 2])
def test_k_de_single_step_matches_oracle(n, dekind, kernel):
    """The KdE chain: K (delay and phase per integration over every channel, direction-independent)
    and dE (direction-dependent, over several channels), two directions; one step of either term."""
    n_ant, n_time, n_chan, n_dir = 5, 4, 40, 2
    P, rng = _problem(31, n_ant=n_ant, n_time=n_time, n_chan=n_chan, n_dir=n_dir)
    kpar, ktm, kfm, freq = _delay(rng, n_ant, n_time, n_chan, nt=n_time)
    kpar = kpar.astype(np.float32).astype(np.float64)
    de = _params(rng, dekind, True, n_ant, n_dir, 2, 5).astype(np.complex64).astype(np.complex128)
    dtm, dfm = _maps(n_time, n_chan, 2, 5)
    ot = [_ok_delay(kpar, ktm, kfm, freq, n == 0), _oterm(dekind, True, dtm, dfm, de, n == 1)]
    dd.solve_term(P, ot, n, damping_mode=0)
    S = _solver(P)
    gt = [_gk_delay(kpar, ktm, kfm, freq, n_ant, n == 0), _gterm(dekind, True, dtm, dfm, de, n_ant, n_dir, n == 1)]
    S.solve(gt, damping_mode=qc.QC_DAMP_CONST, damping=1.0, kernel=kernel)
    S.close()
    if n == 0:
        want, start = ot[0].params[:, :, :, 0], kpar[:, :, :, 0]
        got = np.asarray(gt[0].gains, dtype=np.float64)
    else:
        want, start, got = ot[1].params, de, _gpu_params(gt[1], n_dir)
    err = np.max(np.abs(got - want)) / max(np.max(np.abs(want - start)), 1e-30)
    assert err < 2e-3, (n, err)


def test_k_de_converged_matches_oracle():
    """Noise-free KdE data; two epochs of K then dE from perturbed starts: chi^2 within 1e-5 and
    K's delays and dE's referenced gains within 1e-4 of the oracle's."""
    n_ant, n_time, n_chan, n_dir = 5, 2, 24, 2
    rng = np.random.default_rng(41)
    kpar, ktm, kfm, freq = _delay(rng, n_ant, n_time, n_chan, nt=n_time, spread=0.5)
    de = _params(rng, "diag", True, n_ant, n_dir, 1, 2, spread=0.2)
    dtm, dfm = _maps(n_time, n_chan, 1, 2)
    truth = [_ok_delay(kpar, ktm, kfm, freq, False), _oterm("diag", True, dtm, dfm, de, False)]
    P, _ = _problem(42, n_ant=n_ant, n_time=n_time, n_chan=n_chan, n_dir=n_dir, terms=truth, noise=0.0,
                    flag_frac=0.05)
    k0 = (kpar + 0.05 * rng.standard_normal(kpar.shape)).astype(np.float32).astype(np.float64)
    d0 = de * (1 + 0.05 * rng.standard_normal(de.shape))
    d0[..., 1] = d0[..., 2] = 0
    d0 = d0.astype(np.complex64).astype(np.complex128)
    ot = [_ok_delay(k0, ktm, kfm, freq, True, max_iter=20, tol=1e-7),
          _oterm("diag", True, dtm, dfm, d0, True, max_iter=20, tol=1e-7)]
    for _ in range(2):
        dd.solve_term(P, ot, 0, damping_mode=1)
        dd.solve_term(P, ot, 1, damping_mode=1)
    ochi2, _ = dd.residual(P, ot)
    S = _solver(P)
    gt = [_gk_delay(k0, ktm, kfm, freq, n_ant, True, max_iter=20, tol=1e-7),
          _gterm("diag", True, dtm, dfm, d0, n_ant, n_dir, True, max_iter=20, tol=1e-7)]
    S.solve(gt, n_epochs=2)
    gchi2 = S.residual(gt)
    S.close()
    scale = float(np.sum(P.weight * np.abs(P.data) ** 2))
    assert abs(gchi2 - ochi2) <= max(CHI2_TOL * ochi2, 1e-9 * scale), (gchi2, ochi2)
    kerr = np.max(np.abs(np.asarray(gt[0].gains, np.float64)[..., [1, 3]] - ot[0].params[:, :, :, 0][..., [1, 3]]))
    assert kerr < 1e-3, kerr                         # delays (ns), whose scale is ~0.5
    got, want = _ref_dd(_gpu_params(gt[1], n_dir)), _ref_dd(ot[1].params)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < GAIN_TOL


def test_one_direction_flagged_dd_equals_plain():
    """With n_dir = 1 a term marked direction-dependent is the plain term."""
    obs = synth.plain_small(seed=2, noise=0.01, n_time=8, n_chan=16)
    outs = []
    for isdd in (False, True):
        S = qc.Solver.from_obs(obs)
        t = qc.Term.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6, dd=isdd, n_dir=1)
        S.solve([t])
        S.close()
        outs.append(np.asarray(t.gains))
    assert np.array_equal(outs[0], outs[1])


def test_rejections():
    n_ant, n_time, n_chan, n_dir = 4, 2, 8, 2
    P, rng = _problem(5, n_ant=n_ant, n_time=n_time, n_chan=n_chan, n_dir=n_dir)
    S = _solver(P)
    tm, fm = _maps(n_time, n_chan, 1, 1)
    ph = qc.Term("phase", tm, fm, 1, 1, n_ant)
    with pytest.raises(qc.QCError) as e:
        S.solve([ph])
    assert e.value.code == qc.QC_EUNSUPPORTED
    kdd = qc.Term("delay", tm, fm, 1, 1, n_ant, chan_freq=np.linspace(1, 1.4, n_chan), dd=True, n_dir=n_dir)
    with pytest.raises(qc.QCError) as e:
        S.solve([kdd])
    assert e.value.code == qc.QC_EUNSUPPORTED
    # a solved direction-independent term to the right of a direction-dependent one
    left = _gterm("diag", True, tm, fm, _params(rng, "diag", True, n_ant, n_dir, 1, 1), n_ant, n_dir, False)
    right = _gterm("diag", False, tm, fm, _params(rng, "diag", False, n_ant, n_dir, 1, 1), n_ant, n_dir, True)
    with pytest.raises(qc.QCError) as e:
        S.solve([left, right])
    assert e.value.code == qc.QC_EUNSUPPORTED
    with pytest.raises(qc.QCError) as e:
        S.mad_flag([_gterm("diag", True, tm, fm, _params(rng, "diag", True, n_ant, n_dir, 1, 1), n_ant, n_dir, False)])
    assert e.value.code == qc.QC_EUNSUPPORTED
    S.close()
    with pytest.raises(qc.QCError) as e:
        qc.Solver(P.data.astype(np.complex64), P.model.astype(np.complex64), P.weight.astype(np.float32), P.flag,
                  P.ant1, P.ant2, P.time_idx, n_ant, n_time, model_fp16=True)
    assert e.value.code == qc.QC_EINVAL
