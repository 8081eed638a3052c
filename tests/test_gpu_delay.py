"""Parity of the delay term (QC_TERM_DELAY, Scenario 2) through the C ABI with the FP64 oracle.

Seeded synthetic problems: 7 antennas, 6 times, 48 channels (one full and one ragged
32-channel chunk) at 0.9-1.7 GHz, delays in ns, 10% of samples flagged, noise 0.05.
Gains are compared at every channel, referenced to antenna 0 (a common phase and delay
per correlation is not determined by the data), within 1e-4; chi^2 within 1e-5."""
import numpy as np
import pytest

import oracle as O
from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu

GAIN_TOL = 1e-4
CHI2_TOL = 1e-5
N_ANT, N_TIME, N_CHAN = 7, 6, 48
NU = np.linspace(0.9, 1.7, N_CHAN)


def _delay_gains(par, t_map, f_map, nu):
    """[n_time][n_chan][ant][2] diagonal gains of delay parameters [tint][fint][ant][4]."""
    u = par[t_map][:, f_map]                                   # [time][chan][ant][4]
    w = 2 * np.pi * nu[None, :, None]
    return np.stack([np.exp(1j * (u[..., 0] + u[..., 1] * w)), np.exp(1j * (u[..., 2] + u[..., 3] * w))], -1)


def _problem(seed, n_tint=3, n_fint=1, other=None, nu=NU):
    """Data D = C_p M C_q^H + noise for the chain [K] / [K, B] / [G, K] (other = None / "B" / "G")."""
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(N_ANT)
    ant1, ant2 = np.tile(p, N_TIME), np.tile(q, N_TIME)
    tidx = np.repeat(np.arange(N_TIME, dtype=np.int32), p.size)
    n_row = ant1.size
    shp = (n_row, N_CHAN, 4)
    model = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(2)
    weight = rng.uniform(0.5, 2.0, size=shp)
    flag = (rng.random(shp[:2]) < 0.1).astype(np.uint8)
    t_map = (np.arange(N_TIME) * n_tint // N_TIME).astype(np.int32)
    f_map = (np.arange(N_CHAN) * n_fint // N_CHAN).astype(np.int32)
    truth = np.zeros((n_tint, n_fint, N_ANT, 4))
    truth[..., 0::2] = rng.uniform(-1.0, 1.0, size=(n_tint, n_fint, N_ANT, 2))
    truth[..., 1::2] = rng.uniform(-0.1, 0.1, size=(n_tint, n_fint, N_ANT, 2))
    gk = _delay_gains(truth, t_map, f_map, nu)                 # [time][chan][ant][2]
    C = np.zeros((N_TIME, N_CHAN, N_ANT, 2, 2), dtype=np.complex128)
    C[..., 0, 0], C[..., 1, 1] = gk[..., 0], gk[..., 1]
    fixed = None
    if other == "B":
        gb = np.zeros((1, N_CHAN, N_ANT, 4), dtype=np.complex128)
        gb[..., 0] = 1 + 0.2 * (rng.standard_normal((1, N_CHAN, N_ANT)) + 1j * rng.standard_normal((1, N_CHAN, N_ANT)))
        gb[..., 3] = 1 + 0.2 * (rng.standard_normal((1, N_CHAN, N_ANT)) + 1j * rng.standard_normal((1, N_CHAN, N_ANT)))
        fixed = ("diag", np.zeros(N_TIME, np.int32), np.arange(N_CHAN, dtype=np.int32), 1, N_CHAN, gb)
        B = np.zeros((N_TIME, N_CHAN, N_ANT, 2, 2), dtype=np.complex128)
        B[..., 0, 0] = gb[0][None, :, :, 0]
        B[..., 1, 1] = gb[0][None, :, :, 3]
        C = C @ B
    elif other == "G":
        gg = np.eye(2).reshape(4) + 0.2 * (rng.standard_normal((N_TIME, 1, N_ANT, 4)) +
                                           1j * rng.standard_normal((N_TIME, 1, N_ANT, 4)))
        fixed = ("full", np.arange(N_TIME, dtype=np.int32), np.zeros(N_CHAN, np.int32), N_TIME, 1, gg)
        G = np.broadcast_to(gg.reshape(N_TIME, 1, N_ANT, 2, 2), (N_TIME, N_CHAN, N_ANT, 2, 2))
        C = G @ C
    Cp = C[tidx[:, None], np.arange(N_CHAN)[None, :], ant1[:, None]]      # [row][chan][2][2]
    Cq = C[tidx[:, None], np.arange(N_CHAN)[None, :], ant2[:, None]]
    M = model.reshape(n_row, N_CHAN, 2, 2)
    V = Cp @ M @ np.conj(np.swapaxes(Cq, -1, -2))
    data = V.reshape(shp) + 0.05 * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(2)
    return dict(data=data, model=model, weight=weight, flag=flag, ant1=ant1, ant2=ant2, tidx=tidx, t_map=t_map,
                f_map=f_map, n_tint=n_tint, n_fint=n_fint, fixed=fixed, other=other, nu=nu)


def _oracle_terms(pb, k_params=None, max_iter=30, tol=1e-8, solve_k=True, solve_fixed=False):
    K = O.OracleTerm("delay", pb["t_map"], pb["f_map"], pb["n_tint"], pb["n_fint"], N_ANT, params=k_params,
                     chan_freq=pb["nu"], max_iter=max_iter, tol=tol, solve=solve_k)
    if pb["fixed"] is None:
        return [K], 0
    kind, tm, fm, nt, nf, par = pb["fixed"]
    F = O.OracleTerm(kind, tm, fm, nt, nf, N_ANT, params=par, max_iter=max_iter, tol=tol, solve=solve_fixed)
    return ([K, F], 0) if pb["other"] == "B" else ([F, K], 1)


def _gpu_terms(pb, k_params=None, max_iter=30, tol=1e-8, solve_k=True, solve_fixed=False):
    K = qc.Term("delay", pb["t_map"], pb["f_map"], pb["n_tint"], pb["n_fint"], N_ANT,
                gains=None if k_params is None else k_params.astype(np.float32), chan_freq=pb["nu"],
                max_iter=max_iter, tol=tol, solve=solve_k)
    if pb["fixed"] is None:
        return [K], 0
    kind, tm, fm, nt, nf, par = pb["fixed"]
    F = qc.Term(kind, tm, fm, nt, nf, N_ANT, gains=par.astype(np.complex64), max_iter=max_iter, tol=tol,
                solve=solve_fixed)
    return ([K, F], 0) if pb["other"] == "B" else ([F, K], 1)


def _oracle_problem(pb):
    return O.OracleProblem(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"],
                           N_ANT, N_TIME)


def _solver(pb):
    return qc.Solver(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], N_ANT,
                     N_TIME)


def _referenced(par, pb):
    """Gains of delay parameters at every channel, referenced to antenna 0."""
    g = _delay_gains(np.asarray(par, dtype=np.float64), np.arange(pb["n_tint"]),
                     pb["f_map"], pb["nu"])                      # [tint][chan][ant][2]
    return g * np.conj(g[:, :, :1, :])


# kernel 0: the streaming delay kernel (chain rule per sample, sums per interval);
# kernel 2: the generic kernels on per-channel bins, reduced by the chain rule in the update
KERNELS = [0, 2]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("other", [None, "B", "G"])
def test_one_step_matches_oracle(other, kernel):
    """One Gauss-Newton step (alpha = 1) from zero gives the same step as the oracle's sums over
    every sample of the interval."""
    pb = _problem(101, other=other)
    P = _oracle_problem(pb)
    ot, n = _oracle_terms(pb, max_iter=1)
    O.solve_term(P, ot, n, damping=1.0, damping_mode=0)
    S = _solver(pb)
    gt, n = _gpu_terms(pb, max_iter=1)
    S.solve(gt, damping_mode=qc.QC_DAMP_CONST, damping=1.0, kernel=kernel)
    S.close()
    g_gpu = _delay_gains(np.asarray(gt[n].gains, np.float64), np.arange(pb["n_tint"]), pb["f_map"], pb["nu"])
    g_ora = _delay_gains(ot[n].params, np.arange(pb["n_tint"]), pb["f_map"], pb["nu"])
    assert np.abs(g_gpu - g_ora).max() <= GAIN_TOL
    assert np.array_equal(np.asarray(gt[n].gain_flags), ot[n].gain_flags)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("other,n_fint", [(None, 1), (None, 2), ("B", 1), ("G", 1)])
def test_converged_solution_matches_oracle(other, n_fint, kernel):
    pb = _problem(202 + n_fint, n_fint=n_fint, other=other)
    P = _oracle_problem(pb)
    ot, n = _oracle_terms(pb)
    its_o = O.solve(P, ot, damping_mode=1)[n]
    chi_o = O.residual(P, ot)
    S = _solver(pb)
    gt, n = _gpu_terms(pb)
    S.solve(gt, kernel=kernel)
    chi_g = S.residual(gt)
    S.close()
    a = _referenced(gt[n].gains, pb)
    b = _referenced(ot[n].params, pb)
    assert np.abs(a - b).max() <= GAIN_TOL
    assert abs(chi_g - chi_o) <= CHI2_TOL * chi_o
    assert np.all(np.asarray(gt[n].iters) >= 1) and np.all(its_o >= 1)


def test_residual_with_delay_term_matches_oracle():
    pb = _problem(303, other="G")
    rng = np.random.default_rng(5)
    par = np.zeros((pb["n_tint"], 1, N_ANT, 4))
    par[..., 0::2] = rng.uniform(-1, 1, par[..., 0::2].shape)
    par[..., 1::2] = rng.uniform(-0.1, 0.1, par[..., 1::2].shape)
    ot, _ = _oracle_terms(pb, k_params=par, solve_k=False)
    chi_o, r_o = O.residual(_oracle_problem(pb), ot, want_resid=True)
    S = _solver(pb)
    gt, _ = _gpu_terms(pb, k_params=par, solve_k=False)
    chi_g, r_g = S.residual(gt, want_resid=True)
    S.close()
    assert abs(chi_g - chi_o) <= CHI2_TOL * chi_o
    scale = np.abs(r_o).max()
    assert np.abs(r_g - r_o).max() <= 1e-4 * scale


def test_delay_term_held_fixed_while_another_is_solved():
    """[K, B] with K fixed at given parameters and B (per channel) solved."""
    pb = _problem(404, other="B")
    rng = np.random.default_rng(9)
    par = np.zeros((pb["n_tint"], 1, N_ANT, 4))
    par[..., 0::2] = rng.uniform(-1, 1, par[..., 0::2].shape)
    par[..., 1::2] = rng.uniform(-0.1, 0.1, par[..., 1::2].shape)
    _, _, _, _, _, gb = pb["fixed"]
    unit = np.zeros_like(gb)
    unit[..., 0] = unit[..., 3] = 1
    pb["fixed"] = pb["fixed"][:5] + (unit,)
    P = _oracle_problem(pb)
    ot, _ = _oracle_terms(pb, k_params=par, solve_k=False, solve_fixed=True)
    O.solve(P, ot, damping_mode=1)
    chi_o = O.residual(P, ot)
    S = _solver(pb)
    gt, _ = _gpu_terms(pb, k_params=par, solve_k=False, solve_fixed=True)
    S.solve(gt)
    chi_g = S.residual(gt)
    S.close()
    gb_o = ot[1].params[..., [0, 3]]
    gb_g = np.asarray(gt[1].gains, np.complex128)[..., [0, 3]]
    ref = lambda g: g * np.conj(g[:, :, :1, :]) / np.abs(g[:, :, :1, :])
    assert np.abs(ref(gb_g) - ref(gb_o)).max() <= GAIN_TOL * np.abs(gb_o).max()
    assert abs(chi_g - chi_o) <= CHI2_TOL * chi_o
    # the fixed delay term comes back unchanged
    np.testing.assert_array_equal(np.asarray(gt[0].gains), par.astype(np.float32))


@pytest.mark.parametrize("kernel", KERNELS)
def test_single_frequency_block_is_singular_and_left_unchanged(kernel):
    pb = _problem(505, nu=np.full(N_CHAN, 1.3))
    rng = np.random.default_rng(3)
    par = rng.uniform(-0.5, 0.5, size=(pb["n_tint"], 1, N_ANT, 4)).astype(np.float32)
    S = _solver(pb)
    gt, n = _gpu_terms(pb, k_params=par.astype(np.float64))
    S.solve(gt, kernel=kernel)
    S.close()
    assert np.all(np.asarray(gt[n].gain_flags) == 1)
    np.testing.assert_array_equal(np.asarray(gt[n].gains), par)


def test_delay_term_without_frequencies_is_rejected():
    pb = _problem(606)
    S = _solver(pb)
    gt, _ = _gpu_terms(pb)
    gt[0].chan_freq = None
    with pytest.raises(qc.QCError):
        S.solve(gt)
    bad = NU.copy()
    bad[3] = np.nan
    gt[0].chan_freq = bad
    with pytest.raises(qc.QCError):
        S.solve(gt)
    S.close()


# ---------------------------------------------------------------------------
# initial estimate (qc_delay_init) against the oracle's FFT-peak estimate
# ---------------------------------------------------------------------------

def _init_problem(seed, n_time=4, n_chan=48, noise=0.02, big=3.0):
    """Data of [K] with delays up to `big` ns (far outside a zero start's basin), 10% flagged."""
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(N_ANT)
    ant1, ant2 = np.tile(p, n_time), np.tile(q, n_time)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    shp = (ant1.size, n_chan, 4)
    nu = np.linspace(0.9, 1.7, n_chan)
    model = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(2)
    weight = rng.uniform(0.5, 2.0, size=shp)
    flag = (rng.random(shp[:2]) < 0.1).astype(np.uint8)
    truth = np.zeros((n_time, 1, N_ANT, 4))
    truth[..., 0::2] = rng.uniform(-2, 2, (n_time, 1, N_ANT, 2))
    truth[..., 1::2] = rng.uniform(-big, big, (n_time, 1, N_ANT, 2))
    g = _delay_gains(truth, np.arange(n_time), np.zeros(n_chan, np.int32), nu)     # [time][chan][ant][2]
    gp = g[tidx[:, None], np.arange(n_chan)[None, :], ant1[:, None]]
    gq = g[tidx[:, None], np.arange(n_chan)[None, :], ant2[:, None]]
    data = model.copy()
    data[..., 0] *= gp[..., 0] * np.conj(gq[..., 0])
    data[..., 1] *= gp[..., 0] * np.conj(gq[..., 1])
    data[..., 2] *= gp[..., 1] * np.conj(gq[..., 0])
    data[..., 3] *= gp[..., 1] * np.conj(gq[..., 1])
    data = data + noise * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    return dict(data=data, model=model, weight=weight, flag=flag, ant1=ant1, ant2=ant2, tidx=tidx, nu=nu,
                n_time=n_time, n_chan=n_chan)


@pytest.mark.parametrize("ref,n_fint,m16", [(0, 1, False), (3, 2, False), (0, 1, True)])
def test_delay_init_matches_oracle(ref, n_fint, m16):
    from oracle.delay_init import delay_init
    pb = _init_problem(707 + ref + n_fint)
    n_time, n_chan = pb["n_time"], pb["n_chan"]
    t_map = np.arange(n_time, dtype=np.int32)
    f_map = (np.arange(n_chan) * n_fint // n_chan).astype(np.int32)
    model = pb["model"]
    if m16:   # the oracle sees the model the GPU stores: FP16 (re, im) x per-baseline scale
        n_bl = N_ANT * (N_ANT - 1) // 2
        bl = np.tile(np.arange(n_bl), n_time)
        m = model.astype(np.complex64)
        comp = np.stack([m.real, m.imag], -1)
        scale = np.zeros(n_bl, np.float32)
        np.maximum.at(scale, bl, np.abs(comp).reshape(comp.shape[0], -1).max(1))
        scale[scale == 0] = 1
        h = (comp / scale[bl][:, None, None, None]).astype(np.float16).astype(np.float32) * scale[bl][:, None, None, None]
        model = h[..., 0] + 1j * h[..., 1]
    P = O.OracleProblem(pb["data"], model, pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], N_ANT, n_time)
    want = delay_init(P, t_map, f_map, n_time, n_fint, pb["nu"], ref=ref, oversample=4)
    S = qc.Solver(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], N_ANT,
                  n_time, model_fp16=m16)
    K = qc.Term("delay", t_map, f_map, n_time, n_fint, N_ANT, chan_freq=pb["nu"])
    S.delay_init(K, ref=ref, oversample=4)
    S.close()
    got = np.asarray(K.gains, np.float64)
    # the same peak bin: identical delays on the grid
    np.testing.assert_allclose(got[..., 1::2], want[..., 1::2], rtol=1e-6, atol=0)
    assert np.abs(np.angle(np.exp(1j * (got[..., 0::2] - want[..., 0::2])))).max() <= 1e-3
    assert np.all(got[:, :, ref] == 0)


def test_solve_from_the_estimate_matches_the_oracle():
    """Delays up to 3 ns: both sides start from their own estimate and reach the same solution."""
    from oracle.delay_init import delay_init
    pb = _init_problem(808)
    n_time, n_chan = pb["n_time"], pb["n_chan"]
    t_map, f_map = np.arange(n_time, dtype=np.int32), np.zeros(n_chan, np.int32)
    P = O.OracleProblem(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], N_ANT,
                        n_time)
    est = delay_init(P, t_map, f_map, n_time, 1, pb["nu"])
    ok = O.OracleTerm("delay", t_map, f_map, n_time, 1, N_ANT, params=est, chan_freq=pb["nu"], max_iter=40, tol=1e-8)
    O.solve(P, [ok], damping_mode=1)
    chi_o = O.residual(P, [ok])
    S = qc.Solver(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], N_ANT, n_time)
    K = qc.Term("delay", t_map, f_map, n_time, 1, N_ANT, chan_freq=pb["nu"], max_iter=40, tol=1e-8)
    S.delay_init(K)
    S.solve([K])
    chi_g = S.residual([K])
    S.close()
    pbk = dict(n_tint=n_time, f_map=f_map, nu=pb["nu"])
    assert np.abs(_referenced(K.gains, pbk) - _referenced(ok.params, pbk)).max() <= GAIN_TOL
    assert abs(chi_g - chi_o) <= CHI2_TOL * chi_o


def test_delay_init_rejects_bad_requests():
    pb = _init_problem(909)
    n_time, n_chan = pb["n_time"], pb["n_chan"]
    S = qc.Solver(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], N_ANT, n_time)
    t_map, f_map = np.arange(n_time, dtype=np.int32), np.zeros(n_chan, np.int32)
    uneven = pb["nu"].copy()
    uneven[5] += 0.003
    with pytest.raises(qc.QCError):
        S.delay_init(qc.Term("delay", t_map, f_map, n_time, 1, N_ANT, chan_freq=uneven))
    with pytest.raises(qc.QCError):
        S.delay_init(qc.Term("delay", t_map, f_map, n_time, 1, N_ANT, chan_freq=pb["nu"]), ref=N_ANT)
    with pytest.raises(qc.QCError):
        S.delay_init(qc.Term("delay", t_map, f_map, n_time, 1, N_ANT, chan_freq=pb["nu"]), oversample=1024)
    with pytest.raises(qc.QCError):
        S.delay_init(qc.Term("diag", t_map, f_map, n_time, 1, N_ANT))
    S.close()
