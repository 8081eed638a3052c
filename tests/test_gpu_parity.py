"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: referenced gains within 1e-4 relative (complex64 arithmetic,
FP64 accumulators) and chi^2 within 1e-5 relative, as the solver's
accuracy target states; single normal-equation steps and residuals are
compared element by element at FP32 rounding level.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from oracle.gauge import chain_products, reference_chain, reference_diag, rel_err
from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu

GAIN_TOL = 1e-4
CHI2_TOL = 1e-5


def run_oracle(obs, kinds_params=None, n_epochs=1, max_iter=20, tol=1e-6, damping_mode=1, damping=1.0):
    P = O.OracleProblem.from_obs(obs)
    terms = [O.OracleTerm.from_spec(s, obs.n_ant, params=None if kinds_params is None else kinds_params[i],
                                    max_iter=max_iter, tol=tol) for i, s in enumerate(obs.terms)]
    its = O.solve(P, terms, n_epochs=n_epochs, damping_mode=damping_mode, damping=damping)
    return terms, its, O.residual(P, terms)


def run_gpu(obs, kinds_params=None, n_epochs=1, max_iter=20, tol=1e-6, damping_mode=1, damping=1.0, **kw):
    S = qc.Solver.from_obs(obs, model_fp16=kw.pop("model_fp16", False))
    terms = [qc.Term.from_spec(s, obs.n_ant, gains=None if kinds_params is None else kinds_params[i],
                               max_iter=max_iter, tol=tol) for i, s in enumerate(obs.terms)]
    st = S.solve(terms, n_epochs=n_epochs, damping_mode=damping_mode, damping=damping, want_chi2=True, **kw)
    chi2 = S.residual(terms)
    S.close()
    return terms, st, chi2


def jones_of(t):
    if t.kind == "phase":
        return synth.phase_to_jones(np.asarray(t.gains, dtype=np.float64))
    return np.asarray(t.gains, dtype=np.complex128)


def products(obs, terms):
    return chain_products([jones_of(t) for t in terms], [t.t_map for t in terms], [t.f_map for t in terms],
                          obs.n_time, obs.n_chan)


def assert_chain_parity(obs, gterms, oterms, tol=GAIN_TOL):
    Cg = reference_chain(products(obs, gterms))
    Co = reference_chain(chain_products([t.jones() for t in oterms], [t.t_map for t in oterms],
                                        [t.f_map for t in oterms], obs.n_time, obs.n_chan))
    err = rel_err(Cg, Co)
    assert err < tol, err
    return err


# ---------------------------------------------------------------------------
# the small plain workload: 7 antennas, 60 x 16, diagonal gains on 4 x 4 intervals
# ---------------------------------------------------------------------------

def test_plain_small_workload_matches_oracle():
    obs = synth.plain_small(seed=0, noise=0.01)
    ot, oits, ochi2 = run_oracle(obs)
    gt, st, gchi2 = run_gpu(obs)
    err = rel_err(reference_diag(jones_of(gt[0])), reference_diag(ot[0].params))
    assert err < GAIN_TOL, err
    assert abs(gchi2 - ochi2) <= CHI2_TOL * ochi2
    assert abs(st.chi2_after - ochi2) <= CHI2_TOL * ochi2
    # iteration counts agree up to the last step of the tolerance test
    assert np.max(np.abs(gt[0].iters - oits[0])) <= 2
    assert np.all(gt[0].gain_flags == 0)
    assert st.vis_iters > 0 and st.acc_launches >= 1


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("use_graph", [True, False])
def test_plain_small_tile_orders_and_graph_agree(order, use_graph, kernel):
    obs = synth.plain_small(seed=1, noise=0.01)
    ot, _, ochi2 = run_oracle(obs)
    gt, st, gchi2 = run_gpu(obs, order=order, use_graph=use_graph, kernel=kernel)
    assert rel_err(reference_diag(jones_of(gt[0])), reference_diag(ot[0].params)) < GAIN_TOL
    assert abs(gchi2 - ochi2) <= CHI2_TOL * ochi2


# ---------------------------------------------------------------------------
# one Gauss-Newton step, element by element (JHJ / JHr / block solve parity)
# ---------------------------------------------------------------------------

def random_chain_obs(seed, kinds, n_ant=6, n_time=5, n_chan=45, t_int=(2, 5, 1), f_int=(7, 1, 45), noise=0.1,
                     flag_frac=0.2):
    """Polarised random model, random per-correlation weights, ragged channel count (45),
    intervals not aligned with 32-channel tiles, flags, mixed baseline orientation."""
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(n_ant)
    swap = rng.random(p.size) < 0.3
    p, q = np.where(swap, q, p), np.where(swap, p, q)
    ant1, ant2 = np.tile(p, n_time), np.tile(q, n_time)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    shp = (ant1.size, n_chan, 4)
    model = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    terms = []
    for i, k in enumerate(kinds):
        ti, fi = t_int[i % len(t_int)], f_int[i % len(f_int)]
        nt, nf = -(-n_time // ti), -(-n_chan // fi)
        spec = synth.TermSpec(k, synth.interval_map(n_time, ti), synth.interval_map(n_chan, fi), nt, nf)
        if k == "phase":
            spec.truth = 0.5 * rng.standard_normal((nt, nf, n_ant, 2))
        elif k == "diag":
            spec.truth = synth.diag_truth(n_ant, nt, nf, rng)
        else:
            spec.truth = synth.full_truth(n_ant, nt, nf, rng, leakage=0.2)
        terms.append(spec)
    data = synth.corrupt(model, terms, ant1, ant2, tidx, n_chan)
    data = data + noise * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    weight = rng.uniform(0.5, 2.0, size=shp)
    flag = (rng.random((ant1.size, n_chan)) < flag_frac).astype(np.uint8)
    return synth.Observation(n_ant, n_time, n_chan, data.astype(np.complex64), model.astype(np.complex64),
                             weight.astype(np.float32), flag, ant1.astype(np.int32), ant2.astype(np.int32), tidx,
                             np.zeros(n_chan), terms, {})


def start_params(obs, rng):
    out = []
    for s in obs.terms:
        if s.kind == "phase":
            out.append(s.truth + 0.2 * rng.standard_normal(s.truth.shape))
        else:
            g = s.truth + 0.1 * (rng.standard_normal(s.truth.shape) + 1j * rng.standard_normal(s.truth.shape))
            if s.kind == "diag":
                g[..., 1] = 0
                g[..., 2] = 0
            out.append(g)
    return out


CHAINS = [("diag",), ("full",), ("phase",), ("full", "diag"), ("diag", "full"), ("phase", "full", "diag"),
          ("full", "phase", "diag", "diag")]


@pytest.mark.parametrize("kinds", CHAINS)
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5])
def test_single_step_matches_oracle_for_every_chain_position(kinds, order, kernel):
    obs = random_chain_obs(7, kinds)
    rng = np.random.default_rng(3)
    start = start_params(obs, rng)
    start32 = [np.asarray(s, dtype=np.float32 if k == "phase" else np.complex64) for s, k in zip(start, kinds)]
    for n in range(len(kinds)):
        P = O.OracleProblem.from_obs(obs)
        ot = [O.OracleTerm.from_spec(s, obs.n_ant, params=np.asarray(p, np.float64 if s.kind == "phase" else np.complex128),
                                     solve=(i == n), max_iter=1, tol=0.0)
              for i, (s, p) in enumerate(zip(obs.terms, start32))]
        O.solve(P, ot, damping_mode=0, damping=1.0)
        S = qc.Solver.from_obs(obs)
        gt = [qc.Term.from_spec(s, obs.n_ant, gains=p, solve=(i == n), max_iter=1, tol=0.0)
              for i, (s, p) in enumerate(zip(obs.terms, start32))]
        S.solve(gt, damping_mode=0, damping=1.0, order=order, kernel=kernel)
        S.close()
        want = ot[n].params
        got = np.asarray(gt[n].gains, dtype=np.float64 if kinds[n] == "phase" else np.complex128)
        step = want - np.asarray(start32[n], dtype=want.dtype)
        err = np.max(np.abs(got - want)) / max(np.max(np.abs(step)), 1e-30)
        assert err < 2e-3, (kinds, n, err)          # relative to the size of the step itself
        assert np.array_equal(gt[n].gain_flags, ot[n].gain_flags)


@pytest.mark.parametrize("kinds", [("diag",), ("full", "diag"), ("diag", "full")])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("kernel", [4, 5])
def test_single_step_with_rows_of_more_than_32_chunks(kinds, order, kernel):
    """Rows of 1100 channels (35 chunks of 32, the last one ragged): the warp-specialised kernel's
    rows need two words of chunk bits and its strips span 35 chunk units each; intervals of 7
    channels straddle the chunks, so the other term's entries per chunk vary in number."""
    obs = random_chain_obs(13, kinds, n_ant=5, n_time=3, n_chan=1100, t_int=(1, 3), f_int=(7, 1100),
                           flag_frac=0.3)
    rng = np.random.default_rng(4)
    start = start_params(obs, rng)
    start32 = [np.asarray(s_, dtype=np.complex64) for s_ in start]
    for n in range(len(kinds)):
        P = O.OracleProblem.from_obs(obs)
        ot = [O.OracleTerm.from_spec(s_, obs.n_ant, params=np.asarray(p_, np.complex128), solve=(i == n),
                                     max_iter=1, tol=0.0) for i, (s_, p_) in enumerate(zip(obs.terms, start32))]
        O.solve(P, ot, damping_mode=0, damping=1.0)
        S = qc.Solver.from_obs(obs)
        gt = [qc.Term.from_spec(s_, obs.n_ant, gains=p_, solve=(i == n), max_iter=1, tol=0.0)
              for i, (s_, p_) in enumerate(zip(obs.terms, start32))]
        S.solve(gt, damping_mode=0, damping=1.0, order=order, kernel=kernel)
        S.close()
        want = ot[n].params
        got = np.asarray(gt[n].gains, dtype=np.complex128)
        step = want - np.asarray(start32[n], dtype=want.dtype)
        err = np.max(np.abs(got - want)) / max(np.max(np.abs(step)), 1e-30)
        assert err < 2e-3, (kinds, n, err)
        assert np.array_equal(gt[n].gain_flags, ot[n].gain_flags)


# ---------------------------------------------------------------------------
# residual and chi^2
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kinds", [("full", "diag"), ("phase", "full", "diag")])
def test_residual_matches_oracle_elementwise(kinds):
    obs = random_chain_obs(11, kinds)
    rng = np.random.default_rng(5)
    start = start_params(obs, rng)
    P = O.OracleProblem.from_obs(obs)
    ot = [O.OracleTerm.from_spec(s, obs.n_ant, params=p) for s, p in zip(obs.terms, start)]
    ochi2, ores = O.residual(P, ot, want_resid=True)
    S = qc.Solver.from_obs(obs)
    gt = [qc.Term.from_spec(s, obs.n_ant, gains=p, solve=False) for s, p in zip(obs.terms, start)]
    gchi2, gres = S.residual(gt, want_resid=True)
    S.close()
    scale = np.max(np.abs(obs.data))
    assert np.max(np.abs(gres - ores)) < 1e-5 * scale
    assert abs(gchi2 - ochi2) <= 1e-5 * ochi2


# ---------------------------------------------------------------------------
# converged multi-term chains
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5])
def test_two_term_chain_matches_oracle(kernel):
    obs = synth.plain_large(seed=3, n_ant=10, n_time=12, n_chan=40, noise=0.05, flag_row_frac=0.1, n_src=8)
    ot, _, ochi2 = run_oracle(obs, n_epochs=3)
    gt, st, gchi2 = run_gpu(obs, n_epochs=3, kernel=kernel)
    assert_chain_parity(obs, gt, ot)
    assert abs(gchi2 - ochi2) <= CHI2_TOL * ochi2


@pytest.mark.parametrize("kind", ["full", "phase"])
def test_single_term_kinds_converge_like_oracle(kind):
    rng = np.random.default_rng(21)
    n_ant, n_time, n_chan = 8, 8, 24
    freqs = synth.meerkat_band(n_chan)
    spec = synth.TermSpec(kind, synth.interval_map(n_time, 2), synth.interval_map(n_chan, 8), 4, 3)
    spec.truth = (0.4 * rng.standard_normal((4, 3, n_ant, 2)) if kind == "phase"
                  else synth.full_truth(n_ant, 4, 3, rng, leakage=0.1))
    obs = synth.make_observation(n_ant, n_time, freqs, [spec], n_src=6, seed=21, noise=0.02, rng=rng,
                                 max_baseline_m=4000.0, flag_row_frac=0.05)
    ot, _, ochi2 = run_oracle(obs, max_iter=40)
    gt, _, gchi2 = run_gpu(obs, max_iter=40)
    assert_chain_parity(obs, gt, ot)
    assert abs(gchi2 - ochi2) <= CHI2_TOL * ochi2


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [0, 3, 4, 5])
def test_flagged_nan_data_and_dead_antenna(kernel):
    obs = synth.plain_small(seed=4, noise=0.01, n_time=16, n_chan=16)
    dead = (obs.ant1 == 3) | (obs.ant2 == 3)
    obs.flag[dead] = 1
    obs.flag[::5, 3] = 1
    obs.data[obs.flag.astype(bool)] = np.nan
    ot, _, ochi2 = run_oracle(obs)
    gt, _, gchi2 = run_gpu(obs, kernel=kernel)
    assert np.all(gt[0].gain_flags[:, :, 3] == 1)
    assert np.all(np.asarray(gt[0].gains)[:, :, 3, [0, 3]] == 1)
    assert np.array_equal(gt[0].gain_flags, ot[0].gain_flags)
    good = [a for a in range(obs.n_ant) if a != 3]
    g = reference_diag(jones_of(gt[0])[:, :, good])
    o = reference_diag(ot[0].params[:, :, good])
    assert rel_err(g, o) < GAIN_TOL
    assert np.isfinite(gchi2) and abs(gchi2 - ochi2) <= CHI2_TOL * ochi2


@pytest.mark.parametrize("kernel", [0, 3, 4, 5])
def test_autocorrelations_are_ignored(kernel):
    obs = synth.plain_small(seed=5, noise=0.01, n_time=8, n_chan=8)
    base = run_gpu(obs, kernel=kernel)[0][0].gains.copy()
    n_t = obs.n_time
    auto_rows = np.arange(obs.n_ant)
    ant = np.concatenate([obs.ant1, np.tile(auto_rows, n_t)])
    ant2 = np.concatenate([obs.ant2, np.tile(auto_rows, n_t)])
    tt = np.concatenate([obs.time_idx, np.repeat(np.arange(n_t, dtype=np.int32), obs.n_ant)])
    extra = np.full((obs.n_ant * n_t, obs.n_chan, 4), 7.0 + 3j)
    obs2 = synth.Observation(obs.n_ant, n_t, obs.n_chan, np.concatenate([obs.data, extra]),
                             np.concatenate([obs.model, extra]), np.ones((ant.size, obs.n_chan, 4)),
                             np.zeros((ant.size, obs.n_chan), np.uint8), ant.astype(np.int32),
                             ant2.astype(np.int32), tt, obs.freqs, obs.terms, {})
    got = run_gpu(obs2, kernel=kernel)[0][0].gains
    assert np.allclose(got, base, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("kernel", [0, 3, 4, 5])
def test_empty_problem_and_fully_flagged(kernel):
    obs = synth.plain_small(seed=6, noise=0.01, n_time=4, n_chan=4)
    obs.flag[:] = 1
    gt, st, chi2 = run_gpu(obs, kernel=kernel)
    assert chi2 == 0.0
    assert np.all(gt[0].gain_flags == 1)
    assert np.all(gt[0].iters == 1)
    S = qc.Solver(np.zeros((0, 4, 4), np.complex64), np.zeros((0, 4, 4), np.complex64),
                  np.zeros((0, 4, 4), np.float32), None, np.zeros(0, np.int32), np.zeros(0, np.int32),
                  np.zeros(0, np.int32), 3, 1)
    t = qc.Term("diag", np.zeros(1, np.int32), np.zeros(4, np.int32), 1, 1, 3)
    S.solve([t], kernel=kernel)
    assert np.all(t.gain_flags == 1)
    assert S.residual([t]) == 0.0
    S.close()


def test_solve_rejects_bad_terms():
    obs = synth.plain_small(seed=0, noise=0.01, n_time=4, n_chan=4)
    S = qc.Solver.from_obs(obs)
    bad_fmap = qc.Term("diag", np.zeros(4, np.int32), np.array([0, 1, 0, 1], np.int32), 1, 2, obs.n_ant)
    with pytest.raises(qc.QCError) as e:
        S.solve([bad_fmap])
    assert e.value.code == qc.QC_EINVAL
    bad_range = qc.Term("diag", np.full(4, 3, np.int32), np.zeros(4, np.int32), 1, 1, obs.n_ant)
    with pytest.raises(qc.QCError):
        S.solve([bad_range])
    with pytest.raises(qc.QCError):
        S.solve([qc.Term("diag", np.zeros(4, np.int32), np.zeros(4, np.int32), 1, 1, obs.n_ant, max_iter=0)])
    S.close()


# ---------------------------------------------------------------------------
# FP16 model storage (mixed precision)
# ---------------------------------------------------------------------------

def fp16_dequantized_model(obs):
    """The model as the FP16 packing stores it: per baseline (ant1, ant2) a scale s = the largest
    finite |component| over its samples, components multiplied by 1/s in float32 and rounded to
    float16, read back as float16 * s in float32."""
    m = np.ascontiguousarray(obs.model, dtype=np.complex64)
    f = m.view(np.float32).reshape(m.shape[0], -1)
    deq = np.empty_like(f)
    keys = obs.ant1.astype(np.int64) * 65536 + obs.ant2.astype(np.int64)
    for k in np.unique(keys):
        rows = np.nonzero(keys == k)[0]
        a = np.abs(f[rows])
        a = a[np.isfinite(a)]
        s = np.float32(a.max()) if a.size and a.max() > 0 else np.float32(1.0)
        inv = np.float32(1.0) / s
        q = (f[rows] * inv).astype(np.float16)
        deq[rows] = q.astype(np.float32) * s
    return deq.view(np.complex64).reshape(m.shape)


@pytest.mark.parametrize("kernel", [0, 2, 4, 5])
def test_fp16_model_matches_oracle_on_the_dequantized_model(kernel):
    """With the model the FP16 packing actually stores, the GPU solve (FP16 model, FP32 sums, FP64
    solves and accumulators) must meet the complex64 tolerances against the FP64 oracle."""
    obs = synth.plain_large(seed=3, n_ant=10, n_time=12, n_chan=40, noise=0.05, flag_row_frac=0.1, n_src=8)
    deq = dataclasses.replace(obs, model=fp16_dequantized_model(obs))
    ot, _, ochi2 = run_oracle(deq, n_epochs=3)
    gt, st, gchi2 = run_gpu(obs, n_epochs=3, kernel=kernel, model_fp16=True)
    assert_chain_parity(obs, gt, ot)
    assert abs(gchi2 - ochi2) <= CHI2_TOL * ochi2


def test_fp16_model_error_against_the_exact_model_is_bounded():
    """Against the oracle on the unquantized model the error is set by float16 rounding of the
    model (relative 2^-11 of each baseline's largest component), well inside 1e-3."""
    obs = synth.plain_large(seed=5, n_ant=10, n_time=12, n_chan=40, noise=0.05, flag_row_frac=0.1, n_src=8)
    ot, _, ochi2 = run_oracle(obs, n_epochs=3)
    gt, st, gchi2 = run_gpu(obs, n_epochs=3, model_fp16=True)
    err = assert_chain_parity(obs, gt, ot, tol=1e-3)
    assert err > 0
    assert abs(gchi2 - ochi2) <= 1e-3 * ochi2
