"""Terms solved from per-(interval, antenna pair) sums (qc_opts.moments), against the oracle and
against the per-sample GPU path.

- One Gauss-Newton step of a diagonal, full or phase-only single term from the sums equals the
  oracle's step (relative to the size of the step), with both row orientations, random
  per-correlation weights, flags, a ragged last chunk (45 channels) and intervals that straddle
  the 32-channel chunks; gain flags bit for bit.
- Two-term chains: each term's single step against the oracle, the first from the full form with
  the second folded into the model, the second from the diagonal form when it is diagonal or
  phase-only (a full second term takes the per-sample path); converged G+B and G+phase chains.
- Converged solves: gains after referencing within 1e-4 and chi^2 within 1e-5 of the oracle for
  the small plain workload and for full and phase-only terms; intervals one time wide that span
  several chunks; dead antennas with NaN data under their flags; fully flagged intervals;
  autocorrelations; robust reweighting across epochs.
- Three-term chains are not solved from sums: the option changes nothing.
- Statistics: the pass time lies inside the accumulate time, and the byte count is one pass over
  the samples plus, per iteration and active interval, the sums read on both sides and the
  accumulators written.
"""
import numpy as np
import pytest

import oracle as O
from oracle import robust
from oracle.gauge import chain_products, reference_chain, reference_diag, rel_err
from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu

GAIN_TOL = 1e-4
CHI2_TOL = 1e-5
MOM_WORDS = 100          # FP32 words of sums per (interval, antenna pair)


def _obs(seed, kind, n_ant=6, n_time=5, n_chan=45, ti=2, fi=7, noise=0.1, flag_frac=0.2):
    """Polarised random model, random per-correlation weights, flags, mixed baseline orientation."""
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(n_ant)
    swap = rng.random(p.size) < 0.4
    p, q = np.where(swap, q, p), np.where(swap, p, q)
    ant1, ant2 = np.tile(p, n_time), np.tile(q, n_time)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    shp = (ant1.size, n_chan, 4)
    model = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    nt, nf = -(-n_time // ti), -(-n_chan // fi)
    spec = synth.TermSpec(kind, synth.interval_map(n_time, ti), synth.interval_map(n_chan, fi), nt, nf)
    if kind == "phase":
        spec.truth = 0.5 * rng.standard_normal((nt, nf, n_ant, 2))
    elif kind == "diag":
        spec.truth = synth.diag_truth(n_ant, nt, nf, rng)
    else:
        spec.truth = synth.full_truth(n_ant, nt, nf, rng, leakage=0.2)
    data = synth.corrupt(model, [spec], ant1, ant2, tidx, n_chan)
    data = data + noise * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    weight = rng.uniform(0.5, 2.0, size=shp)
    flag = (rng.random((ant1.size, n_chan)) < flag_frac).astype(np.uint8)
    return synth.Observation(n_ant, n_time, n_chan, data.astype(np.complex64), model.astype(np.complex64),
                             weight.astype(np.float32), flag, ant1.astype(np.int32), ant2.astype(np.int32), tidx,
                             np.zeros(n_chan), [spec], {})


def _start(spec, rng):
    if spec.kind == "phase":
        return (spec.truth + 0.2 * rng.standard_normal(spec.truth.shape)).astype(np.float32)
    g = spec.truth + 0.1 * (rng.standard_normal(spec.truth.shape) + 1j * rng.standard_normal(spec.truth.shape))
    if spec.kind == "diag":
        g[..., 1] = 0
        g[..., 2] = 0
    return g.astype(np.complex64)


def _jones(t):
    if t.kind == "phase":
        return synth.phase_to_jones(np.asarray(t.gains, dtype=np.float64))
    return np.asarray(t.gains, dtype=np.complex128)


def _oracle(obs, params=None, max_iter=20, tol=1e-6, damping_mode=1, damping=1.0, n_epochs=1):
    P = O.OracleProblem.from_obs(obs)
    T = [O.OracleTerm.from_spec(s, obs.n_ant, params=params, max_iter=max_iter, tol=tol) for s in obs.terms]
    its = O.solve(P, T, n_epochs=n_epochs, damping_mode=damping_mode, damping=damping)
    return T, its, O.residual(P, T)


def _gpu(obs, gains=None, max_iter=20, tol=1e-6, moments=True, **kw):
    S = qc.Solver.from_obs(obs)
    T = [qc.Term.from_spec(s, obs.n_ant, gains=gains, max_iter=max_iter, tol=tol) for s in obs.terms]
    st = S.solve(T, want_chi2=True, moments=moments, **kw)
    S.close()
    return T, st


def _chain_err(obs, gt, ot):
    Cg = reference_chain(chain_products([_jones(t) for t in gt], [t.t_map for t in gt], [t.f_map for t in gt],
                                        obs.n_time, obs.n_chan))
    Co = reference_chain(chain_products([t.jones() for t in ot], [t.t_map for t in ot], [t.f_map for t in ot],
                                        obs.n_time, obs.n_chan))
    return rel_err(Cg, Co)


@pytest.mark.parametrize("kind", ["diag", "full", "phase"])
@pytest.mark.parametrize("seed", [0, 1])
def test_single_step_from_sums_matches_oracle(kind, seed):
    obs = _obs(30 + seed, kind)
    start = _start(obs.terms[0], np.random.default_rng(seed))
    pdt = np.float64 if kind == "phase" else np.complex128
    T, _, _ = _oracle(obs, params=start.astype(pdt), max_iter=1, tol=0.0, damping_mode=0)
    gt, st = _gpu(obs, gains=start, max_iter=1, tol=0.0, damping_mode=0, damping=1.0)
    want = T[0].params
    got = np.asarray(gt[0].gains, dtype=pdt)
    step = want - start.astype(pdt)
    err = np.max(np.abs(got - want)) / max(np.max(np.abs(step)), 1e-30)
    assert err < 2e-3, (kind, err)
    assert np.array_equal(gt[0].gain_flags, T[0].gain_flags)
    assert st.pass_ms > 0 and st.pass_ms <= st.acc_ms


def test_small_plain_workload_matches_oracle():
    obs = synth.plain_small(seed=0, noise=0.01)
    T, its, ochi2 = _oracle(obs)
    gt, st = _gpu(obs)
    assert rel_err(reference_diag(_jones(gt[0])), reference_diag(T[0].params)) < GAIN_TOL
    assert abs(st.chi2_after - ochi2) <= CHI2_TOL * ochi2
    assert np.max(np.abs(gt[0].iters - its[0])) <= 2
    # the per-sample path reaches the same gains
    gp, _ = _gpu(obs, moments=False)
    assert rel_err(reference_diag(_jones(gt[0])), reference_diag(_jones(gp[0]))) < GAIN_TOL


@pytest.mark.parametrize("kind", ["full", "phase", "diag"])
def test_converged_kinds_match_oracle(kind):
    obs = _obs(41, kind, n_ant=8, n_time=8, n_chan=45, ti=2, fi=9, noise=0.02, flag_frac=0.05)
    T, _, ochi2 = _oracle(obs, max_iter=40)
    gt, st = _gpu(obs, max_iter=40)
    assert _chain_err(obs, gt, T) < GAIN_TOL
    assert abs(st.chi2_after - ochi2) <= CHI2_TOL * ochi2


def test_intervals_one_time_wide_spanning_chunks():
    """Interval 1 time x 100 channels over four chunks (the last ragged): a warp's keys stay the
    same across the chunks of a row, so each row's sums are flushed once per chunk group."""
    obs = _obs(52, "full", n_ant=10, n_time=6, n_chan=100, ti=1, fi=100, noise=0.02, flag_frac=0.1)
    T, _, ochi2 = _oracle(obs, max_iter=40)
    gt, st = _gpu(obs, max_iter=40)
    assert _chain_err(obs, gt, T) < GAIN_TOL
    assert abs(st.chi2_after - ochi2) <= CHI2_TOL * ochi2


def test_dead_antenna_nan_data_and_fully_flagged_interval():
    obs = synth.plain_small(seed=4, noise=0.01, n_time=16, n_chan=16)
    dead = (obs.ant1 == 3) | (obs.ant2 == 3)
    obs.flag[dead] = 1
    obs.flag[::5, 3] = 1
    obs.flag[obs.time_idx < 4] = 1                      # the first time interval: nothing usable
    obs.data[obs.flag.astype(bool)] = np.nan
    T, _, ochi2 = _oracle(obs)
    gt, st = _gpu(obs)
    assert np.array_equal(gt[0].gain_flags, T[0].gain_flags)
    assert np.all(gt[0].gain_flags[:, :, 3] == 1) and np.all(gt[0].gain_flags[0] == 1)
    good = [a for a in range(obs.n_ant) if a != 3]
    assert rel_err(reference_diag(_jones(gt[0])[1:, :, good]), reference_diag(T[0].params[1:, :, good])) < GAIN_TOL
    assert np.isfinite(st.chi2_after) and abs(st.chi2_after - ochi2) <= CHI2_TOL * ochi2


def test_autocorrelations_are_ignored():
    obs = synth.plain_small(seed=5, noise=0.01, n_time=8, n_chan=8)
    base = _gpu(obs)[0][0].gains.copy()
    n_t = obs.n_time
    auto = np.arange(obs.n_ant)
    a1 = np.concatenate([obs.ant1, np.tile(auto, n_t)])
    a2 = np.concatenate([obs.ant2, np.tile(auto, n_t)])
    tt = np.concatenate([obs.time_idx, np.repeat(np.arange(n_t, dtype=np.int32), obs.n_ant)])
    extra = np.full((obs.n_ant * n_t, obs.n_chan, 4), 7.0 + 3j)
    obs2 = synth.Observation(obs.n_ant, n_t, obs.n_chan, np.concatenate([obs.data, extra]),
                             np.concatenate([obs.model, extra]), np.ones((a1.size, obs.n_chan, 4)),
                             np.zeros((a1.size, obs.n_chan), np.uint8), a1.astype(np.int32), a2.astype(np.int32),
                             tt, obs.freqs, obs.terms, {})
    got = _gpu(obs2)[0][0].gains
    assert np.allclose(got, base, rtol=1e-5, atol=1e-6)


def test_robust_reweighting_from_sums_matches_oracle():
    obs = synth.plain_small(seed=7, noise=0.01)
    rng = np.random.default_rng(3)
    bad = rng.random(obs.flag.shape) < 0.01
    obs.data[bad] += 5.0 * (rng.standard_normal((bad.sum(), 4)) + 1j * rng.standard_normal((bad.sum(), 4)))
    P = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    robust.solve_robust(P, [T], 3, 3.0)
    ochi2 = O.residual(P, [T])
    gt, st = _gpu(obs, n_epochs=3, robust_nu=3.0)
    assert rel_err(reference_diag(_jones(gt[0])), reference_diag(T.params)) < GAIN_TOL
    assert abs(st.chi2_after - ochi2) <= CHI2_TOL * ochi2


def test_chains_outside_the_option_solve_as_without_it():
    """Three-term chains are not solved from sums: the option changes nothing."""
    obs = _chain_obs(90, ("full", "diag", "phase"), t_int=(2, 5, 1), f_int=(7, 1, 45), noise=0.05)
    a, sa = _gpu(obs, max_iter=10, moments=True)
    b, sb = _gpu(obs, max_iter=10, moments=False)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x.gains), np.asarray(y.gains))
    assert sa.pass_ms == 0 and sb.pass_ms == 0


def test_byte_count_is_one_pass_plus_the_sums():
    obs = _obs(60, "full", n_ant=7, n_time=4, n_chan=40, ti=2, fi=8)
    start = _start(obs.terms[0], np.random.default_rng(0))
    _, plain = _gpu(obs, gains=start, max_iter=1, tol=0.0, moments=False)
    _, mom = _gpu(obs, gains=start, max_iter=1, tol=0.0, moments=True)
    spec = obs.terms[0]
    n_bins = spec.n_tint * spec.n_fint
    n_pairs = len({(min(p, q), max(p, q)) for p, q in zip(obs.ant1, obs.ant2) if p != q})
    per_iter = 2 * n_pairs * MOM_WORDS * 4 + 8 * obs.n_ant * 24
    assert mom.acc_bytes == plain.acc_bytes + n_bins * per_iter
    assert mom.vis_iters == plain.vis_iters


# ---------------------------------------------------------------------------
# two-term chains: the full form with the term to the right folded into the model, and the
# diagonal form for a diagonal or phase-only term with a term to its left
# ---------------------------------------------------------------------------

def _chain_obs(seed, kinds, n_ant=6, n_time=5, n_chan=45, t_int=(2, 5), f_int=(7, 1), noise=0.1, flag_frac=0.2):
    """Polarised random model, random per-correlation weights, flags, mixed baseline orientation,
    intervals not aligned with the chunks, a ragged last chunk."""
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(n_ant)
    swap = rng.random(p.size) < 0.4
    p, q = np.where(swap, q, p), np.where(swap, p, q)
    ant1, ant2 = np.tile(p, n_time), np.tile(q, n_time)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    shp = (ant1.size, n_chan, 4)
    model = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    specs = []
    for i, kind in enumerate(kinds):
        ti, fi = t_int[i], f_int[i]
        nt, nf = -(-n_time // ti), -(-n_chan // fi)
        spec = synth.TermSpec(kind, synth.interval_map(n_time, ti), synth.interval_map(n_chan, fi), nt, nf)
        if kind == "phase":
            spec.truth = 0.5 * rng.standard_normal((nt, nf, n_ant, 2))
        elif kind == "diag":
            spec.truth = synth.diag_truth(n_ant, nt, nf, rng)
        else:
            spec.truth = synth.full_truth(n_ant, nt, nf, rng, leakage=0.2)
        specs.append(spec)
    data = synth.corrupt(model, specs, ant1, ant2, tidx, n_chan)
    data = data + noise * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    weight = rng.uniform(0.5, 2.0, size=shp)
    flag = (rng.random((ant1.size, n_chan)) < flag_frac).astype(np.uint8)
    return synth.Observation(n_ant, n_time, n_chan, data.astype(np.complex64), model.astype(np.complex64),
                             weight.astype(np.float32), flag, ant1.astype(np.int32), ant2.astype(np.int32), tidx,
                             np.zeros(n_chan), specs, {})


CHAINS = [("full", "diag"), ("full", "phase"), ("diag", "diag"), ("phase", "full"), ("diag", "full"),
          ("full", "full")]


@pytest.mark.parametrize("kinds", CHAINS)
def test_two_term_single_step_from_sums_matches_oracle(kinds):
    """Each term of the chain takes one step with the other fixed: the first term (nothing to
    its left) from the full form with the second folded into the model; the second, if diagonal
    or phase-only, from the diagonal form (a full second term takes the per-sample path)."""
    obs = _chain_obs(70 + CHAINS.index(kinds), kinds)
    rng = np.random.default_rng(5)
    start = [_start(s, rng) for s in obs.terms]
    for n in range(2):
        P = O.OracleProblem.from_obs(obs)
        ot = [O.OracleTerm.from_spec(s, obs.n_ant, params=g.astype(np.float64 if s.kind == "phase" else np.complex128),
                                     solve=(i == n), max_iter=1, tol=0.0)
              for i, (s, g) in enumerate(zip(obs.terms, start))]
        O.solve(P, ot, damping_mode=0, damping=1.0)
        S = qc.Solver.from_obs(obs)
        gt = [qc.Term.from_spec(s, obs.n_ant, gains=g, solve=(i == n), max_iter=1, tol=0.0)
              for i, (s, g) in enumerate(zip(obs.terms, start))]
        st = S.solve(gt, damping_mode=0, damping=1.0, moments=True)
        S.close()
        want = ot[n].params
        got = np.asarray(gt[n].gains, dtype=want.dtype)
        step = want - start[n].astype(want.dtype)
        err = np.max(np.abs(got - want)) / max(np.max(np.abs(step)), 1e-30)
        assert err < 2e-3, (kinds, n, err)
        assert np.array_equal(gt[n].gain_flags, ot[n].gain_flags)
        from_sums = n == 0 or kinds[1] != "full"
        assert (st.pass_ms > 0) == from_sums, (kinds, n, st.pass_ms)


@pytest.mark.parametrize("kinds", [("full", "diag"), ("full", "phase")])
def test_two_term_chain_from_sums_converges_like_oracle(kinds):
    """The large workload's shape at a small size (G full per time, B per channel over all times),
    three epochs, both terms from sums: chain products within 1e-4 and chi^2 within 1e-5 of the
    oracle, and the same as the per-sample path."""
    obs = synth.plain_large(seed=3, n_ant=10, n_time=12, n_chan=40, noise=0.05, flag_row_frac=0.1, n_src=8)
    if kinds[1] == "phase":
        rng = np.random.default_rng(4)
        B = obs.terms[1]
        spec = synth.TermSpec("phase", B.t_map, B.f_map, B.n_tint, B.n_fint)
        spec.truth = 0.3 * rng.standard_normal((B.n_tint, B.n_fint, obs.n_ant, 2))
        obs.terms = [obs.terms[0], spec]
        obs.data = synth.corrupt(obs.model, obs.terms, obs.ant1, obs.ant2, obs.time_idx, obs.n_chan).astype(
            np.complex64) + (0.05 * (rng.standard_normal(obs.data.shape) + 1j * rng.standard_normal(obs.data.shape))
                             ).astype(np.complex64)
    T, _, ochi2 = _oracle(obs, n_epochs=3)
    gt, st = _gpu(obs, n_epochs=3)
    assert _chain_err(obs, gt, T) < GAIN_TOL
    assert abs(st.chi2_after - ochi2) <= CHI2_TOL * ochi2
    assert st.pass_ms > 0
    gp, _ = _gpu(obs, n_epochs=3, moments=False)
    Cm = [_jones(t) for t in gt]
    Cp = [_jones(t) for t in gp]
    err = rel_err(reference_chain(chain_products(Cm, [t.t_map for t in gt], [t.f_map for t in gt], obs.n_time,
                                                 obs.n_chan)),
                  reference_chain(chain_products(Cp, [t.t_map for t in gp], [t.f_map for t in gp], obs.n_time,
                                                 obs.n_chan)))
    assert err < GAIN_TOL
