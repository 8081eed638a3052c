"""MAD residual flagging through the C ABI (qc_mad_flag) against the oracle, bit for bit.

With unit diagonal gains the chain is the identity, so the kernel's residual is exactly the
float32 difference D - M, which the oracle forms the same way; the statistics and the
decision are float32 in the same order on both sides, so the flags must be identical."""
import numpy as np
import pytest

from oracle.mad_flag import mad_flag
from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu


def _problem(seed, n_ant=9, n_time=5, n_chan=37, flag_frac=0.1, n_out=40, autos=True, zero=False):
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(n_ant)
    if autos:
        p = np.concatenate([p, np.arange(n_ant)])
        q = np.concatenate([q, np.arange(n_ant)])
    ant1, ant2 = np.tile(p, n_time).astype(np.int32), np.tile(q, n_time).astype(np.int32)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    shp = (ant1.size, n_chan, 4)
    model = ((rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(2)).astype(np.complex64)
    noise = 0.0 if zero else 0.1
    data = (model + noise * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))).astype(np.complex64)
    idx = rng.choice(shp[0] * shp[1], size=n_out, replace=False)
    r, c = np.unravel_index(idx, shp[:2])
    data[r, c, rng.integers(0, 4, n_out)] += (rng.uniform(2, 20, n_out) * np.exp(2j * np.pi * rng.random(n_out))
                                              ).astype(np.complex64)
    weight = rng.uniform(0.5, 2.0, size=shp).astype(np.float32)
    flag = (rng.random(shp[:2]) < flag_frac).astype(np.uint8)
    return dict(data=data, model=model, weight=weight, flag=flag, ant1=ant1, ant2=ant2, tidx=tidx, n_ant=n_ant,
                n_time=n_time, n_chan=n_chan)


def _unit_term(pb):
    g = np.zeros((1, 1, pb["n_ant"], 4), np.complex64)
    g[..., 0] = g[..., 3] = 1
    return qc.Term("diag", np.zeros(pb["n_time"], np.int32), np.zeros(pb["n_chan"], np.int32), 1, 1, pb["n_ant"],
                   gains=g, solve=False)


@pytest.mark.parametrize("seed,threshold", [(1, 5.0), (2, 3.0), (3, 8.0)])
def test_flags_match_the_oracle_bit_for_bit(seed, threshold):
    pb = _problem(seed)
    S = qc.Solver(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], pb["n_ant"],
                  pb["n_time"])
    got, n = S.mad_flag([_unit_term(pb)], threshold=threshold)
    S.close()
    want, (med, mad, n_want) = mad_flag(pb["data"] - pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"],
                                        threshold=threshold)
    np.testing.assert_array_equal(got, want)
    assert n == n_want and n > 0


def test_all_flagged_and_zero_residuals():
    pb = _problem(4, flag_frac=1.0)
    S = qc.Solver(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], pb["n_ant"],
                  pb["n_time"])
    got, n = S.mad_flag([_unit_term(pb)])
    S.close()
    assert n == 0 and not got.any()
    # residuals zero except the planted ones: median and MAD are 0, every planted sample is flagged
    pb = _problem(5, flag_frac=0.0, zero=True, n_out=7, autos=False)
    S = qc.Solver(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], pb["n_ant"],
                  pb["n_time"])
    got, n = S.mad_flag([_unit_term(pb)])
    S.close()
    want, (med, mad, n_want) = mad_flag(pb["data"] - pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"])
    assert med == 0 and mad == 0
    np.testing.assert_array_equal(got, want)
    assert n == n_want == 7


def test_bad_threshold_is_rejected():
    pb = _problem(6)
    S = qc.Solver(pb["data"], pb["model"], pb["weight"], pb["flag"], pb["ant1"], pb["ant2"], pb["tidx"], pb["n_ant"],
                  pb["n_time"])
    for thr in (0.0, -1.0, float("nan")):
        with pytest.raises(qc.QCError):
            S.mad_flag([_unit_term(pb)], threshold=thr)
    S.close()


@pytest.mark.parametrize("seed,threshold", [(11, 5.0), (12, 3.0)])
def test_per_baseline_flags_match_the_oracle_bit_for_bit(seed, threshold):
    """Median and MAD per baseline (rows in either orientation grouped together)."""
    from oracle.mad_flag import mad_flag_per_baseline
    pb = _problem(seed)
    rng = np.random.default_rng(seed)
    swap = (rng.random(pb["ant1"].size) < 0.3) & (pb["ant1"] != pb["ant2"])
    a1, a2 = pb["ant1"].copy(), pb["ant2"].copy()
    a1[swap], a2[swap] = pb["ant2"][swap], pb["ant1"][swap]
    # a swapped row carries the conjugate-transposed visibilities of its baseline; for the flagger
    # only the residual's norm matters, which that leaves unchanged
    S = qc.Solver(pb["data"], pb["model"], pb["weight"], pb["flag"], a1, a2, pb["tidx"], pb["n_ant"], pb["n_time"])
    got, n = S.mad_flag([_unit_term(pb)], threshold=threshold, per_baseline=True)
    S.close()
    want, n_want = mad_flag_per_baseline(pb["data"] - pb["model"], pb["weight"], pb["flag"], a1, a2,
                                         threshold=threshold)
    np.testing.assert_array_equal(got, want)
    assert n == n_want and n > 0


@pytest.mark.parametrize("threshold", [3.0, 5.0])
def test_flags_after_a_solved_chain(threshold):
    """After a solved two-term chain (G full, B diagonal) with planted outliers:
    - bit for bit against the oracle's decision on the GPU's own residual at the solved gains
      (qc_residual forms the same float32 residual as the flagger);
    - against the oracle's FP64 residual at the same gains, rounded to complex64: median and MAD
      agree to float32 rounding, and the flags differ only for samples whose deviation lies within
      a relative 1e-4 of the threshold (float32 residual rounding decides those)."""
    import oracle as O
    from oracle.mad_flag import whitened_norm
    obs = synth.plain_large(seed=8, n_ant=10, n_time=12, n_chan=40, noise=0.05, flag_row_frac=0.1, n_src=8)
    rng = np.random.default_rng(8)
    bad = rng.random(obs.flag.shape) < 0.005
    obs.data[bad] += 2.0 * (rng.standard_normal((bad.sum(), 4)) + 1j * rng.standard_normal((bad.sum(), 4)))
    S = qc.Solver.from_obs(obs)
    terms = [qc.Term.from_spec(s, obs.n_ant, max_iter=20, tol=1e-6) for s in obs.terms]
    S.solve(terms, n_epochs=2)
    fixed = [qc.Term.from_spec(s, obs.n_ant, gains=np.asarray(t.gains).copy(), solve=False)
             for s, t in zip(obs.terms, terms)]
    got, n = S.mad_flag(fixed, threshold=threshold)
    _, res = S.residual(fixed, want_resid=True)
    S.close()
    w32 = np.asarray(obs.weight, np.float32)
    want, (med, mad, n_want) = mad_flag(res, w32, obs.flag, obs.ant1, obs.ant2, threshold=threshold)
    np.testing.assert_array_equal(got, want)
    assert n == n_want and n > 0
    P = O.OracleProblem.from_obs(obs)
    ot = [O.OracleTerm.from_spec(s, obs.n_ant, params=np.asarray(t.gains, np.complex128), solve=False)
          for s, t in zip(obs.terms, fixed)]
    _, ores = O.residual(P, ot, want_resid=True)
    r64 = ores.astype(np.complex64)
    w64, (med64, mad64, _) = mad_flag(r64, w32, obs.flag, obs.ant1, obs.ant2, threshold=threshold)
    assert abs(float(med64) - float(med)) <= 1e-5 * float(med)
    assert abs(float(mad64) - float(mad)) <= 1e-4 * float(mad)
    dev = np.abs(whitened_norm(r64, w32) - med64)
    thr = np.float32(threshold * 1.4826) * mad64
    diff = got != w64
    assert np.all(np.abs(dev[diff] - thr) <= 1e-4 * thr), int(diff.sum())
