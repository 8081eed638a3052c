"""Pin of the 4x4 full-Jones sufficient statistics (oracle/moments.py): the normal equations and
chi^2 formed from the per-(interval, baseline) sums equal the sample-by-sample ones of the C
oracle (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified, Eq. min) for a full term, and, in
their (0, 3) rows and columns, for a diagonal term, with random polarised models, random
per-correlation weights, flags, rows of both orientations and several intervals."""
import numpy as np
import pytest

import oracle as O
from oracle import moments
from paper_2412_10072_gb300 import synth


def _problem(seed, n_ant=5, n_time=4, n_chan=6):
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(n_ant)
    swap = rng.random(p.size) < 0.4
    p, q = np.where(swap, q, p), np.where(swap, p, q)
    a1, a2 = np.tile(p, n_time).astype(np.int32), np.tile(q, n_time).astype(np.int32)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    shp = (a1.size, n_chan, 4)
    data = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    model = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    weight = rng.uniform(0.5, 2.0, shp)
    flag = (rng.random(shp[:2]) < 0.2).astype(np.uint8)
    return O.OracleProblem(data, model, weight, flag, a1, a2, tidx, n_ant, n_time), rng


@pytest.mark.parametrize("kind", ["full", "diag"])
def test_full_moments_reproduce_sample_normal_equations_and_chi2(kind):
    P, rng = _problem(1)
    nt, nf = 2, 3
    tm = (np.arange(4) * nt // 4).astype(np.int32)
    fm = (np.arange(6) * nf // 6).astype(np.int32)
    g = np.eye(2).reshape(4) + 0.4 * (rng.standard_normal((nt, nf, P.n_ant, 4)) +
                                      1j * rng.standard_normal((nt, nf, P.n_ant, 4)))
    if kind == "diag":
        g[..., 1] = g[..., 2] = 0
    T = O.OracleTerm(kind, tm, fm, nt, nf, P.n_ant, params=g)
    cj, cr = O.normal_equations(P, [T], 0)
    S, Tm, U = moments.moments_full(P, tm, fm, nt, nf)
    jhj, jhr = moments.normal_equations_full(S, Tm, g.reshape(nt * nf, P.n_ant, 4))
    jhj = jhj.reshape(nt, nf, P.n_ant, 4, 4)
    jhr = jhr.reshape(nt, nf, P.n_ant, 4)
    if kind == "diag":
        jhj, jhr = jhj[..., [0, 3], :][..., [0, 3]], jhr[..., [0, 3]]
    scale = np.abs(cj).max()
    assert np.abs(jhj - cj).max() <= 1e-12 * scale
    assert np.abs(jhr - cr).max() <= 1e-12 * np.abs(cr).max()
    chi = moments.chi2_from_moments_full(S, Tm, U, g.reshape(nt * nf, P.n_ant, 4))
    want = O.residual(P, [T])
    assert abs(chi - want) <= 1e-12 * want
