"""Pins of the sufficient-statistics pre-reduction (oracle/moments.py): the normal equations and
chi^2 formed from the per-baseline sums S, T, U equal the oracle's sample-by-sample normal
equations (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified) and chi^2 (Eq. min) of a single
diagonal term, with flags, both row orientations and several solution intervals."""
import numpy as np
import pytest

import oracle as O
from oracle.moments import chi2_from_moments, moments, normal_equations_from_moments
from paper_2412_10072_gb300 import synth


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_moments_give_the_sample_normal_equations_and_chi2(seed):
    rng = np.random.default_rng(seed)
    na, nt, nc = 5, 4, 6
    p, q = synth.baselines(na)
    a1, a2 = np.tile(p, nt), np.tile(q, nt)
    swap = rng.random(a1.size) < 0.5                   # rows in either orientation
    a1, a2 = np.where(swap, a2, a1).astype(np.int32), np.where(swap, a1, a2).astype(np.int32)
    tidx = np.repeat(np.arange(nt, dtype=np.int32), p.size)
    shp = (a1.size, nc, 4)
    d = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    m = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    w = rng.uniform(0.5, 2, shp)
    f = (rng.random(shp[:2]) < 0.2).astype(np.uint8)
    P = O.OracleProblem(d, m, w, f, a1, a2, tidx, na, nt)
    tm = (np.arange(nt) // 2).astype(np.int32)
    par = 1 + 0.3 * (rng.standard_normal((2, 1, na, 4)) + 1j * rng.standard_normal((2, 1, na, 4)))
    K = O.OracleTerm("diag", tm, np.zeros(nc, np.int32), 2, 1, na, params=par)
    jhj, jhr = O.normal_equations(P, [K], 0)
    S, T, U = moments(P, tm, 2)
    g = K.params[:, 0][..., [0, 3]]
    mj, mr = normal_equations_from_moments(S, T, g)
    assert np.abs(jhj[:, 0] - mj).max() <= 1e-13 * np.abs(jhj).max()
    assert np.abs(jhr[:, 0] - mr).max() <= 1e-13 * np.abs(jhr).max()
    chi = O.residual(P, [K])
    assert abs(chi - chi2_from_moments(S, T, U, g)) <= 1e-13 * chi
