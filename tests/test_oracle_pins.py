"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against
finite differences of its forward model, a closed form, an invariant, data
ratios, or exact recovery of gains that the independent generator used.
"""
import numpy as np
import pytest

import oracle as O
from oracle.gauge import chain_products, reference_chain, reference_diag, rel_err
from paper_2412_10072_gb300 import synth

GOLDEN_P = np.loadtxt(__file__.replace("test_oracle_pins.py", "golden/permutation_P.txt"))
PERM = [int(np.argmax(r)) for r in GOLDEN_P]          # index form of Eq. permutation


# ---------------------------------------------------------------------------
# helpers: a small random problem with a three-term chain
# ---------------------------------------------------------------------------

def random_problem(seed, n_ant=3, n_time=2, n_chan=3, flag_frac=0.2, kinds=("diag", "full", "phase"),
                   n_bins=(1, 1)):
    rng = np.random.default_rng(seed)
    p, q = synth.baselines(n_ant)
    ant1 = np.tile(p, n_time)
    ant2 = np.tile(q, n_time)
    tidx = np.repeat(np.arange(n_time, dtype=np.int32), p.size)
    n_row = ant1.size
    shp = (n_row, n_chan, 4)
    data = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    model = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)      # polarised, generic
    weight = rng.uniform(0.5, 2.0, size=shp)
    flag = (rng.random((n_row, n_chan)) < flag_frac).astype(np.uint8)
    prob = O.OracleProblem(data, model, weight, flag, ant1, ant2, tidx, n_ant, n_time)
    terms = []
    nt, nf = n_bins
    for kind in kinds:
        tm = (np.arange(n_time) * nt // n_time).astype(np.int32)
        fm = (np.arange(n_chan) * nf // n_chan).astype(np.int32)
        if kind == "phase":
            par = rng.uniform(-np.pi, np.pi, size=(nt, nf, n_ant, 2))
        else:
            par = 1.0 + 0.3 * (rng.standard_normal((nt, nf, n_ant, 4)) + 1j * rng.standard_normal((nt, nf, n_ant, 4)))
        terms.append(O.OracleTerm(kind, tm, fm, nt, nf, n_ant, params=par))
    return prob, terms


def residual_vector(prob, terms):
    _, r = O.residual(prob, terms, want_resid=True)
    return r.reshape(-1)


def sample_weights(prob):
    w = prob.weight.copy()
    w[prob.flag.astype(bool)] = 0.0
    w[prob.ant1 == prob.ant2] = 0.0
    return w.reshape(-1)


def fd_blocks(prob, terms, n, h=1e-6):
    """Finite-difference JHJ and JHr blocks of term n for every (bin, antenna).

    Complex terms: Wirtinger derivatives d/dg = (d/dx - i d/dy)/2 of the stacked residual
    [r; conj(r)] give the left half of J (Eq. jacobian); the AllJones block is the diagonal
    block of J^H W J (Eq. jhj_entry) and the top half of J^H W r is -JHr (Eq. jhr_entry with
    J = -dv/dg, Eq. jacobian_A).  Phase terms: real derivatives, JHJ = 2 Re(J^H W J),
    JHr = -2 Re(J^H W r) (Eq. jhj_entry_param, Eq. jhwr_entry_param).
    """
    T = terms[n]
    w = sample_weights(prob)
    r0 = residual_vector(prob, terms)
    out_jhj = np.zeros((T.n_tint, T.n_fint, prob.n_ant, T.n_param, T.n_param), dtype=np.complex128)
    out_jhr = np.zeros((T.n_tint, T.n_fint, prob.n_ant, T.n_param), dtype=np.complex128)
    for it in range(T.n_tint):
        for jf in range(T.n_fint):
            for a in range(prob.n_ant):
                if T.kind == "phase":
                    cols = []
                    for k in range(2):
                        base = T.params[it, jf, a, k]
                        T.params[it, jf, a, k] = base + h
                        rp = residual_vector(prob, terms)
                        T.params[it, jf, a, k] = base - h
                        rm = residual_vector(prob, terms)
                        T.params[it, jf, a, k] = base
                        cols.append((rp - rm) / (2 * h))
                    Jr = np.stack(cols, axis=1)
                    out_jhj[it, jf, a] = 2 * np.real(Jr.conj().T @ (w[:, None] * Jr))
                    out_jhr[it, jf, a] = -2 * np.real(Jr.conj().T @ (w * r0))
                    continue
                elems = [0, 3] if T.kind == "diag" else [0, 1, 2, 3]
                Jul, Jll = [], []
                for k in elems:
                    base = T.params[it, jf, a, k]
                    d = []
                    for step in (h, 1j * h):
                        T.params[it, jf, a, k] = base + step
                        rp = residual_vector(prob, terms)
                        T.params[it, jf, a, k] = base - step
                        rm = residual_vector(prob, terms)
                        T.params[it, jf, a, k] = base
                        d.append((rp - rm) / (2 * h))
                    dx, dy = d
                    Jul.append(0.5 * (dx - 1j * dy))                   # dr/dg
                    Jll.append(np.conj(0.5 * (dx + 1j * dy)))          # d conj(r)/dg
                Jul = np.stack(Jul, axis=1)
                Jll = np.stack(Jll, axis=1)
                out_jhj[it, jf, a] = Jul.conj().T @ (w[:, None] * Jul) + Jll.conj().T @ (w[:, None] * Jll)
                out_jhr[it, jf, a] = -(Jul.conj().T @ (w * r0) + Jll.conj().T @ (w * np.conj(r0)))
    return out_jhj, out_jhr


# ---------------------------------------------------------------------------
# finite-difference Jacobians (3 antennas, every term type, every chain position)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2])
@pytest.mark.parametrize("kinds", [("diag", "full", "phase"), ("full", "phase", "diag"), ("phase", "diag", "full")])
def test_normal_equations_match_finite_differences(n, kinds):
    prob, terms = random_problem(seed=11 + n, kinds=kinds, n_bins=(2, 2), n_time=2, n_chan=4)
    jhj, jhr = O.normal_equations(prob, terms, n)
    fj, fr = fd_blocks(prob, terms, n)
    scale_j = np.max(np.abs(fj))
    scale_r = np.max(np.abs(fr))
    assert np.max(np.abs(jhj - fj)) <= 1e-7 * scale_j
    assert np.max(np.abs(jhr - fr)) <= 1e-7 * scale_r


def test_phase_jhr_is_minus_chi2_gradient():
    prob, terms = random_problem(seed=5, kinds=("full", "phase"), n_bins=(1, 1))
    _, jhr = O.normal_equations(prob, terms, 1)
    h = 1e-6
    T = terms[1]
    for a in range(prob.n_ant):
        for k in range(2):
            base = T.params[0, 0, a, k]
            T.params[0, 0, a, k] = base + h
            cp = O.residual(prob, terms)
            T.params[0, 0, a, k] = base - h
            cm = O.residual(prob, terms)
            T.params[0, 0, a, k] = base
            grad = (cp - cm) / (2 * h)
            assert abs(jhr[0, 0, a, k].real + grad) <= 1e-6 * max(1.0, abs(grad))


@pytest.mark.parametrize("kind", ["diag", "full"])
def test_complex_jhr_is_minus_wirtinger_gradient(kind):
    """JHr = -d chi^2 / d conj(g) with d/d conj(g) = (d/dx + i d/dy)/2."""
    prob, terms = random_problem(seed=9, kinds=(kind,), n_bins=(1, 1))
    _, jhr = O.normal_equations(prob, terms, 0)
    T = terms[0]
    h = 1e-6
    elems = [0, 3] if kind == "diag" else [0, 1, 2, 3]
    for a in range(prob.n_ant):
        for col, k in enumerate(elems):
            base = T.params[0, 0, a, k]
            g = []
            for step in (h, 1j * h):
                T.params[0, 0, a, k] = base + step
                cp = O.residual(prob, terms)
                T.params[0, 0, a, k] = base - step
                cm = O.residual(prob, terms)
                T.params[0, 0, a, k] = base
                g.append((cp - cm) / (2 * h))
            wirt = 0.5 * (g[0] + 1j * g[1])
            assert abs(jhr[0, 0, a, col] + wirt) <= 1e-6 * max(1.0, abs(wirt))


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2])
def test_jhj_blocks_are_hermitian_psd(n):
    prob, terms = random_problem(seed=21, n_ant=5, n_time=3, n_chan=5, n_bins=(2, 3))
    jhj, _ = O.normal_equations(prob, terms, n)
    blocks = jhj.reshape(-1, jhj.shape[-1], jhj.shape[-1])
    for B in blocks:
        assert np.allclose(B, B.conj().T, rtol=0, atol=1e-12 * max(1.0, np.abs(B).max()))
        ev = np.linalg.eigvalsh(0.5 * (B + B.conj().T))
        assert ev.min() >= -1e-12 * max(1.0, np.abs(B).max())


@pytest.mark.parametrize("n", [0, 1, 2])
@pytest.mark.parametrize("kinds", [("diag", "full", "diag"), ("full", "diag", "full")])
def test_jhr_plus_jhj_g_does_not_depend_on_the_blocks_own_gains(n, kinds):
    """The model of a sample is linear in the solved gains of either of its antennas (V = E g_p,
    with E free of g_p), so JHr_p + JHJ_p g_p = J^H W d (Eq. jhr_entry_simplified with
    r = d - E g_p) is the same for any g_p while the other gains stay fixed; the streaming
    kernels sum J^H W d and form JHr in the update from this identity.  Another antenna's
    block, whose E holds g_p, does change."""
    prob, terms = random_problem(seed=31 + n, n_ant=4, n_time=2, n_chan=4, kinds=kinds, n_bins=(1, 2))
    T = terms[n]
    cols = [0, 3] if T.kind == "diag" else [0, 1, 2, 3]
    rng = np.random.default_rng(7 + n)
    jhj0, jhr0 = O.normal_equations(prob, terms, n)
    scale = max(np.abs(jhj0).max(), np.abs(jhr0).max())
    for it, jf, a, b in [(0, 0, 1, 2), (0, 1, 3, 0)]:
        g0 = T.params[it, jf, a, cols].copy()
        before_a = jhr0[it, jf, a] + jhj0[it, jf, a] @ g0
        before_b = jhr0[it, jf, b] + jhj0[it, jf, b] @ T.params[it, jf, b, cols]
        T.params[it, jf, a, cols] = g0 + 0.5 * (rng.standard_normal(len(cols)) + 1j * rng.standard_normal(len(cols)))
        jhj1, jhr1 = O.normal_equations(prob, terms, n)
        after_a = jhr1[it, jf, a] + jhj1[it, jf, a] @ T.params[it, jf, a, cols]
        after_b = jhr1[it, jf, b] + jhj1[it, jf, b] @ T.params[it, jf, b, cols]
        T.params[it, jf, a, cols] = g0
        assert np.max(np.abs(jhj1[it, jf, a] - jhj0[it, jf, a])) <= 1e-12 * scale
        assert np.max(np.abs(after_a - before_a)) <= 1e-10 * scale
        assert np.max(np.abs(after_b - before_b)) > 1e-3 * scale


def _swap_rows(prob, rows):
    """Swap ant1/ant2 of the given rows: D, M -> D^H, M^H and weights permuted by P (Eq. permutation)."""
    data, model, weight = prob.data.copy(), prob.model.copy(), prob.weight.copy()
    a1, a2 = prob.ant1.copy(), prob.ant2.copy()
    for r in rows:
        data[r] = np.conj(data[r][:, PERM])
        model[r] = np.conj(model[r][:, PERM])
        weight[r] = weight[r][:, PERM]
        a1[r], a2[r] = prob.ant2[r], prob.ant1[r]
    return O.OracleProblem(data, model, weight, prob.flag, a1, a2, prob.time_idx, prob.n_ant, prob.n_time)


@pytest.mark.parametrize("n", [0, 1, 2])
def test_invariant_to_row_order_and_baseline_orientation(n):
    prob, terms = random_problem(seed=31, n_ant=4, n_time=3, n_chan=4, n_bins=(2, 2))
    j0, r0 = O.normal_equations(prob, terms, n)
    c0 = O.residual(prob, terms)
    perm = np.random.default_rng(0).permutation(prob.n_row)
    pp = O.OracleProblem(prob.data[perm], prob.model[perm], prob.weight[perm], prob.flag[perm],
                         prob.ant1[perm], prob.ant2[perm], prob.time_idx[perm], prob.n_ant, prob.n_time)
    j1, r1 = O.normal_equations(pp, terms, n)
    ps = _swap_rows(prob, rows=range(0, prob.n_row, 2))
    j2, r2 = O.normal_equations(ps, terms, n)
    c2 = O.residual(ps, terms)
    for j, r in ((j1, r1), (j2, r2)):
        assert np.allclose(j, j0, rtol=1e-12, atol=1e-12)
        assert np.allclose(r, r0, rtol=1e-12, atol=1e-12)
    assert abs(c2 - c0) <= 1e-12 * c0


def test_flagged_samples_with_nan_are_ignored():
    prob, terms = random_problem(seed=41, n_ant=4, n_time=3, n_chan=4, flag_frac=0.3)
    j0, r0 = O.normal_equations(prob, terms, 1)
    c0 = O.residual(prob, terms)
    data = prob.data.copy()
    model = prob.model.copy()
    data[prob.flag.astype(bool)] = np.nan
    model[prob.flag.astype(bool)] = np.nan
    pn = O.OracleProblem(data, model, prob.weight, prob.flag, prob.ant1, prob.ant2, prob.time_idx,
                         prob.n_ant, prob.n_time)
    j1, r1 = O.normal_equations(pn, terms, 1)
    assert np.array_equal(j0, j1) and np.array_equal(r0, r1)
    assert O.residual(pn, terms) == c0


def test_all_flagged_antenna_is_flagged_and_unchanged():
    obs = synth.plain_small(seed=3, noise=0.01, n_time=8, n_chan=8)
    obs.flag[(obs.ant1 == 2) | (obs.ant2 == 2)] = 1
    prob = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, max_iter=30)
    g0 = T.params.copy()
    O.solve(prob, [T], damping_mode=1)
    assert np.all(T.gain_flags[:, :, 2] == 1)
    assert np.all(T.gain_flags[:, :, [0, 1, 3, 4, 5, 6]] == 0)
    assert np.array_equal(T.params[:, :, 2], g0[:, :, 2])


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

def test_single_iteration_equals_stefcal_closed_form():
    """L = R = I, one diagonal term, alpha = 1: one step gives the alternating-least-squares
    update g_p = sum conj(y) w d / sum w |y|^2 per correlation, y = M_ij conj(g_q,jj)."""
    obs = synth.plain_small(seed=7, noise=0.05, n_time=4, n_chan=4, t_int=4, f_int=4)
    prob = O.OracleProblem.from_obs(obs)
    rng = np.random.default_rng(1)
    g0 = np.zeros((1, 1, obs.n_ant, 4), dtype=np.complex128)
    g0[..., 0] = 1 + 0.2 * (rng.standard_normal(obs.n_ant) + 1j * rng.standard_normal(obs.n_ant))
    g0[..., 3] = 1 + 0.2 * (rng.standard_normal(obs.n_ant) + 1j * rng.standard_normal(obs.n_ant))
    T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, params=g0, max_iter=1, tol=0.0)
    O.solve(prob, [T], damping=1.0, damping_mode=0)
    num = np.zeros((obs.n_ant, 2), dtype=np.complex128)
    den = np.zeros((obs.n_ant, 2))
    g = g0[0, 0][:, [0, 3]]
    for r in range(obs.n_row):
        p, q = obs.ant1[r], obs.ant2[r]
        D = obs.data[r].reshape(-1, 2, 2)
        M = obs.model[r].reshape(-1, 2, 2)
        W = obs.weight[r].reshape(-1, 2, 2)
        for a, b, Dm, Mm, Wm in ((p, q, D, M, W), (q, p, np.conj(np.swapaxes(D, 1, 2)),
                                                    np.conj(np.swapaxes(M, 1, 2)), np.swapaxes(W, 1, 2))):
            for i in range(2):
                for j in range(2):
                    y = Mm[:, i, j] * np.conj(g[b, j])
                    num[a, i] += np.sum(np.conj(y) * Wm[:, i, j] * Dm[:, i, j])
                    den[a, i] += np.sum(Wm[:, i, j] * np.abs(y) ** 2)
    expect = num / den
    got = T.params[0, 0][:, [0, 3]]
    assert np.allclose(got, expect, rtol=1e-12, atol=1e-12)


def test_three_antenna_closure_relations():
    """Noise-free diagonal gains, unpolarised sky: |g_1|^2 = |R_12 R_13 / R_23| with the
    data/model ratios R_pq = d_pq / m_pq = g_p conj(g_q), and the phase closure of the solution."""
    obs = synth.plain_small(seed=13, noise=0.0, n_ant=3, n_time=4, n_chan=4, t_int=4, f_int=4)
    prob = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, max_iter=400, tol=1e-15)
    O.solve(prob, [T], damping_mode=1)
    g = T.params[0, 0]
    ratio = obs.data[:, 0, [0, 3]] / obs.model[:, 0, [0, 3]]          # row -> (p, q) ratio
    R = {(int(obs.ant1[r]), int(obs.ant2[r])): ratio[r] for r in range(3)}
    for c, k in ((0, 0), (1, 3)):
        R01, R02, R12 = R[(0, 1)][c], R[(0, 2)][c], R[(1, 2)][c]
        assert abs(abs(g[0, k]) ** 2 - abs(R01 * R02 / R12)) < 1e-10
        assert abs(abs(g[1, k]) ** 2 - abs(R01 * R12 / R02)) < 1e-10
        assert abs(abs(g[2, k]) ** 2 - abs(R02 * R12 / R01)) < 1e-10
        # phase of g_p conj(g_q) equals the phase of the data ratio on every baseline
        for (p, q), val in R.items():
            assert abs(np.angle(g[p, k] * np.conj(g[q, k]) / val[c])) < 1e-10


# ---------------------------------------------------------------------------
# exact recovery on noise-free data (generator truths, gauge referenced)
# ---------------------------------------------------------------------------

def test_exact_recovery_diag_small_workload():
    obs = synth.plain_small(seed=0, noise=0.0)
    prob = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, max_iter=500, tol=1e-15)
    O.solve(prob, [T], damping_mode=1)
    assert rel_err(reference_diag(T.params), reference_diag(obs.terms[0].truth)) < 1e-10
    chi2 = O.residual(prob, [T])
    assert chi2 <= 1e-20 * np.sum(np.abs(obs.data) ** 2)
    _, jhr = O.normal_equations(prob, [T], 0)
    assert np.max(np.abs(jhr)) < 1e-9


def test_chi2_is_zero_at_the_truth_for_chains():
    obs = synth.plain_large(seed=2, n_ant=6, n_time=4, n_chan=6, noise=0.0, flag_row_frac=0.2, n_src=4)
    prob = O.OracleProblem.from_obs(obs)
    terms = [O.OracleTerm.from_spec(s, obs.n_ant, params=s.truth) for s in obs.terms]
    assert O.residual(prob, terms) <= 1e-24 * np.sum(np.abs(obs.data) ** 2)
    for n in range(2):
        _, jhr = O.normal_equations(prob, terms, n)
        assert np.max(np.abs(jhr)) < 1e-10


def test_exact_recovery_full_jones():
    rng = np.random.default_rng(4)
    n_ant, n_time, n_chan = 6, 3, 8
    freqs = synth.meerkat_band(n_chan)
    spec = synth.TermSpec("full", synth.interval_map(n_time, 1), np.zeros(n_chan, np.int32), n_time, 1)
    spec.truth = synth.full_truth(n_ant, n_time, 1, rng, leakage=0.1)
    obs = synth.make_observation(n_ant, n_time, freqs, [spec], n_src=6, seed=4, noise=0.0, rng=rng,
                                 max_baseline_m=8000.0)
    prob = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(spec, n_ant, max_iter=600, tol=1e-15)
    O.solve(prob, [T], damping_mode=1)
    got = reference_chain(T.params)
    want = reference_chain(spec.truth)
    assert rel_err(got, want) < 1e-9


def test_exact_recovery_phase_only():
    rng = np.random.default_rng(8)
    n_ant, n_time, n_chan = 5, 4, 4
    freqs = 1.4e9 + 1e6 * np.arange(n_chan)
    spec = synth.TermSpec("phase", synth.interval_map(n_time, 2), synth.interval_map(n_chan, 2), 2, 2)
    spec.truth = 0.4 * rng.standard_normal((2, 2, n_ant, 2))
    obs = synth.make_observation(n_ant, n_time, freqs, [spec], n_src=5, seed=8, noise=0.0, rng=rng)
    prob = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(spec, n_ant, max_iter=300, tol=1e-15)
    O.solve(prob, [T], damping_mode=0, damping=1.0)
    got = reference_diag(T.jones())
    want = reference_diag(synth.phase_to_jones(spec.truth))
    assert rel_err(got, want) < 1e-10


def test_exact_recovery_two_term_chain_products():
    """G (full, per time) then B (diagonal, per channel): the referenced product chain
    G_a(t) B_a(f) converges to the truth over epochs."""
    obs = synth.plain_large(seed=5, n_ant=6, n_time=4, n_chan=6, noise=0.0, flag_row_frac=0.0, n_src=6)
    prob = O.OracleProblem.from_obs(obs)
    terms = [O.OracleTerm.from_spec(s, obs.n_ant, max_iter=200, tol=1e-15) for s in obs.terms]
    O.solve(prob, terms, n_epochs=60, damping_mode=1)
    Cg = chain_products([t.jones() for t in terms], [t.t_map for t in terms], [t.f_map for t in terms],
                        obs.n_time, obs.n_chan)
    Ct = chain_products([s.truth_jones() for s in obs.terms], [s.t_map for s in obs.terms],
                        [s.f_map for s in obs.terms], obs.n_time, obs.n_chan)
    assert rel_err(reference_chain(Cg), reference_chain(Ct)) < 1e-8
    assert O.residual(prob, terms) <= 1e-16 * np.sum(np.abs(obs.data) ** 2)


# ---------------------------------------------------------------------------
# block solve and statistics
# ---------------------------------------------------------------------------

def test_block_solve_against_dense_and_singular_cases():
    rng = np.random.default_rng(2)
    for n in (2, 4):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        A = A @ A.conj().T + n * np.eye(n)
        b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        x, sing = O.block_solve(A, b)
        assert not sing and np.allclose(A @ x, b, rtol=1e-12, atol=1e-12)
    assert O.block_solve(np.zeros((2, 2)), np.ones(2))[1]
    assert O.block_solve(np.array([[1.0, 1.0], [1.0, 1.0]]), np.ones(2))[1]
    assert O.block_solve(np.diag([1.0, 1e-14]), np.ones(2))[1]


def test_chi2_statistics_on_noisy_data():
    """chi^2 / (2 sigma^2 N) ~ 1 - N_params / (2 N) for unit weights (a sanity check)."""
    sigma = 0.01
    obs = synth.plain_small(seed=0, noise=sigma)
    prob = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, max_iter=200, tol=1e-12)
    O.solve(prob, [T], damping_mode=1)
    chi2 = O.residual(prob, [T])
    n_obs = obs.n_row * obs.n_chan * 4
    n_par = 2 * (T.n_tint * T.n_fint * obs.n_ant * 2)
    expect = 2 * sigma ** 2 * n_obs * (1 - n_par / (2 * n_obs))
    sd = 2 * sigma ** 2 * np.sqrt(n_obs)
    assert abs(chi2 - expect) < 5 * sd
