"""Batched persistent solver (one launch, many independent intervals) against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from oracle.gauge import reference_diag, rel_err
from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu


def small_batch(n=24, seed_base=50, **kw):
    shapes = synth.batch_shapes(n, seed_base=seed_base, ant=(3, 12), times=(1, 4), chans=(1, 40), flag_max=0.5)
    return synth.make_batch(shapes, **kw)


def solver_of(b, **kw):
    return qc.BatchSolver(b.data, b.model, b.weight, b.flag, b.ant1, b.ant2, b.row_offset, b.vis_offset, b.n_chan,
                          b.n_ant, **kw)


def oracle_problem(b, i):
    r0, r1 = b.row_offset[i], b.row_offset[i + 1]
    v0, v1 = b.vis_offset[i], b.vis_offset[i + 1]
    nc = int(b.n_chan[i])
    rows = int(r1 - r0)
    P = O.OracleProblem(np.asarray(b.data[v0:v1]).reshape(rows, nc, 4), np.asarray(b.model[v0:v1]).reshape(rows, nc, 4),
                        np.asarray(b.weight[v0:v1]).reshape(rows, nc, 4), np.asarray(b.flag[v0:v1]).reshape(rows, nc),
                        b.ant1[r0:r1], b.ant2[r0:r1], np.zeros(rows, np.int32), int(b.n_ant[i]), 1)
    return P


def oracle_solve(b, i, max_iter=20, tol=1e-6):
    P = oracle_problem(b, i)
    T = O.OracleTerm("diag", np.zeros(1, np.int32), np.zeros(int(b.n_chan[i]), np.int32), 1, 1, int(b.n_ant[i]),
                     max_iter=max_iter, tol=tol)
    it = O.solve(P, [T], damping_mode=1)[0]
    return T, int(it[0, 0]), O.residual(P, [T])


def sub_batch(b, i):
    """Problem i of a host batch as a batch of its own."""
    r0, r1 = int(b.row_offset[i]), int(b.row_offset[i + 1])
    v0, v1 = int(b.vis_offset[i]), int(b.vis_offset[i + 1])
    return synth.Batch(b.shapes[i:i + 1], b.data[v0:v1], b.model[v0:v1], b.weight[v0:v1], b.flag[v0:v1],
                       b.ant1[r0:r1], b.ant2[r0:r1], np.array([0, r1 - r0], np.int64), np.array([0, v1 - v0], np.int64),
                       b.n_chan[i:i + 1], b.n_ant[i:i + 1], [], [])


def gains_of(b, g, i):
    o = b.n_ant[:i].sum()
    gi = np.zeros((int(b.n_ant[i]), 4), np.complex128)
    gi[:, 0] = g[o:o + b.n_ant[i], 0]
    gi[:, 3] = g[o:o + b.n_ant[i], 1]
    return gi


def compare(b, g, flags, iters, tol=1e-4, it_slack=2):
    offs = np.concatenate([[0], np.cumsum(b.n_ant)])
    for i in range(b.n_prob):
        T, it, _ = oracle_solve(b, i)
        of = T.gain_flags[0, 0]
        gf = flags[offs[i]:offs[i + 1]]
        assert np.array_equal(gf, of), (i, gf, of)
        good = np.where(of == 0)[0]
        if good.size < 2:
            continue
        want = reference_diag(T.params[0, 0][good][None])[0]
        got = reference_diag(gains_of(b, g, i)[good][None])[0]
        assert rel_err(got, want) < tol, (i, rel_err(got, want))
        assert abs(int(iters[i]) - it) <= it_slack, (i, iters[i], it)


def test_batch_matches_oracle_per_problem():
    b = small_batch()
    S = solver_of(b)
    g, flags, iters, st = S.solve()
    compare(b, g, flags, iters)
    assert st.vis_iters > 0 and st.grid >= 1
    S.close()


@pytest.mark.parametrize("schedule", [qc.QC_SCHED_LPT, qc.QC_SCHED_STATIC])
@pytest.mark.parametrize("threads,depth", [(64, 3), (256, 4), (512, 4), (256, 6)])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_launch_shapes_agree(schedule, threads, depth, use_graph):
    b = small_batch(n=16, seed_base=80)
    S = solver_of(b)
    ref, _, _, _ = S.solve(schedule=qc.QC_SCHED_LPT, threads=128, use_graph=False)
    g, _, _, st = S.solve(schedule=schedule, threads=threads, use_graph=use_graph, depth=depth)
    assert st.threads == threads and st.schedule == schedule and st.depth == depth
    assert np.max(np.abs(g - ref)) < 1e-5
    S.close()


@pytest.mark.parametrize("depth", [3, 6])
def test_batch_large_problems_match_oracle(depth):
    """Problems of 24 and 40 antennas over up to 64 channels: thousands of 32-sample steps per
    problem, split across every warp of the CTA, steps straddling rows (n_chan not a multiple
    of 32), ragged last steps, per-sample flags."""
    shapes = [(900, 40, 6, 64, 0.3), (901, 24, 5, 45, 0.1), (902, 33, 3, 7, 0.45), (903, 24, 2, 1, 0.0)]
    b = synth.make_batch(shapes)
    S = solver_of(b)
    g, flags, iters, st = S.solve(threads=512 if depth == 3 else 256, depth=depth)
    S.close()
    compare(b, g, flags, iters)


def test_batch_fully_flagged_and_autocorrelation_rows():
    """A problem whose samples are all flagged keeps its gains and flags every antenna; rows
    with ant1 == ant2 are skipped."""
    b = small_batch(n=6, seed_base=700)
    flag = np.asarray(b.flag).copy()
    flag[b.vis_offset[2]:b.vis_offset[3]] = 1
    b.flag = flag
    a2 = b.ant2.copy()
    a2[b.row_offset[4]] = b.ant1[b.row_offset[4]]          # first row of problem 4 becomes an autocorrelation
    b.ant2 = a2
    S = solver_of(b)
    g0 = S.unit_gains()
    g, flags, iters, _ = S.solve(g0.copy())
    S.close()
    offs = np.concatenate([[0], np.cumsum(b.n_ant)])
    assert np.all(flags[offs[2]:offs[3]] == 1)
    assert np.array_equal(g[offs[2]:offs[3]], g0[offs[2]:offs[3]])
    compare(sub_batch(b, 4), g[offs[4]:offs[5]], flags[offs[4]:offs[5]], iters[4:5])


# ---------------------------------------------------------------------------
# the same solve from per-baseline sufficient statistics (qc_batch_solve_moments)
# ---------------------------------------------------------------------------

def test_moments_solve_matches_oracle_per_problem():
    b = small_batch(n=24, seed_base=900)
    S = solver_of(b)
    g, flags, iters, st = S.solve(moments=True)
    S.close()
    compare(b, g, flags, iters)
    assert st.vis_iters > 0


@pytest.mark.parametrize("m16", [False, True])
def test_moments_solve_matches_the_sample_solve(m16):
    """Both solves form the same normal equations (the sums in another order), so they reach the
    same gains within the solver tolerance and the same iteration counts within two (the slack of
    the oracle comparisons: float32 sums in another order can move an interval across its
    tolerance by an iteration either way)."""
    b = small_batch(n=48, seed_base=950)
    S = solver_of(b, model_fp16=m16)
    g1, f1, it1, _ = S.solve()
    g2, f2, it2, s2 = S.solve(moments=True)
    S.close()
    assert np.array_equal(f1, f2)
    offs = np.concatenate([[0], np.cumsum(b.n_ant)])
    for i in range(b.n_prob):
        good = np.where(f1[offs[i]:offs[i + 1]] == 0)[0]
        if good.size < 2:
            continue
        a = reference_diag(gains_of(b, g1, i)[good][None])[0]
        c = reference_diag(gains_of(b, g2, i)[good][None])[0]
        assert rel_err(c, a) < 1e-4, (i, rel_err(c, a))
    d = np.abs(it1.astype(int) - it2.astype(int))
    two = np.nonzero(d == 2)[0]
    print(f"\niteration-count differences (sample vs moments, m16={m16}): "
          f"{np.bincount(d, minlength=3).tolist()} for |d| = 0, 1, 2 ...; |d| = 2 at problems "
          f"{[(int(i), int(it1[i]), int(it2[i])) for i in two]}")
    assert d.max() <= 2 and two.size <= 2
    # one pass over the data instead of one per iteration
    assert s2.bytes * 2 < s2.vis_iters * 64


def test_moments_solve_fully_flagged_and_autocorrelations():
    b = small_batch(n=6, seed_base=710)
    flag = np.asarray(b.flag).copy()
    flag[b.vis_offset[2]:b.vis_offset[3]] = 1
    b.flag = flag
    a2 = b.ant2.copy()
    a2[b.row_offset[4]] = b.ant1[b.row_offset[4]]
    b.ant2 = a2
    S = solver_of(b)
    g0 = S.unit_gains()
    g, flags, iters, _ = S.solve(g0.copy(), moments=True)
    S.close()
    offs = np.concatenate([[0], np.cumsum(b.n_ant)])
    assert np.all(flags[offs[2]:offs[3]] == 1)
    assert np.array_equal(g[offs[2]:offs[3]], g0[offs[2]:offs[3]])
    compare(b, g, flags, iters)


def test_size_split_matches_oracle_and_the_single_class_solve():
    """A size threshold splits the batch into concurrent launches of large and small CTAs; every
    problem's result equals the single-class solve's and the oracle's."""
    b = small_batch(n=40, seed_base=300)
    samples = np.diff(b.vis_offset)
    split = int(np.median(samples))
    S = solver_of(b)
    g1, f1, it1, st1 = S.solve(split=-1)
    g2, f2, it2, st2 = S.solve(split=split, small_threads=64, small_ctas_per_sm=4)
    assert st1.split <= 0 and st1.n_small == 0
    assert st2.split == split and st2.n_small == int(np.sum(samples < split)) > 0
    assert st2.small_threads == 64 and st2.small_ctas_per_sm == 4
    # CTAs of another size add the FP32 per-sample terms in another order, so the two solves agree
    # to the bound of the launch-shape test above (1e-5), not bit for bit (seen: 1.4e-6), and an
    # interval whose last relative change lies at the tolerance may stop one iteration apart
    assert np.array_equal(f1, f2) and np.max(np.abs(it1.astype(int) - it2.astype(int))) <= 1
    np.testing.assert_allclose(g2, g1, rtol=0, atol=1e-5)
    compare(b, g2, f2, it2)
    S.close()


def test_autotune_chooses_a_shape_caches_it_per_shape_class_and_matches_oracle():
    b = small_batch(n=48, seed_base=400)
    S = solver_of(b)
    best, n_tried = S.autotune()
    assert n_tried >= 20
    assert best.threads in (128, 256, 512) and best.depth in (3, 4, 6) and best.ms > 0
    # a solve that leaves the shape to the tuner uses the tuned one
    g, flags, iters, st = S.solve(use_graph=False)
    assert (st.threads, st.ctas_per_sm, st.depth, st.split) == (best.threads, best.ctas_per_sm, best.depth,
                                                                best.split)
    compare(b, g, flags, iters)
    S.close()
    # another batch of the same shape class (the same problems) reuses the cached shape untuned
    S2 = solver_of(b)
    g2, flags2, iters2, st2 = S2.solve(use_graph=False)
    assert (st2.threads, st2.ctas_per_sm, st2.depth, st2.split, st2.small_threads) == \
        (st.threads, st.ctas_per_sm, st.depth, st.split, st.small_threads)
    assert np.array_equal(flags2, flags)
    S2.close()
    # a batch of another shape class does not
    other = small_batch(n=12, seed_base=500)
    S3 = solver_of(other)
    _, _, _, st3 = S3.solve(use_graph=False)
    assert st3.threads == 256 and st3.split <= 0
    S3.close()


def test_skewed_batch_one_large_problem():
    """One problem of about 2e6 samples (64 antennas, 16 times x 62 channels) among 63 small ones:
    the batched launch solves it correctly (the same gains as qc_solve's per-sample path on that
    interval, the small ones against the oracle), and since a problem never spans CTAs the large
    one sets the launch's duration (printed beside the launch without it)."""
    import time
    small = synth.batch_shapes(63, seed_base=1300, ant=(3, 10), times=(1, 3), chans=(1, 24), flag_max=0.3)
    shapes = [(1299, 64, 16, 62, 0.1)] + list(small)
    b = synth.make_batch(shapes)
    S = solver_of(b)
    t0 = time.perf_counter()
    g, flags, iters, st = S.solve()
    t_all = time.perf_counter() - t0
    S.close()
    rest = synth.make_batch(list(small))
    S2 = solver_of(rest)
    t0 = time.perf_counter()
    S2.solve()
    t_rest = time.perf_counter() - t0
    S2.close()
    print(f"\nskewed batch: {t_all * 1e3:.1f} ms with the 2e6-sample problem, {t_rest * 1e3:.1f} ms without")
    # the large problem against qc_solve on the same interval
    r1, v1 = int(b.row_offset[1]), int(b.vis_offset[1])
    nc, na = int(b.n_chan[0]), int(b.n_ant[0])
    rows = r1
    one = qc.Solver(np.asarray(b.data[:v1]).reshape(rows, nc, 4).astype(np.complex64),
                    np.asarray(b.model[:v1]).reshape(rows, nc, 4).astype(np.complex64),
                    np.asarray(b.weight[:v1]).reshape(rows, nc, 4).astype(np.float32),
                    np.asarray(b.flag[:v1]).reshape(rows, nc), b.ant1[:r1], b.ant2[:r1], np.zeros(rows, np.int32), na, 1)
    t = qc.Term("diag", np.zeros(1, np.int32), np.zeros(nc, np.int32), 1, 1, na, max_iter=20, tol=1e-6)
    one.solve([t], damping_mode=1)
    one.close()
    good = np.where(flags[:na] == 0)[0]
    want = reference_diag(np.asarray(t.gains, np.complex128)[0, 0][good][None])[0]
    got = reference_diag(gains_of(b, g, 0)[good][None])[0]
    assert rel_err(got, want) < 1e-4
    sub = synth.Batch(b.shapes[1:], b.data[v1:], b.model[v1:], b.weight[v1:], b.flag[v1:], b.ant1[r1:], b.ant2[r1:],
                      b.row_offset[1:] - r1, b.vis_offset[1:] - v1, b.n_chan[1:], b.n_ant[1:], [], [])
    compare(sub, g[na:], flags[na:], iters[1:])
