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
@pytest.mark.parametrize("threads", [64, 256, 512])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_launch_shapes_agree(schedule, threads, use_graph):
    b = small_batch(n=16, seed_base=80)
    S = solver_of(b)
    ref, _, _, _ = S.solve(schedule=qc.QC_SCHED_LPT, threads=128, use_graph=False)
    g, _, _, st = S.solve(schedule=schedule, threads=threads, use_graph=use_graph)
    assert st.threads == threads and st.schedule == schedule
    assert np.max(np.abs(g - ref)) < 1e-5
    S.close()


def test_autotune_picks_a_shape_and_keeps_results():
    b = small_batch(n=40, seed_base=120)
    S = solver_of(b)
    before, _, _, _ = S.solve()
    best, n_tried = S.autotune()
    assert n_tried >= 3 and best.ms > 0 and best.threads in (128, 256, 512)
    after, _, _, st = S.solve()
    assert (st.threads, st.ctas_per_sm, st.schedule) == (best.threads, best.ctas_per_sm, best.schedule)
    assert np.max(np.abs(after - before)) < 1e-5
    S.close()


def test_batch_matches_looped_single_problem_solves():
    b = small_batch(n=10, seed_base=200)
    S = solver_of(b)
    g, _, _, _ = S.solve()
    S.close()
    for i in range(b.n_prob):
        r0, r1 = b.row_offset[i], b.row_offset[i + 1]
        v0, v1 = b.vis_offset[i], b.vis_offset[i + 1]
        nc, rows = int(b.n_chan[i]), int(r1 - r0)
        s1 = qc.Solver(b.data[v0:v1].reshape(rows, nc, 4), b.model[v0:v1].reshape(rows, nc, 4),
                       b.weight[v0:v1].reshape(rows, nc, 4), b.flag[v0:v1].reshape(rows, nc), b.ant1[r0:r1],
                       b.ant2[r0:r1], np.zeros(rows, np.int32), int(b.n_ant[i]), 1)
        t = qc.Term("diag", np.zeros(1, np.int32), np.zeros(nc, np.int32), 1, 1, int(b.n_ant[i]))
        s1.solve([t])
        s1.close()
        gi = gains_of(b, g, i)
        assert np.max(np.abs(t.gains[0, 0][:, [0, 3]] - gi[:, [0, 3]])) < 1e-5


def test_batch_residual_matches_oracle():
    b = small_batch(n=12, seed_base=300)
    S = solver_of(b)
    g, _, _, _ = S.solve()
    chi2 = S.residual(g)
    S.close()
    for i in range(b.n_prob):
        P = oracle_problem(b, i)
        T = O.OracleTerm("diag", np.zeros(1, np.int32), np.zeros(int(b.n_chan[i]), np.int32), 1, 1, int(b.n_ant[i]),
                         params=gains_of(b, g, i)[None, None])
        want = O.residual(P, [T])
        assert abs(chi2[i] - want) <= 1e-5 * max(want, 1e-12), (i, chi2[i], want)


def test_batch_on_device_arrays():
    import torch
    shapes = synth.batch_shapes(12, seed_base=400, ant=(3, 10), times=(1, 3), chans=(1, 40))
    host = synth.make_batch(shapes)
    dev = synth.make_batch(shapes, device="cuda:0")
    S = solver_of(dev)
    g0 = torch.ones((S.total_ant, 2), dtype=torch.complex64, device="cuda:0")
    g, flags, iters, st = S.solve(g0)
    S.close()
    # the device generator draws its own noise: compare each problem with the oracle on the device data
    b = synth.Batch(dev.shapes, dev.data.cpu().numpy(), dev.model.cpu().numpy(), dev.weight.cpu().numpy(),
                    dev.flag.cpu().numpy(), dev.ant1, dev.ant2, dev.row_offset, dev.vis_offset, dev.n_chan, dev.n_ant,
                    dev.truths, dev.setups)
    compare(b, g.cpu().numpy(), flags.cpu().numpy(), iters.cpu().numpy())
    assert host.n_vis == dev.n_vis


def test_batch_fp16_model_error_is_bounded():
    """FP16 model storage: the error against the FP64 oracle is set by float16 rounding of the
    model (relative 2^-11 of each baseline's largest component), not by the solver."""
    b = small_batch(n=16, seed_base=500)
    S = solver_of(b, model_fp16=True)
    g, flags, iters, _ = S.solve()
    S.close()
    compare(b, g, flags, iters, tol=3e-3, it_slack=20)
