"""The exchange hook of a term whose intervals span processes (reduce = 1), on one GPU.

qc_solve hands the term's FP64 accumulator buffer [bins][ant][KG] to the
options' allreduce callback after every accumulate pass and updates from what
the callback leaves there.  The buffer holds sums over samples (JHJ and the
right-hand side of Eq. update, as J^H W r or as J^H W d), so a process group
sums it word by word.  A callback that doubles every word (the sum over two
processes holding the same rows) must give the solve without the exchange: the
step JHJ^-1 JHr is unchanged when JHJ and its right-hand side are scaled
together.  A callback that zeroes every word leaves every block singular."""
import numpy as np
import pytest

from paper_2412_10072_gb300 import qc, shard, synth

pytestmark = pytest.mark.gpu


def _obs():
    return synth.plain_large(seed=4, n_ant=8, n_time=10, n_chan=24, noise=0.05, flag_row_frac=0.1, n_src=6)


def _terms(obs, reduce_b):
    G, B = obs.terms
    return [qc.Term.from_spec(G, obs.n_ant, max_iter=8, tol=1e-7),
            qc.Term.from_spec(B, obs.n_ant, max_iter=8, tol=1e-7, reduce=reduce_b)]


def _solve_g_then_b(obs, terms, **b_opts):
    """G alone, then B with G fixed at the result (both runs see the same G)."""
    S = qc.Solver.from_obs(obs)
    S.solve(terms[:1] + [qc.Term.from_spec(obs.terms[1], obs.n_ant, solve=False)])
    S.solve([qc.Term.from_spec(obs.terms[0], obs.n_ant, gains=terms[0].gains, solve=False), terms[1]], **b_opts)
    S.close()


def _scaling_callback(factor, calls):
    import torch

    def cb(ptr, n, stream, user):
        t = torch.as_tensor(shard._DeviceView(ptr, n), device="cuda")
        with torch.cuda.stream(torch.cuda.ExternalStream(int(stream))):
            t.mul_(factor)
        calls.append(int(n))
        return 0
    return cb


def test_callback_feeds_the_update():
    obs = _obs()
    n_b = obs.terms[1].n_tint * obs.terms[1].n_fint

    calls = []
    ta = _terms(obs, True)
    _solve_g_then_b(obs, ta, allreduce=_scaling_callback(2.0, calls))
    tb = _terms(obs, False)
    _solve_g_then_b(obs, tb)
    assert calls and all(c == n_b * obs.n_ant * 8 for c in calls)
    assert len(calls) == 8          # one exchange per enqueued iteration (max_iter of B)
    np.testing.assert_allclose(np.asarray(ta[1].gains), np.asarray(tb[1].gains), rtol=0, atol=2e-6)
    assert np.array_equal(np.asarray(ta[1].iters), np.asarray(tb[1].iters))
    assert np.array_equal(np.asarray(ta[1].gain_flags), np.asarray(tb[1].gain_flags))

    # the update reads what the callback leaves: all-zero blocks are singular, so every antenna is
    # flagged and keeps its starting gains, and the intervals stop after one iteration
    calls = []
    tz = _terms(obs, True)
    start = np.array(np.asarray(tz[1].gains))
    _solve_g_then_b(obs, tz, allreduce=_scaling_callback(0.0, calls))
    assert calls
    assert np.all(np.asarray(tz[1].gain_flags) == 1)
    assert np.array_equal(np.asarray(tz[1].gains), start)
    assert np.all(np.asarray(tz[1].iters) == 1)


def test_failing_callback_is_an_error_and_the_context_stays_usable():
    obs = _obs()
    S = qc.Solver.from_obs(obs)
    with pytest.raises(qc.QCError):
        S.solve(_terms(obs, True), allreduce=lambda ptr, n, stream, user: 1)
    # a reduce term without a callback is rejected before any work
    with pytest.raises(qc.QCError):
        S.solve(_terms(obs, True))
    t = _terms(obs, False)
    S.solve(t)
    assert np.all(np.isfinite(np.asarray(t[1].gains)))
    S.close()
