"""The exchange hook of a term whose intervals span processes (reduce = 1), on one GPU.

qc_solve hands the term's FP64 accumulator buffer [bins][ant][KG] to the
options' allreduce callback after every accumulate pass and updates from what
the callback leaves there.  A callback that halves the JHr words (KG layout of
a diagonal term: JHJ in words 0..3, JHr in 4..7) must therefore give the same
solve as constant damping alpha = 1/2, which halves every step (Eq. update)."""
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


def test_callback_feeds_the_update():
    import torch
    obs = _obs()
    calls = []

    def halve_jhr(ptr, n, stream, user):
        t = torch.as_tensor(shard._DeviceView(ptr, n), device="cuda")
        with torch.cuda.stream(torch.cuda.ExternalStream(int(stream))):
            t.view(-1, 8)[:, 4:] *= 0.5
        calls.append(int(n))
        return 0

    S = qc.Solver.from_obs(obs)
    ta = _terms(obs, True)
    # the G term (solved first) with alpha = 1/2 as well, so both runs see the same G
    S.solve(ta[:1] + [qc.Term.from_spec(obs.terms[1], obs.n_ant, solve=False)], damping_mode=qc.QC_DAMP_CONST,
            damping=0.5)
    S.solve([qc.Term.from_spec(obs.terms[0], obs.n_ant, gains=ta[0].gains, solve=False), ta[1]],
            damping_mode=qc.QC_DAMP_CONST, damping=1.0, allreduce=halve_jhr)
    S.close()

    S = qc.Solver.from_obs(obs)
    tb = _terms(obs, False)
    S.solve(tb[:1] + [qc.Term.from_spec(obs.terms[1], obs.n_ant, solve=False)], damping_mode=qc.QC_DAMP_CONST,
            damping=0.5)
    S.solve([qc.Term.from_spec(obs.terms[0], obs.n_ant, gains=tb[0].gains, solve=False), tb[1]],
            damping_mode=qc.QC_DAMP_CONST, damping=0.5)
    S.close()

    n_b = obs.terms[1].n_tint * obs.terms[1].n_fint
    assert calls and all(c == n_b * obs.n_ant * 8 for c in calls)
    assert len(calls) == 8          # one exchange per enqueued iteration (max_iter of B)
    np.testing.assert_allclose(np.asarray(ta[1].gains), np.asarray(tb[1].gains), rtol=0, atol=2e-6)
    assert np.array_equal(np.asarray(ta[1].iters), np.asarray(tb[1].iters))


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
