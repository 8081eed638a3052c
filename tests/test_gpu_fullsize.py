"""The bench's own workload at full size (64 antennas, 300 times x 512 channels, G full
per time then B diagonal per channel, 3 epochs, 10% of rows flagged), solved by the
GPU in the launch configurations bench.py times (per sample, and from per-(interval, pair)
sums), checked on sampled intervals by the FP64 oracle.

The oracle cannot solve 3.1e8 samples in a test, but stationarity holds at any size:
at the GPU's gains, the oracle's Gauss-Newton step JHJ^-1 JHr (Eq. update) of a
sampled interval must be negligible against the gains.  G intervals (one time) are
checked on that time's rows; B intervals (one channel) on that channel of every row.
G was last solved before the last B solve, so its step also carries the B change of
the final epoch; both are held to the gain tolerance 1e-4."""
import numpy as np
import pytest

import oracle as O
from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu

GAIN_TOL = 1e-4


@pytest.fixture(scope="module", params=[False, True], ids=["per_sample", "from_sums"])
def solved(request):
    """The full-size solve as bench.py times it: the per-sample path (the default line) and the
    solve from per-(interval, pair) sums (bench.py --moments)."""
    import torch
    setup = synth.plain_large_setup(seed=1, n_ant=64, n_time=300, n_chan=512)
    obs = synth.make_observation_device(setup, noise=0.05, noise_seed=1000, device="cuda:0")
    S = qc.Solver(obs["data"], obs["model"], obs["weight"], obs["flag"], setup.ant1, setup.ant2, setup.time_idx,
                  setup.n_ant, setup.n_time)
    terms = [qc.Term.from_spec(s, setup.n_ant, max_iter=20, tol=1e-6) for s in setup.terms]
    st = S.solve(terms, n_epochs=3, moments=request.param)
    torch.cuda.synchronize()
    assert (st.pass_ms > 0) == request.param
    yield setup, obs, terms
    S.close()
    del obs
    torch.cuda.empty_cache()


def _step_norms(jhj, jhr, params, kind):
    """|JHJ^-1 JHr| / |g| per (interval, antenna), from the oracle's normal equations."""
    out = []
    for it in np.ndindex(jhj.shape[:3]):
        A, b = jhj[it], jhr[it]
        if not np.all(np.isfinite(A)) or np.real(np.trace(A)) <= 0:
            continue
        x, singular = O.block_solve(A, b)
        if singular:
            continue
        g = params[it][[0, 3]] if kind == "diag" else params[it]
        out.append(np.linalg.norm(x) / np.linalg.norm(g))
    return np.array(out)


def test_sampled_g_intervals_are_stationary(solved):
    setup, obs, terms = solved
    n_bl = setup.n_ant * (setup.n_ant - 1) // 2
    worst = []
    for t in (0, 117, 299):
        rows = slice(t * n_bl, (t + 1) * n_bl)
        P = O.OracleProblem(obs["data"][rows].cpu().numpy(), obs["model"][rows].cpu().numpy(),
                            obs["weight"][rows].cpu().numpy(), obs["flag"][rows].cpu().numpy(),
                            setup.ant1[rows], setup.ant2[rows], np.zeros(n_bl, np.int32), setup.n_ant, 1)
        gG = np.asarray(terms[0].gains, dtype=np.complex128)[t:t + 1]
        gB = np.asarray(terms[1].gains, dtype=np.complex128)
        tG = O.OracleTerm("full", np.zeros(1, np.int32), np.zeros(512, np.int32), 1, 1, setup.n_ant, params=gG)
        tB = O.OracleTerm("diag", np.zeros(1, np.int32), np.arange(512, dtype=np.int32), 1, 512, setup.n_ant,
                          params=gB)
        jhj, jhr = O.normal_equations(P, [tG, tB], 0)
        steps = _step_norms(jhj, jhr, tG.params, "full")
        assert steps.size > 0.9 * setup.n_ant
        worst.append(steps.max())
    assert max(worst) < GAIN_TOL, worst


def test_sampled_b_intervals_are_stationary(solved):
    setup, obs, terms = solved
    worst = []
    for c in (0, 255, 511):
        P = O.OracleProblem(obs["data"][:, c:c + 1].cpu().numpy(), obs["model"][:, c:c + 1].cpu().numpy(),
                            obs["weight"][:, c:c + 1].cpu().numpy(), obs["flag"][:, c:c + 1].cpu().numpy(),
                            setup.ant1, setup.ant2, setup.time_idx, setup.n_ant, setup.n_time)
        gG = np.asarray(terms[0].gains, dtype=np.complex128)
        gB = np.asarray(terms[1].gains, dtype=np.complex128)[:, c:c + 1]
        tG = O.OracleTerm("full", np.arange(300, dtype=np.int32), np.zeros(1, np.int32), 300, 1, setup.n_ant,
                          params=gG)
        tB = O.OracleTerm("diag", np.zeros(300, np.int32), np.zeros(1, np.int32), 1, 1, setup.n_ant, params=gB)
        jhj, jhr = O.normal_equations(P, [tG, tB], 1)
        steps = _step_norms(jhj, jhr, tB.params, "diag")
        assert steps.size > 0.9 * setup.n_ant
        worst.append(steps.max())
    assert max(worst) < GAIN_TOL, worst


def test_full_size_chi2_matches_oracle_on_sampled_rows(solved):
    """chi^2 of the solved chain, restricted to sampled times, from the GPU's qc_residual on those
    rows and from the oracle."""
    setup, obs, terms = solved
    n_bl = setup.n_ant * (setup.n_ant - 1) // 2
    for t in (5, 150):
        rows = slice(t * n_bl, (t + 1) * n_bl)
        args = [obs[k][rows].contiguous() for k in ("data", "model", "weight", "flag")]
        S = qc.Solver(*args, setup.ant1[rows], setup.ant2[rows], np.zeros(n_bl, np.int32), setup.n_ant, 1)
        gG = np.asarray(terms[0].gains)[t:t + 1].copy()
        tg = [qc.Term("full", np.zeros(1, np.int32), np.zeros(512, np.int32), 1, 1, setup.n_ant, gains=gG),
              qc.Term("diag", np.zeros(1, np.int32), np.arange(512, dtype=np.int32), 1, 512, setup.n_ant,
                      gains=np.asarray(terms[1].gains).copy())]
        chi_gpu = S.residual(tg)
        S.close()
        P = O.OracleProblem(*[a.cpu().numpy() for a in args], setup.ant1[rows], setup.ant2[rows],
                            np.zeros(n_bl, np.int32), setup.n_ant, 1)
        to = [O.OracleTerm("full", np.zeros(1, np.int32), np.zeros(512, np.int32), 1, 1, setup.n_ant,
                           params=gG.astype(np.complex128)),
              O.OracleTerm("diag", np.zeros(1, np.int32), np.arange(512, dtype=np.int32), 1, 512, setup.n_ant,
                           params=np.asarray(terms[1].gains, dtype=np.complex128))]
        chi_o = O.residual(P, to)
        assert abs(chi_gpu - chi_o) <= 1e-5 * chi_o, (t, chi_gpu, chi_o)
