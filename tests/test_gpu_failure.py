"""Failure paths, exercised without faulting the GPU.

* Allocation failure is made on the host: the library's allocation wrapper is told to
  fail its n-th call as cudaMalloc would (qc_test_fail_alloc), without calling it.  Every
  call that meets it must return QC_ENOMEM and free what it had allocated.
* A bounded wait is made to run out: a test hook leaves one ring stage of the bulk-copy
  accumulate kernel without its arrival, so the kernel's wait on that stage's barrier gives
  up after a short limit.  The kernel records the error, waits for its own copies in flight
  and returns; qc_solve reports QC_ETIMEOUT and the same context then solves normally.
"""
import numpy as np
import pytest

import oracle as O
from oracle.gauge import reference_diag, rel_err
from paper_2412_10072_gb300 import qc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GAIN_TOL = 1e-4


@pytest.fixture
def lib():
    lib = qc.load()
    yield lib
    lib.qc_test_fail_alloc(0)
    lib.qc_test_wait_limit(0, -1)


def _oracle_gains(obs, max_iter=20, tol=1e-6):
    P = O.OracleProblem.from_obs(obs)
    T = O.OracleTerm.from_spec(obs.terms[0], obs.n_ant, max_iter=max_iter, tol=tol)
    O.solve(P, [T], damping_mode=1)
    return T.params


def test_create_returns_enomem_at_every_allocation_and_leaks_nothing(lib):
    obs = synth.plain_small(seed=1, noise=0.01)
    torch.cuda.synchronize()
    base = lib.qc_test_live_allocs()
    n_fail = 0
    for n in range(1, 64):
        lib.qc_test_fail_alloc(n)
        try:
            S = qc.Solver.from_obs(obs)
        except qc.QCError as e:
            assert e.code == qc.QC_ENOMEM, e
            assert lib.qc_test_live_allocs() == base, n
            n_fail += 1
            continue
        # n is past the number of allocations create makes: it succeeded
        lib.qc_test_fail_alloc(0)
        S.close()
        assert lib.qc_test_live_allocs() == base
        break
    else:
        pytest.fail("qc_create never succeeded")
    assert n_fail >= 3, n_fail        # host inputs: rows, strips, data, model, weights, ... all fail in turn


def test_solve_returns_enomem_then_the_context_still_solves(lib):
    obs = synth.plain_small(seed=2, noise=0.01)
    torch.cuda.synchronize()
    base0 = lib.qc_test_live_allocs()
    S = qc.Solver.from_obs(obs)
    base = lib.qc_test_live_allocs()
    term = qc.Term.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    lib.qc_test_fail_alloc(1)                      # the first buffer the solve allocates
    with pytest.raises(qc.QCError) as ei:
        S.solve([term])
    assert ei.value.code == qc.QC_ENOMEM
    assert lib.qc_test_live_allocs() <= base + 64  # buffers made before the failure stay with the context
    lib.qc_test_fail_alloc(0)
    term = qc.Term.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    S.solve([term])
    S.close()
    assert lib.qc_test_live_allocs() == base0      # closed: nothing of S remains
    err = rel_err(reference_diag(term.gains.astype(np.complex128)), reference_diag(_oracle_gains(obs)))
    assert err < GAIN_TOL, err


def test_solve_from_sums_returns_enomem_at_every_allocation(lib):
    """The solve from per-(interval, pair) sums allocates its sums and row table in the solve:
    a failure at each allocation in turn gives QC_ENOMEM, the context keeps working, and the
    solve that finally succeeds matches the oracle; closing frees everything."""
    obs = synth.plain_small(seed=3, noise=0.01)
    torch.cuda.synchronize()
    base0 = lib.qc_test_live_allocs()
    S = qc.Solver.from_obs(obs)
    n_fail = 0
    for n in range(1, 64):
        lib.qc_test_fail_alloc(n)
        term = qc.Term.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
        try:
            st = S.solve([term], moments=True)
        except qc.QCError as e:
            assert e.code == qc.QC_ENOMEM, e
            n_fail += 1
            continue
        lib.qc_test_fail_alloc(0)
        break
    else:
        pytest.fail("the solve never succeeded")
    assert n_fail >= 2 and st.pass_ms > 0
    S.close()
    assert lib.qc_test_live_allocs() == base0
    err = rel_err(reference_diag(term.gains.astype(np.complex128)), reference_diag(_oracle_gains(obs)))
    assert err < GAIN_TOL, err


def test_batch_create_returns_enomem_and_leaks_nothing(lib):
    shapes = [(100 + i, 7 + i, 2, 8, 0.1) for i in range(4)]
    b = synth.make_batch(shapes)
    torch.cuda.synchronize()
    base = lib.qc_test_live_allocs()
    for n in (1, 2, 3):
        lib.qc_test_fail_alloc(n)
        with pytest.raises(qc.QCError) as ei:
            qc.BatchSolver(b.data, b.model, b.weight, b.flag, b.ant1, b.ant2, b.row_offset, b.vis_offset, b.n_chan,
                           b.n_ant)
        assert ei.value.code == qc.QC_ENOMEM
        assert lib.qc_test_live_allocs() == base
    lib.qc_test_fail_alloc(0)
    B = qc.BatchSolver(b.data, b.model, b.weight, b.flag, b.ant1, b.ant2, b.row_offset, b.vis_offset, b.n_chan,
                       b.n_ant)
    B.close()
    assert lib.qc_test_live_allocs() == base


@pytest.mark.parametrize("kernel", [1, 4, 5])
@pytest.mark.parametrize("order", [0, 1])
def test_bounded_wait_gives_up_with_etimeout_and_the_context_recovers(lib, order, kernel):
    obs = synth.plain_small(seed=3, noise=0.01)
    S = qc.Solver.from_obs(obs)
    lib.qc_test_wait_limit(2_000_000, 0)           # 2 ms; every warp's first stage is never filled
    term = qc.Term.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    with pytest.raises(qc.QCError) as ei:
        S.solve([term], kernel=kernel, order=order, use_graph=False)
    assert ei.value.code == qc.QC_ETIMEOUT
    lib.qc_test_wait_limit(0, -1)
    torch.cuda.synchronize()                       # the context and the device are still usable
    term = qc.Term.from_spec(obs.terms[0], obs.n_ant, max_iter=20, tol=1e-6)
    S.solve([term], kernel=kernel, order=order)
    S.close()
    err = rel_err(reference_diag(term.gains.astype(np.complex128)), reference_diag(_oracle_gains(obs)))
    assert err < GAIN_TOL, err
