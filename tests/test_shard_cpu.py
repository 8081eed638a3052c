"""Time-block sharding across processes (CPU, gloo, world size 2).

Each rank takes its block of times, forms the normal equations of a two-term
chain (G: diagonal per 3 times x 4 channels, local to a block; B: diagonal per
all times x 1 channel, spanning blocks) with the FP64 oracle on its own rows,
sums the spanning term's partial sums with the same exchange the GPU path uses,
and checks both against the single-process normal equations."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2412_10072_gb300 import shard, synth


def test_time_blocks_partition_the_times():
    for n_time in (1, 2, 7, 60, 300):
        for world in range(1, min(n_time, 9) + 1):
            blocks = [shard.time_block(n_time, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n_time
            assert all(b[0] == a[1] for a, b in zip(blocks, blocks[1:]))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        shard.time_block(3, 0, 4)


def test_shard_term_local_and_reduced():
    n_time = 60
    per_time = np.arange(n_time)
    g = [shard.shard_term(per_time, n_time, n_time, 4, r) for r in range(4)]
    assert not any(s.reduce for s in g)
    assert [s.tint_offset for s in g] == [0, 15, 30, 45] and all(s.n_tint == 15 for s in g)
    assert np.array_equal(g[1].t_map, np.arange(15))
    whole = np.zeros(n_time, np.int32)
    b = [shard.shard_term(whole, 1, n_time, 4, r) for r in range(4)]
    assert all(s.reduce and s.n_tint == 1 and s.tint_offset == 0 for s in b)
    # intervals of 4 times: aligned with 3 blocks of 20 (local), not with 7 blocks (reduced)
    four = np.arange(n_time) // 4
    assert not shard.shard_term(four, 15, n_time, 3, 1).reduce
    assert shard.shard_term(four, 15, n_time, 7, 1).reduce
    # an interval made of times in two blocks is reduced even when the boundary times differ
    mixed = np.array([0, 1, 0, 1])
    assert shard.shard_term(mixed, 2, 4, 2, 0).reduce


def _problem():
    obs = synth.plain_small(seed=3, n_time=12, n_chan=8, t_int=3)
    rng = np.random.default_rng(5)
    n_ant = obs.n_ant
    G = O.OracleTerm("diag", np.arange(12) // 3, np.arange(8) // 4, 4, 2, n_ant, params=obs.terms[0].truth.copy())
    gb = np.zeros((1, 8, n_ant, 4), np.complex128)
    gb[..., 0] = 1 + 0.1 * (rng.standard_normal((1, 8, n_ant)) + 1j * rng.standard_normal((1, 8, n_ant)))
    gb[..., 3] = 1 + 0.1 * (rng.standard_normal((1, 8, n_ant)) + 1j * rng.standard_normal((1, 8, n_ant)))
    return obs, G, gb


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        obs, G, gb = _problem()
        n_time, n_ant = obs.n_time, obs.n_ant
        rows_arrays = dict(data=obs.data, model=obs.model, weight=obs.weight, flag=obs.flag, ant1=obs.ant1,
                           ant2=obs.ant2)
        loc, (t0, t1), _ = shard.shard_observation(rows_arrays, obs.time_idx, n_time, world, rank)
        P = O.OracleProblem(loc["data"], loc["model"], loc["weight"], loc["flag"], loc["ant1"], loc["ant2"],
                            loc["time_idx"], n_ant, t1 - t0)
        sg = shard.shard_term(np.arange(n_time) // 3, 4, n_time, world, rank)
        sb = shard.shard_term(np.zeros(n_time, np.int32), 1, n_time, world, rank)
        full_g = np.array(G.params)
        Gl = O.OracleTerm("diag", sg.t_map, np.arange(8) // 4, sg.n_tint, 2, n_ant,
                          params=full_g[sg.tint_offset:sg.tint_offset + sg.n_tint].copy())
        B = O.OracleTerm("diag", sb.t_map, np.arange(8), 1, 8, n_ant, params=gb.copy())
        jhj_g, jhr_g = O.normal_equations(P, [Gl, B], 0)
        jhj_b, jhr_b = O.normal_equations(P, [Gl, B], 1)
        buf = torch.from_numpy(np.concatenate([jhj_b.view(np.float64).ravel(), jhr_b.view(np.float64).ravel()]))
        shard.allreduce_inplace(buf, None, None)
        # the right-hand side as the streaming kernel sums it: J^H W d = JHr + JHJ g per block
        wd = torch.from_numpy(np.ascontiguousarray((jhr_b + np.einsum("...ij,...j->...i", jhj_b, gb[..., [0, 3]]))
                                                   .view(np.float64).ravel()))
        shard.allreduce_inplace(wd, None, None)
        q.put((rank, sg.reduce, sb.reduce, sg.tint_offset, sg.n_tint, jhj_g, jhr_g, buf.numpy(), wd.numpy()))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_ranks_sum_to_the_single_process_normal_equations():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    obs, G, gb = _problem()
    P = O.OracleProblem(obs.data, obs.model, obs.weight, obs.flag, obs.ant1, obs.ant2, obs.time_idx, obs.n_ant,
                        obs.n_time)
    B = O.OracleTerm("diag", np.zeros(obs.n_time, np.int32), np.arange(8), 1, 8, obs.n_ant, params=gb.copy())
    jhj_g, jhr_g = O.normal_equations(P, [G, B], 0)
    jhj_b, jhr_b = O.normal_equations(P, [G, B], 1)
    want_b = np.concatenate([jhj_b.view(np.float64).ravel(), jhr_b.view(np.float64).ravel()])
    scale = np.abs(want_b).max()
    # J^H W d summed over ranks, less the summed JHJ times the gains, is the single-process JHr
    wd_sum = res[0][8].view(np.complex128).reshape(jhr_b.shape)
    jhj_sum = res[0][7][:jhj_b.size * 2].view(np.complex128).reshape(jhj_b.shape)
    got = wd_sum - np.einsum("...ij,...j->...i", jhj_sum, gb[..., [0, 3]])
    np.testing.assert_allclose(got, jhr_b, rtol=0, atol=1e-10 * scale)
    for rank, g_red, b_red, off, n_t, jg, rg, buf, _ in res:
        assert not g_red and b_red
        # the local term: the rank's slice of the single-process normal equations, exactly
        np.testing.assert_allclose(jg, jhj_g[off:off + n_t], rtol=1e-12, atol=1e-12 * np.abs(jhj_g).max())
        np.testing.assert_allclose(rg, jhr_g[off:off + n_t], rtol=1e-12, atol=1e-12 * np.abs(jhr_g).max())
        # the spanning term: the sum over ranks equals the single-process sums (to FP64 reordering)
        np.testing.assert_allclose(buf, want_b, rtol=1e-12, atol=1e-12 * scale)
    assert res[0][3] == 0 and res[1][3] == res[0][4]


def test_bench_shards_one_observation_by_time_block():
    """The benchmark's multi-GPU mode: every rank takes a block of the one observation's times
    (together all rows once), solves G on its own intervals and B over all of them with reduce."""
    import bench
    from paper_2412_10072_gb300 import qc
    setup = synth.plain_large_setup(seed=1, n_ant=6, n_time=10, n_chan=8, flag_row_frac=0.1, n_src=3)
    for world in (2, 3):
        seen = []
        g_ints = []
        for rank in range(world):
            sub, local_time, n_local = bench.shard_setup(setup, world, rank)
            t0, t1 = shard.time_block(setup.n_time, rank, world)
            assert n_local == t1 - t0 and np.all((local_time >= 0) & (local_time < n_local))
            assert np.array_equal(sub.time_idx - t0, local_time)
            seen.append(np.nonzero((setup.time_idx >= t0) & (setup.time_idx < t1))[0])
            assert np.array_equal(sub.ant1, setup.ant1[seen[-1]]) and np.array_equal(sub.uvw, setup.uvw[seen[-1]])
            G, B = bench.make_terms(qc, setup, setup.n_ant, 5, world, rank)
            assert not G.reduce and G.n_tint == n_local and np.array_equal(G.t_map, np.arange(n_local))
            assert B.reduce and B.n_tint == 1 and B.n_fint == 8
            g_ints.append(G.n_tint)
        assert np.array_equal(np.sort(np.concatenate(seen)), np.arange(setup.ant1.size))
        assert sum(g_ints) == setup.n_time
