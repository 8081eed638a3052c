"""Time-block sharding of one observation across processes, one GPU each.

Solution intervals are independent of one another (Section 4.3), so the rows of
an observation can be split into contiguous blocks of times, one per rank:

* a term whose every interval lies inside one block (the gain G of 1 time x
  all channels) is solved locally, on the rank's own intervals only;
* a term with an interval that spans blocks (the bandpass B of all times x 1
  channel) is solved on every rank over all its intervals, and the partial
  normal equations of each rank's rows are summed across ranks before every
  update (JHJ and JHr are plain sums over samples, Eq. jhj_entry_simplified,
  Eq. jhr_entry_simplified).  ``qc_solve`` does this through the options'
  ``allreduce`` callback for terms with ``reduce = 1``; every rank then makes
  the same FP64 update from the same sums, so the gains stay identical.

This module holds the host logic: the split, the per-rank term maps and the
callback on a ``torch.distributed`` process group.
"""
from __future__ import annotations

import dataclasses
from typing import Tuple

import numpy as np


def time_block(n_time: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous block [t0, t1) of times of `rank` (sizes differ by at most one)."""
    if not (0 <= rank < world) or n_time < world:
        raise ValueError("need 0 <= rank < world <= n_time")
    base, extra = divmod(n_time, world)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def block_rows(time_idx: np.ndarray, t0: int, t1: int) -> np.ndarray:
    """Indices of the rows whose time lies in [t0, t1)."""
    time_idx = np.asarray(time_idx)
    return np.nonzero((time_idx >= t0) & (time_idx < t1))[0]


@dataclasses.dataclass
class TermShard:
    t_map: np.ndarray      # [t1 - t0] local time -> interval of the rank's term
    n_tint: int            # intervals of the rank's term
    tint_offset: int       # first global interval (local terms); 0 for reduced terms
    reduce: bool           # partial normal equations summed across ranks


def shard_term(t_map: np.ndarray, n_tint: int, n_time: int, world: int, rank: int) -> TermShard:
    """Per-rank view of a term's time map for the time-block split."""
    t_map = np.asarray(t_map, dtype=np.int64)
    if t_map.shape != (n_time,):
        raise ValueError("t_map must have n_time entries")
    bounds = [time_block(n_time, r, world) for r in range(world)]
    # local only if every interval's times lie in one block and every block's intervals
    # form a contiguous range (then each rank owns a slice of the gain table)
    owner = np.full(int(n_tint), -1)
    local = True
    for r, (a, b) in enumerate(bounds):
        ints = np.unique(t_map[a:b])
        if np.any((owner[ints] >= 0) & (owner[ints] != r)) or ints[-1] - ints[0] + 1 != ints.size:
            local = False
            break
        owner[ints] = r
    t0, t1 = bounds[rank]
    if not local:
        return TermShard(t_map[t0:t1].astype(np.int32), int(n_tint), 0, True)
    lo = int(t_map[t0:t1].min())
    hi = int(t_map[t0:t1].max())
    return TermShard((t_map[t0:t1] - lo).astype(np.int32), hi - lo + 1, lo, False)


class _DeviceView:
    """Zero-copy float64 device array for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 2, "strides": None, "stream": None}


def allreduce_inplace(t, group=None, stream=None):
    """Sum a tensor across the ranks of `group` in place, ordered after the work already
    queued on `stream` (a CUDA stream handle) and before the work queued after it."""
    import torch
    import torch.distributed as dist
    if t.is_cuda and stream is not None:
        with torch.cuda.stream(torch.cuda.ExternalStream(int(stream), device=t.device)):
            dist.all_reduce(t, group=group)
    else:
        dist.all_reduce(t, group=group)


def allreduce_callback(group=None):
    """A ``qc_opts.allreduce`` callback summing the library's FP64 accumulator buffer
    across the ranks of `group` (NCCL for CUDA tensors).  Keep a reference to the
    returned function while the solve runs."""
    import torch

    def cb(ptr, n, stream, user):
        try:
            t = torch.as_tensor(_DeviceView(ptr, n), device="cuda")
            allreduce_inplace(t, group, stream)
            return 0
        except Exception:       # a failed exchange is reported to the library as an error status
            return 1
    return cb


def shard_observation(arrays: dict, time_idx: np.ndarray, n_time: int, world: int, rank: int):
    """Rows of rank's block from per-row arrays (first axis = rows), with local time indices."""
    t0, t1 = time_block(n_time, rank, world)
    rows = block_rows(time_idx, t0, t1)
    out = {k: v[rows] for k, v in arrays.items()}
    out["time_idx"] = (np.asarray(time_idx)[rows] - t0).astype(np.int32)
    return out, (t0, t1), rows
