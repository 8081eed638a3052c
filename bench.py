#!/usr/bin/env python
"""Throughput benchmark of the GB300 gain-calibration solver.

Workload (default): 64 antennas (2016 baselines), 300 times x 512 channels,
4 correlations, complex64 data/model and float32 weights resident in HBM
(25.1 GB), 50 point sources, noise sigma 0.05, 10% of rows flagged; the
chain is G (full 2x2, one interval per time) then B (diagonal bandpass, one
interval per channel), 3 epochs, at most 20 iterations per term solve,
tolerance 1e-6.  One step = one qc_solve of that chain from unit gains.

Metric: visibility-iterations per second (samples of active intervals summed
over every iteration of every term solve, divided by device time).  The JSON
line also carries the roofline of the accumulate kernel (algorithmic bytes /
event-timed duration vs measured HBM bandwidth), an end-to-end figure through
the C ABI with host buffers, the FP64 oracle timed on a bounded sample on the
host cores, and SM clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {ours,reference}] [--mixed]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "vis*iterations/s"
UNIT = "vis*iter/s"
WORKLOAD = "plain two-term solve: 64 ant, 300 t x 512 ch, G full 1t x 512ch then B diag 300t x 1ch, 3 epochs"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain", choices=["plain", "mixed", "batched", "warmstart", "delay", "mad",
                                                            "kde", "moments"],
                    help="plain: the large two-term solve; mixed: the same with FP16 model storage; batched: 4096 "
                         "independent intervals in one persistent launch; warmstart: the batched solve at 64 "
                         "antennas from cold, previous-interval and network starts; delay: a delay and phase "
                         "term per integration over all channels on the large observation; mad: MAD residual "
                         "flagging of the large observation; kde: the KdE chain with two directions (K per "
                         "integration, direction-dependent dE over 16 integrations x 128 channels)")
    ap.add_argument("--mixed", action="store_true", help="same as --workload mixed")
    ap.add_argument("--n-prob", type=int, default=4096, help="problems of the batched / warmstart workloads")
    ap.add_argument("--looped", type=int, default=256, help="problems timed one by one for the comparison")
    ap.add_argument("--checkpoint", default=None, help="warm-start network (.npz)")
    ap.add_argument("--n-time", type=int, default=300)
    ap.add_argument("--n-chan", type=int, default=512)
    ap.add_argument("--n-ant", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--max-iter", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--moments", action="store_true",
                    help="plain workload: solve each term from per-(interval, pair) sums (qc_opts.moments)")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="process group of the multi-GPU mode (gloo: host-staged exchange, for checking the "
                         "sharded flow with several ranks on fewer GPUs)")
    ap.add_argument("--block", type=int, default=0, help="threads per CTA of the accumulate kernel (0: auto)")
    ap.add_argument("--kernel", type=int, default=0,
                    help="accumulate kernel: 0 auto (streaming), 1 bulk-copy pipeline, 2 prefetching, 3 streaming, "
                         "4 warp-specialised")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


ACC_KERNEL_NAME = {0: "acc_stream_kernel", 1: "acc_pipe_kernel", 2: "acc_kernel", 3: "acc_stream_kernel",
                   4: "acc_ws_kernel", 5: "acc_run_kernel"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("qc_kernels.cuh", "qc_stream.cuh", "qc_ws.cuh", "qc_jones.cuh", "qc_async.cuh", "qc_acc_inst.cuh",
                 "qc_acc_diag.cu", "qc_acc_full.cu"):
        with open(os.path.join(ROOT, "paper_2412_10072_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per full accumulate launch from the committed ncu summary, if it was taken on
    the current kernel source (its hash is recorded next to the figure); else None."""
    path = os.path.join(ROOT, "profiles", "acc_stream_kernel_plain_large.md")
    try:
        text = open(path).read()
    except OSError:
        return None, None
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", text)
    t = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    a = re.search(r"algorithmic_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not (m and t) or m.group(1) != kernel_source_hash():
        return None, None
    return float(t.group(1)), (float(a.group(1)) if a else None)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="qc_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


# ---------------------------------------------------------------------------
# the workload
# ---------------------------------------------------------------------------

def make_terms(qc, setup, n_ant, max_iter, world=1, rank=0):
    """The chain's terms; with world > 1 each rank's view of them under the time-block split:
    a term whose intervals lie inside one block (G) is solved on the rank's own intervals, a term
    with an interval spanning blocks (B) over all of them with reduce = 1."""
    if world == 1:
        return [qc.Term.from_spec(s, n_ant, max_iter=max_iter, tol=1e-6) for s in setup.terms]
    from paper_2412_10072_gb300 import shard
    out = []
    for s in setup.terms:
        ts = shard.shard_term(s.t_map, s.n_tint, setup.n_time, world, rank)
        out.append(qc.Term(s.kind, ts.t_map, s.f_map, ts.n_tint, s.n_fint, n_ant, max_iter=max_iter, tol=1e-6,
                           reduce=ts.reduce))
    return out


def shard_setup(setup, world, rank):
    """Rank's rows of the observation (a contiguous block of times) and their local time index."""
    import dataclasses
    import numpy as np
    from paper_2412_10072_gb300 import shard
    t0, t1 = shard.time_block(setup.n_time, rank, world)
    rows = shard.block_rows(setup.time_idx, t0, t1)
    sub = dataclasses.replace(setup, ant1=setup.ant1[rows], ant2=setup.ant2[rows], time_idx=setup.time_idx[rows],
                              uvw=setup.uvw[rows], flag_rows=setup.flag_rows[rows],
                              flag_samples=None if setup.flag_samples is None else setup.flag_samples[rows])
    return sub, (setup.time_idx[rows] - t0).astype(np.int32), t1 - t0


def cpu_baseline(args, dev_obs, setup, n_times=2, max_iter=4):
    """The FP64 oracle on a bounded sample of the same workload: the rows of the first
    ``n_times`` times (all baselines, all channels), one epoch of G then B, ``max_iter``
    iterations each, single-threaded C on the host."""
    import numpy as np
    import oracle as O
    n_bl = setup.n_ant * (setup.n_ant - 1) // 2
    rows = n_times * n_bl
    data = dev_obs["data"][:rows].cpu().numpy()
    model = dev_obs["model"][:rows].cpu().numpy()
    weight = dev_obs["weight"][:rows].cpu().numpy()
    flag = dev_obs["flag"][:rows].cpu().numpy()
    P = O.OracleProblem(data, model, weight, flag, setup.ant1[:rows], setup.ant2[:rows], setup.time_idx[:rows],
                        setup.n_ant, n_times)
    terms = []
    for s in setup.terms:
        tm = s.t_map[:n_times]
        nt = int(tm.max()) + 1
        terms.append(O.OracleTerm(s.kind, tm, s.f_map, nt, s.n_fint, setup.n_ant, max_iter=max_iter, tol=1e-6))
    t0 = time.perf_counter()
    its = O.solve(P, terms, n_epochs=1, damping_mode=1)
    dt = time.perf_counter() - t0
    n_vis = rows * data.shape[1]
    vis_iters = sum(int(n_vis * (it.astype(np.int64).sum() / it.size)) for it in its)
    return {"value": vis_iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n_times} of {setup.n_time} times ({n_vis} vis), 1 epoch G then B, "
                      f"<= {max_iter} iterations each, {dt:.1f} s single-threaded FP64 C"}


def mixed_accuracy(n_ant=16, n_time=8, n_chan=64, epochs=3):
    """Gain and chi^2 errors against the FP64 oracle of the plain complex64 run and of the FP16-model
    run, on a reduced two-term workload of the same recipe (the oracle finishes it in seconds)."""
    import numpy as np
    import oracle as O
    from oracle.gauge import chain_products, reference_chain, rel_err
    from paper_2412_10072_gb300 import qc, synth
    obs = synth.plain_large(seed=7, n_ant=n_ant, n_time=n_time, n_chan=n_chan, noise=0.05, flag_row_frac=0.1)
    P = O.OracleProblem.from_obs(obs)
    ot = [O.OracleTerm.from_spec(s_, obs.n_ant) for s_ in obs.terms]
    O.solve(P, ot, n_epochs=epochs, damping_mode=1)
    ochi2 = O.residual(P, ot)
    Co = reference_chain(chain_products([t.jones() for t in ot], [t.t_map for t in ot], [t.f_map for t in ot],
                                        n_time, n_chan))
    out = {}
    for name, m16 in (("c64", False), ("fp16_model", True)):
        S = qc.Solver.from_obs(obs, model_fp16=m16)
        gt = [qc.Term.from_spec(s_, obs.n_ant) for s_ in obs.terms]
        S.solve(gt, n_epochs=epochs)
        chi2 = S.residual(gt)
        S.close()
        Cg = reference_chain(chain_products([np.asarray(t.gains, np.complex128) for t in gt],
                                            [t.t_map for t in gt], [t.f_map for t in gt], n_time, n_chan))
        out[name] = {"gain_rel_err": rel_err(Cg, Co), "chi2_rel_err": abs(chi2 - ochi2) / ochi2}
    out["case"] = f"{n_ant} ant, {n_time} t x {n_chan} ch, G full + B diag, {epochs} epochs, sigma 0.05"
    return out


def plain_config(args, world=1):
    """The plain workload's config block (shared by the reference arm, so that both lines name the
    same workload)."""
    n_vis = args.n_ant * (args.n_ant - 1) // 2 * args.n_time * args.n_chan
    return {"workload": WORKLOAD + (" (FP16 model)" if args.mixed else "")
            + (", each term from per-(interval, pair) sums" if getattr(args, "moments", False) else ""),
            "n_ant": args.n_ant,
            "n_time": args.n_time, "n_chan": args.n_chan, "n_vis": n_vis,
            "input_bytes_per_gpu": (n_vis * (64 if args.mixed else 80) + n_vis) // world,
            "l2": "inputs (25 GB) larger than L2 (129 MB)", "epochs": args.epochs, "max_iter": args.max_iter,
            "tol": 1e-6, "parallelism": (f"time-block shards x{world}: G per rank, B reduce=1 with an "
                                         f"{getattr(args, 'dist_backend', 'nccl').upper()} allreduce of its normal "
                                         "equations" if world > 1 else "1 GPU")}


def run_reference(args):
    """--impl reference: the FP64 oracle as it stands on the host cores, on a bounded sample of the
    same workload (the first 2 times of the 64-antenna, 512-channel observation; 1 epoch, <= 2
    iterations per term per step)."""
    import numpy as np
    import oracle as O
    from paper_2412_10072_gb300 import synth
    obs = synth.plain_large(seed=1, n_ant=args.n_ant, n_time=2, n_chan=args.n_chan, noise=0.05,
                            flag_row_frac=0.1, n_src=50)
    P = O.OracleProblem.from_obs(obs)

    def step():
        terms = [O.OracleTerm.from_spec(s, obs.n_ant, max_iter=2, tol=1e-6) for s in obs.terms]
        its = O.solve(P, terms, n_epochs=1, damping_mode=1)
        return sum(int(obs.n_vis * it.astype(np.int64).sum() / it.size) for it in its)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    vi = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    value = vi / dt
    sample = (f"first 2 of {args.n_time} times of the same workload ({obs.n_vis} vis), 1 epoch G then B, "
              f"<= 2 iterations each per step, single-threaded FP64 C oracle")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": plain_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    args = parse()
    if args.mixed:
        args.workload = "mixed"
    args.mixed = args.workload == "mixed"
    if args.workload == "batched" and args.impl == "ours":
        return run_batched(args)
    if args.workload == "warmstart" and args.impl == "ours":
        return run_warmstart(args)
    if args.workload == "delay" and args.impl == "ours":
        return run_delay(args)
    if args.workload == "mad" and args.impl == "ours":
        return run_mad(args)
    if args.workload == "kde" and args.impl == "ours":
        return run_kde(args)
    if args.workload == "moments" and args.impl == "ours":
        return run_moments(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    import numpy as np
    import torch
    from paper_2412_10072_gb300 import qc, synth

    local = local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        if args.dist_backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- workload on the device (one observation; with world > 1 every rank holds a block of its
    # times, solves G on its own intervals and B over all of them with an NCCL allreduce of B's
    # partial normal equations before every update) ----
    setup = synth.plain_large_setup(seed=1, n_ant=args.n_ant, n_time=args.n_time, n_chan=args.n_chan,
                                    flag_row_frac=0.1, n_src=50)
    if world > 1:
        gen_setup, local_time, local_n_time = shard_setup(setup, world, rank)
    else:
        gen_setup, local_time, local_n_time = setup, setup.time_idx, setup.n_time
    t_gen = time.perf_counter()
    obs = synth.make_observation_device(gen_setup, noise=0.05, noise_seed=1000 + rank, device=f"cuda:{local}")
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    geo = (gen_setup.ant1, gen_setup.ant2, local_time, setup.n_ant, local_n_time)
    stream = torch.cuda.Stream()
    solver = qc.Solver(obs["data"], obs["model"], obs["weight"], obs["flag"], *geo, model_fp16=args.mixed)
    allreduce = None
    if world > 1:
        from paper_2412_10072_gb300 import shard
        allreduce = shard.allreduce_callback()

    def step():
        terms = make_terms(qc, setup, setup.n_ant, args.max_iter, world, rank)
        return solver.solve(terms, n_epochs=args.epochs, stream=stream, kernel=args.kernel,
                            block_threads=args.block, allreduce=allreduce, moments=args.moments), terms

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        stats = [step()[0] for _ in range(args.steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clock_info = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    vis_iters = sum(s.vis_iters for s in stats)
    acc_bytes = sum(s.acc_bytes for s in stats)
    acc_ms = sum(s.acc_ms for s in stats)
    acc_launches = sum(s.acc_launches for s in stats)
    launches = sum(s.launches for s in stats)
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        v = torch.tensor([float(vis_iters)], dtype=torch.float64, device="cuda")
        dist.all_reduce(v)
        vis_iters_all = float(v.item())
    else:
        vis_iters_all = float(vis_iters)
    value = vis_iters_all / (ms / 1000.0)

    # ---- roofline of the accumulate kernel (event-timed on the solver stream) ----
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # algorithmic bytes: B per vis-iteration (81; 65 with the FP16 model) x the samples of the active
    # intervals each launch processes; the kernel's own reads skip fully flagged rows (read_bytes)
    bpv = 65 if args.mixed else 81
    alg_bytes = bpv * vis_iters
    achieved = (alg_bytes / (acc_ms / 1000.0)) / 1e9 if acc_ms > 0 else None
    # the committed capture is of the complex64 path; the FP16-model path reads other bytes
    traffic, algo_full = profiled_traffic() if not args.mixed else (None, None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                "bytes_per_vis_iteration": bpv,
                "read_bytes_per_launch": acc_bytes / max(1, acc_launches),
                "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                else "fallback 6.8 TB/s", "kernel": ACC_KERNEL_NAME.get(args.kernel, "acc_kernel") + " (JHJ/JHr accumulate)",
                "algorithmic_bytes_per_launch": alg_bytes / max(1, acc_launches),
                "algorithmic_bytes_per_full_launch": algo_full,
                "launch_ms_mean": acc_ms / max(1, acc_launches), "acc_share_of_step": acc_ms / ms if ms else None}

    if args.moments:
        # the dominant kernels are the passes forming the sums (one per term and epoch): each reads
        # the folded weights of every sample and the data and model of usable ones
        n_unflagged = int((obs["flag"] == 0).sum().item())
        n_vis_local = int(obs["flag"].numel())
        pass_bytes = 16 * n_vis_local + 64 * n_unflagged
        n_pass = args.epochs * len(setup.terms) * len(stats)
        pass_ms = sum(s.pass_ms for s in stats)
        p_ach = pass_bytes * n_pass / (pass_ms / 1000.0) / 1e9 if pass_ms > 0 else None
        roofline = {"bound": "hbm", "achieved": p_ach, "peak": hbm, "unit": "GB/s",
                    "frac": (p_ach / hbm) if p_ach else None, "traffic": None,
                    "peak_source": roofline["peak_source"],
                    "kernel": "mom_pass_kernel (the pass forming a term's sums, one per term and epoch)",
                    "algorithmic_bytes_per_launch": pass_bytes, "launch_ms_mean": pass_ms / max(1, n_pass),
                    "pass_share_of_step": pass_ms / ms if ms else None,
                    "iterations_ms_per_step": (acc_ms - pass_ms) / args.steps}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, obs, setup)
    accuracy = mixed_accuracy() if (args.mixed and rank == 0) else None

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region ----
    e2e = None
    if not args.no_e2e:
        host = {k: torch.empty(obs[k].shape, dtype=obs[k].dtype, pin_memory=True) for k in
                ("data", "model", "weight", "flag")}
        for k in host:
            host[k].copy_(obs[k])
        h2d = sum(int(v.numel() * v.element_size()) for v in host.values())
        del solver
        for k in ("data", "model", "weight", "flag"):
            obs[k] = None
        torch.cuda.empty_cache()

        def e2e_step():
            s = qc.Solver(host["data"], host["model"], host["weight"], host["flag"], *geo, model_fp16=args.mixed)
            terms = make_terms(qc, setup, setup.n_ant, args.max_iter, world, rank)
            st = s.solve(terms, n_epochs=args.epochs, kernel=args.kernel, block_threads=args.block,
                         allreduce=allreduce, moments=args.moments)
            s.close()
            d2h = sum(t.gains.nbytes + t.gain_flags.nbytes + t.iters.nbytes for t in terms)
            return st.vis_iters, d2h

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        res = [e2e_step() for _ in range(args.e2e_steps)]
        torch.cuda.synchronize()
        barrier()
        dt = time.perf_counter() - t0
        vi = sum(r[0] for r in res)
        if dist is not None:
            t = torch.tensor([dt, float(vi)], dtype=torch.float64, device="cuda")
            dist.all_reduce(t[:1], op=dist.ReduceOp.MAX)
            tv = torch.tensor([float(vi), float(h2d), float(res[0][1])], dtype=torch.float64, device="cuda")
            dist.all_reduce(tv)
            dt, vi = float(t[0].item()), float(tv[0].item())
            h2d, res[0] = int(tv[1].item()), (res[0][0], int(tv[2].item()))
        e2e = {"value": vi / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": res[0][1],
               "steps": args.e2e_steps, "note": "qc_create from pinned host buffers + qc_solve + gains D2H + qc_destroy"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "c64+f16" if args.mixed else "c64", "data": "synthetic",
            "config": plain_config(args, world), "gen_s": round(t_gen, 2),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock_info,
            **({"accuracy_vs_fp64_oracle": accuracy} if accuracy else {}),
            "gpu_launches": int(launches), "accumulate_launches_with_work": int(acc_launches),
            "vis_iters": int(vis_iters_all),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# delay term K (Scenario 2): phase and delay per correlation over all channels per integration
# ---------------------------------------------------------------------------

DELAY_WORKLOAD = ("delay term K: 64 ant, 300 t x 512 ch, (phi, tau) per correlation over all channels of each "
                  "integration (300 intervals), channels 0.9-1.7 GHz, 1 epoch")


def delay_terms(qc, n_time, n_chan, n_ant, max_iter, nu):
    import numpy as np
    return [qc.Term("delay", np.arange(n_time, dtype=np.int32), np.zeros(n_chan, np.int32), n_time, 1, n_ant,
                    chan_freq=nu, max_iter=max_iter, tol=1e-6)]


def run_delay(args):
    """The delay term solved alone on the large observation (data of the plain workload), device-timed;
    the oracle on the first 2 integrations as the CPU baseline."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2412_10072_gb300 import qc, synth

    torch.cuda.set_device(0)
    setup = synth.plain_large_setup(seed=1, n_ant=args.n_ant, n_time=args.n_time, n_chan=args.n_chan,
                                    flag_row_frac=0.1, n_src=50)
    obs = synth.make_observation_device(setup, noise=0.05, noise_seed=1000, device="cuda:0")
    torch.cuda.synchronize()
    nu = np.linspace(0.9, 1.7, args.n_chan)
    stream = torch.cuda.Stream()
    solver = qc.Solver(obs["data"], obs["model"], obs["weight"], obs["flag"], setup.ant1, setup.ant2,
                       setup.time_idx, setup.n_ant, setup.n_time)

    def step():
        return solver.solve(delay_terms(qc, setup.n_time, args.n_chan, setup.n_ant, args.max_iter, nu),
                            stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        stats = [step() for _ in range(args.steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        clock_info = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    vis_iters = sum(s.vis_iters for s in stats)
    acc_ms = sum(s.acc_ms for s in stats)
    acc_launches = sum(s.acc_launches for s in stats)
    # the initial estimate (qc_delay_init: FFT peak of the reference-antenna baselines), device time
    k0 = delay_terms(qc, setup.n_time, args.n_chan, setup.n_ant, args.max_iter, nu)[0]
    solver.delay_init(k0)
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    i0.record()
    solver.delay_init(k0)
    i1.record()
    torch.cuda.synchronize()
    init_ms = i0.elapsed_time(i1)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (81 * vis_iters / (acc_ms / 1000.0)) / 1e9 if acc_ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None, "traffic": None, "bytes_per_vis_iteration": 81,
                "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                else "fallback 6.8 TB/s",
                "kernel": "acc_delay_kernel (chain rule per sample, sums per parameter interval)",
                "algorithmic_bytes_per_launch": 81 * vis_iters / max(1, acc_launches),
                "launch_ms_mean": acc_ms / max(1, acc_launches), "acc_share_of_step": acc_ms / ms if ms else None}
    cpu = None
    if not args.no_cpu_baseline:
        rows = 2 * (setup.n_ant * (setup.n_ant - 1) // 2)
        P = O.OracleProblem(obs["data"][:rows].cpu().numpy(), obs["model"][:rows].cpu().numpy(),
                            obs["weight"][:rows].cpu().numpy(), obs["flag"][:rows].cpu().numpy(),
                            setup.ant1[:rows], setup.ant2[:rows], setup.time_idx[:rows], setup.n_ant, 2)
        K = O.OracleTerm("delay", np.arange(2, dtype=np.int32), np.zeros(args.n_chan, np.int32), 2, 1, setup.n_ant,
                         chan_freq=nu, max_iter=2, tol=1e-6)
        t0 = time.perf_counter()
        its = O.solve(P, [K])[0]
        dt = time.perf_counter() - t0
        vi = int(rows * args.n_chan * its.astype(np.int64).sum() / its.size)
        cpu = {"value": vi / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first 2 of {setup.n_time} integrations ({rows * args.n_chan} vis), <= 2 iterations, "
                         f"{dt:.1f} s single-threaded FP64 C"}
    line = {"metric": METRIC, "value": vis_iters / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": DELAY_WORKLOAD, "n_ant": args.n_ant, "n_time": args.n_time, "n_chan": args.n_chan,
                       "max_iter": args.max_iter, "tol": 1e-6, "l2": "inputs (25 GB) larger than L2 (129 MB)",
                       "parallelism": "1 GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": None, "clocks": clock_info,
            "gpu_launches": int(sum(s.launches for s in stats)), "accumulate_launches_with_work": int(acc_launches),
            "vis_iters": int(vis_iters), "iterations_max": int(max(s.n_iter_max for s in stats)),
            "initial_estimate_ms": init_ms}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# a single full-Jones term from per-(interval, pair) sums
# ---------------------------------------------------------------------------

MOMENTS_WORKLOAD = ("single full-Jones term G (1 t x 512 ch intervals) on the plain workload's data: 64 ant, "
                    "300 t x 512 ch, 1 epoch, from per-(interval, pair) sums (qc_opts.moments) against the "
                    "per-sample path")


def run_moments(args):
    """G alone solved from per-(interval, antenna pair) sums: one pass over the samples, then each
    iteration on the sums.  Device-timed against the per-sample path on the same data; the pass's
    bandwidth is the roofline (the iterations read 0.97 GB of sums, not the 25 GB of samples)."""
    import torch
    from paper_2412_10072_gb300 import qc, synth

    torch.cuda.set_device(0)
    setup = synth.plain_large_setup(seed=1, n_ant=args.n_ant, n_time=args.n_time, n_chan=args.n_chan,
                                    flag_row_frac=0.1, n_src=50)
    obs = synth.make_observation_device(setup, noise=0.05, noise_seed=1000, device="cuda:0")
    torch.cuda.synchronize()
    n_vis = obs["flag"].numel()
    n_unflagged = int((obs["flag"] == 0).sum().item())
    # the pass reads the folded weights of every sample and the data and model of usable ones
    pass_bytes = 16 * n_vis + 64 * n_unflagged
    stream = torch.cuda.Stream()
    solver = qc.Solver(obs["data"], obs["model"], obs["weight"], obs["flag"], setup.ant1, setup.ant2,
                       setup.time_idx, setup.n_ant, setup.n_time)
    spec = setup.terms[0]

    def timed(moments):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                solver.solve([qc.Term.from_spec(spec, setup.n_ant, max_iter=args.max_iter, tol=1e-6)],
                             stream=stream, moments=moments)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            stats = [solver.solve([qc.Term.from_spec(spec, setup.n_ant, max_iter=args.max_iter, tol=1e-6)],
                                  stream=stream, moments=moments) for _ in range(args.steps)]
            ev1.record(stream)
            torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), stats

    clocks = ClockSampler(0)
    clocks.start()
    ms, stats = timed(True)
    clock_info = clocks.stop()
    ms_plain, stats_plain = timed(False)
    vis_iters = sum(s.vis_iters for s in stats)
    pass_ms = sum(s.pass_ms for s in stats) / len(stats)
    acc_ms = sum(s.acc_ms for s in stats) / len(stats)
    iters = max(s.n_iter_max for s in stats)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = pass_bytes / (pass_ms / 1000.0) / 1e9 if pass_ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None, "traffic": None,
                "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                else "fallback 6.8 TB/s",
                "kernel": "mom_pass_kernel (the one pass forming the sums)",
                "algorithmic_bytes_per_launch": pass_bytes, "launch_ms_mean": pass_ms,
                "iteration_ms_mean": (acc_ms - pass_ms) / max(1, iters)}
    line = {"metric": METRIC, "value": vis_iters / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": MOMENTS_WORKLOAD, "n_ant": args.n_ant, "n_time": args.n_time,
                       "n_chan": args.n_chan, "max_iter": args.max_iter, "tol": 1e-6,
                       "l2": "inputs (25 GB) larger than L2 (129 MB)", "parallelism": "1 GPU"},
            "roofline": roofline, "cpu_baseline": None, "e2e": None, "clocks": clock_info,
            "gpu_launches": int(sum(s.launches for s in stats)), "vis_iters": int(vis_iters),
            "iterations_max": int(iters), "pass_ms": pass_ms,
            "per_sample_path": {"value": sum(s.vis_iters for s in stats_plain) / (ms_plain / 1000.0),
                                "ms_per_step": ms_plain / args.steps},
            "speedup_over_per_sample_path": (ms_plain / ms) if ms else None}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the KdE chain with two directions
# ---------------------------------------------------------------------------

KDE_WORKLOAD = ("KdE chain, 2 directions (field + a 5 Jy source at 1.5 deg): K delay and phase per integration "
                "over all channels, dE direction-dependent diagonal over 16 integrations x 128 channels; 64 ant, "
                "300 t x 512 ch, 2 epochs")


def kde_terms(qc, ks, n_ant, max_iter):
    import numpy as np
    n_time, n_chan = ks.k_truth.shape[0], ks.freqs_ghz.size
    K = qc.Term("delay", ks.k_tmap, np.zeros(n_chan, np.int32), n_time, 1, n_ant, chan_freq=ks.freqs_ghz,
                max_iter=max_iter, tol=1e-6)
    nt, nf = ks.de_truth.shape[:2]
    dE = qc.Term("diag", ks.de_tmap, ks.de_fmap, nt, nf, n_ant, max_iter=max_iter, tol=1e-6, dd=True, n_dir=2)
    return [K, dE]


def run_kde(args):
    """The KdE chain (Section 5) on a 64-antenna, 300 x 512 observation with two directions, device-timed;
    the direction-dependent oracle on a small sample as the CPU baseline."""
    import numpy as np
    import torch
    from oracle import dd
    from paper_2412_10072_gb300 import qc, synth

    torch.cuda.set_device(0)
    ks = synth.kde_setup(seed=3, n_ant=args.n_ant, n_time=args.n_time, n_chan=args.n_chan)
    obs = synth.make_kde_device(ks, noise=0.05, noise_seed=1003, device="cuda:0")
    torch.cuda.synchronize()
    su = ks.base
    stream = torch.cuda.Stream()
    solver = qc.Solver(obs["data"], obs["model"], obs["weight"], obs["flag"], su.ant1, su.ant2, su.time_idx,
                       su.n_ant, su.n_time)
    epochs = 2

    def step():
        return solver.solve(kde_terms(qc, ks, su.n_ant, args.max_iter), n_epochs=epochs, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        stats = [step() for _ in range(args.steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        clock_info = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    vis_iters = sum(s.vis_iters for s in stats)
    acc_ms = sum(s.acc_ms for s in stats)
    acc_launches = sum(s.acc_launches for s in stats)
    bpv = 32 + 2 * 32 + 16 + 1           # d, the model of both directions, weights, flag
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (bpv * vis_iters / (acc_ms / 1000.0)) / 1e9 if acc_ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None, "traffic": None, "bytes_per_vis_iteration": bpv,
                "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                else "fallback 6.8 TB/s",
                "kernel": "dd_stream_kernel (row tiles through a cp.async ring: residual over both directions, "
                          "blocks of dE per direction, K's sums per parameter interval)",
                "algorithmic_bytes_per_launch": bpv * vis_iters / max(1, acc_launches),
                "launch_ms_mean": acc_ms / max(1, acc_launches), "acc_share_of_step": acc_ms / ms if ms else None}
    cpu = None
    if not args.no_cpu_baseline:
        # the direction-dependent oracle (numpy, FP64) on the first integration and 16 channels
        rows, nc = su.n_ant * (su.n_ant - 1) // 2, 16
        P = dd.DDProblem(obs["data"][:rows, :nc].cpu().numpy().astype(np.complex128),
                         obs["model"][:rows, :nc].cpu().numpy().astype(np.complex128),
                         obs["weight"][:rows, :nc].cpu().numpy().astype(np.float64),
                         obs["flag"][:rows, :nc].cpu().numpy(), su.ant1[:rows], su.ant2[:rows],
                         su.time_idx[:rows], su.n_ant)
        K = dd.DDTerm("delay", False, np.zeros(1, np.int32), np.zeros(nc, np.int32), np.zeros((1, 1, su.n_ant, 1, 4)),
                      max_iter=1, tol=1e-6, chan_freq=ks.freqs_ghz[:nc])
        par = np.zeros((1, 1, su.n_ant, 2, 4), np.complex128)
        par[..., 0] = par[..., 3] = 1
        E = dd.DDTerm("diag", True, np.zeros(1, np.int32), np.zeros(nc, np.int32), par, max_iter=1, tol=1e-6)
        t0 = time.perf_counter()
        dd.solve_term(P, [K, E], 0)
        dd.solve_term(P, [K, E], 1)
        dt = time.perf_counter() - t0
        vi = 2 * rows * nc
        cpu = {"value": vi / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first integration, {nc} of {args.n_chan} channels ({rows * nc} vis), one iteration "
                         f"of K then dE, {dt:.1f} s single-threaded FP64 numpy (direction-dependent oracle)"}
    line = {"metric": METRIC, "value": vis_iters / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": KDE_WORKLOAD, "n_ant": args.n_ant, "n_time": args.n_time, "n_chan": args.n_chan,
                       "n_dir": 2, "epochs": epochs, "max_iter": args.max_iter, "tol": 1e-6,
                       "l2": "inputs (35 GB) larger than L2 (129 MB)", "parallelism": "1 GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": None, "clocks": clock_info,
            "gpu_launches": int(sum(s.launches for s in stats)), "accumulate_launches_with_work": int(acc_launches),
            "vis_iters": int(vis_iters), "iterations_max": int(max(s.n_iter_max for s in stats))}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# MAD residual flagging of the large observation
# ---------------------------------------------------------------------------

def run_mad(args):
    """qc_mad_flag on the plain workload's observation with its G and B terms at unit gains
    (the residual is D - M): residual pass, whitened norms, two exact medians (8 radix passes)
    and the flag pass, device-timed per call."""
    import numpy as np
    import torch
    from paper_2412_10072_gb300 import qc, synth

    torch.cuda.set_device(0)
    setup = synth.plain_large_setup(seed=1, n_ant=args.n_ant, n_time=args.n_time, n_chan=args.n_chan,
                                    flag_row_frac=0.1, n_src=50)
    obs = synth.make_observation_device(setup, noise=0.05, noise_seed=1000, device="cuda:0")
    solver = qc.Solver(obs["data"], obs["model"], obs["weight"], obs["flag"], setup.ant1, setup.ant2,
                       setup.time_idx, setup.n_ant, setup.n_time)
    terms = make_terms(qc, setup, setup.n_ant, args.max_iter)
    out = torch.zeros((setup.ant1.size, args.n_chan), dtype=torch.uint8, device="cuda:0")
    for _ in range(args.warmup):
        solver.mad_flag(terms, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    n_flag = [solver.mad_flag(terms, out=out)[1] for _ in range(args.steps)]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    clock_info = clocks.stop()
    # the per-baseline mode (median and MAD over each baseline's samples), timed the same way
    for _ in range(args.warmup):
        solver.mad_flag(terms, out=out, per_baseline=True)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    n_flag_bl = [solver.mad_flag(terms, out=out, per_baseline=True)[1] for _ in range(args.steps)]
    torch.cuda.synchronize()
    dt_bl = time.perf_counter() - t1
    n_vis = setup.ant1.size * args.n_chan
    line = {"metric": "vis/s (MAD flagging)", "value": n_vis * args.steps / dt, "unit": "vis/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "MAD residual flagging (global, threshold 5) of the plain observation: 64 ant, "
                                   "300 t x 512 ch, residual with the G and B terms at unit gains",
                       "n_vis": n_vis, "parallelism": "1 GPU"},
            "flagged": n_flag[-1], "clocks": clock_info,
            "per_baseline": {"value": n_vis * args.steps / dt_bl, "unit": "vis/s", "ms_per_step": 1000 * dt_bl / args.steps,
                             "flagged": n_flag_bl[-1]},
            "note": "wall time of qc_mad_flag per call (residual, norms, 2 x 4 radix passes, flags; 9 host syncs)"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched intervals (4096 independent problems, one persistent launch)
# ---------------------------------------------------------------------------

def _dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    local = local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        if args.dist_backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return world, rank, local, dist


def _referenced(g, offs):
    """Per-problem diagonal gains rotated by the conjugate unit phase of antenna 0 (gauge removal)."""
    import numpy as np
    out = g.copy()
    for i in range(len(offs) - 1):
        r = g[offs[i]:offs[i] + 1]
        ph = np.where(np.abs(r) > 0, np.conj(r) / np.maximum(np.abs(r), 1e-30), 1.0)
        out[offs[i]:offs[i + 1]] = g[offs[i]:offs[i + 1]] * ph
    return out


def _per_problem_err(g, ref, offs):
    import numpy as np
    a, b = _referenced(g, offs), _referenced(ref, offs)
    return np.array([np.max(np.abs(a[offs[i]:offs[i + 1]] - b[offs[i]:offs[i + 1]])) /
                     max(np.max(np.abs(b[offs[i]:offs[i + 1]])), 1e-30) for i in range(len(offs) - 1)])


def _looped_plain(b, idx, tol, max_iter, gains0=None):
    """Solve the problems `idx` one by one through qc_create/qc_solve (config-0-style plain launches).
    Returns (seconds, vis_iters, gains [sum over idx n_ant][2])."""
    import numpy as np
    import torch
    from paper_2412_10072_gb300 import qc
    ctxs = []
    for i in idx:
        r0, r1, v0, v1 = b.row_offset[i], b.row_offset[i + 1], b.vis_offset[i], b.vis_offset[i + 1]
        nc, rows = int(b.n_chan[i]), int(r1 - r0)
        s = qc.Solver(b.data[v0:v1].view(rows, nc, 4), b.model[v0:v1].view(rows, nc, 4),
                      b.weight[v0:v1].view(rows, nc, 4), b.flag[v0:v1].view(rows, nc), b.ant1[r0:r1], b.ant2[r0:r1],
                      np.zeros(rows, np.int32), int(b.n_ant[i]), 1)
        ctxs.append(s)
    torch.cuda.synchronize()
    terms = []
    t0 = time.perf_counter()
    vi = 0
    for k, i in enumerate(idx):
        nc, na = int(b.n_chan[i]), int(b.n_ant[i])
        g = None
        if gains0 is not None:
            g = np.zeros((1, 1, na, 4), np.complex64)
            g[0, 0, :, 0] = gains0[k][:, 0]
            g[0, 0, :, 3] = gains0[k][:, 1]
        t = qc.Term("diag", np.zeros(1, np.int32), np.zeros(nc, np.int32), 1, 1, na, gains=g, max_iter=max_iter,
                    tol=tol)
        st = ctxs[k].solve([t])
        vi += st.vis_iters
        terms.append(t)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for s in ctxs:
        s.close()
    gains = np.concatenate([t.gains[0, 0][:, [0, 3]] for t in terms])
    return dt, vi, gains


def run_batched(args):
    import numpy as np
    import torch
    from paper_2412_10072_gb300 import qc, synth
    world, rank, local, dist = _dist_setup()
    # weak scaling: every rank solves its own 4096 problems (independent intervals, no collective)
    shapes = synth.batch_shapes(args.n_prob, seed_base=1000 + rank * args.n_prob)
    t_gen = time.perf_counter()
    b = synth.make_batch(shapes, device=f"cuda:{local}")
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    S = qc.BatchSolver(b.data, b.model, b.weight, b.flag, b.ant1, b.ant2, b.row_offset, b.vis_offset, b.n_chan,
                       b.n_ant)
    stream = torch.cuda.Stream()
    best, n_tried = S.autotune(stream=stream)
    unit = torch.ones((S.total_ant, 2), dtype=torch.complex64, device="cuda")
    for _ in range(args.warmup):
        S.solve(unit.clone(), stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gains = [unit.clone() for _ in range(args.steps)]
    torch.cuda.synchronize()
    ev0.record(stream)
    stats = [S.solve(gains[k], stream=stream)[3] for k in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clock_info = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    vis_iters = sum(s.vis_iters for s in stats)
    byts = sum(s.bytes for s in stats)
    if dist:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        v = torch.tensor([float(vis_iters)], dtype=torch.float64, device="cuda")
        dist.all_reduce(v)
        ms, vis_all = float(t.item()), float(v.item())
    else:
        vis_all = float(vis_iters)
    value = vis_all / (ms / 1e3)
    # the same solves from per-baseline sufficient statistics (one data pass, iterations on the sums)
    moments = None
    if not dist:
        gm = [unit.clone() for _ in range(args.steps + 1)]
        S.solve(gm[-1], stream=stream, moments=True)
        torch.cuda.synchronize()
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        mstats = [S.solve(gm[k], stream=stream, moments=True)[3] for k in range(args.steps)]
        m1.record(stream)
        torch.cuda.synchronize()
        ms_m = m0.elapsed_time(m1)
        moments = {"value": sum(x.vis_iters for x in mstats) / (ms_m / 1e3), "unit": UNIT,
                   "ms_per_step": ms_m / args.steps, "speedup_over_sample_solve": ms / ms_m,
                   "bytes_per_step": sum(x.bytes for x in mstats) / args.steps,
                   "mean_iters": mstats[-1].mean_iters,
                   "note": "qc_batch_solve_moments: one pass forms per-baseline sums, iterations use them"}
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # algorithmic bytes: 81 B per vis-iteration (every sample of every iteration); the kernel skips
    # copying flagged samples, but they share DRAM bursts with read neighbours
    achieved = 81.0 * vis_iters / (ms / 1e3) / 1e9
    # looped plain launches on a sample of the same problems
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(b.n_prob, size=min(args.looped, b.n_prob), replace=False))
    dt_loop, vi_loop, _ = _looped_plain(b, idx, 1e-6, 20)
    loop_value = vi_loop / dt_loop
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        t0 = time.perf_counter()
        vi = 0
        k = 0
        while time.perf_counter() - t0 < 10.0 and k < b.n_prob:
            i = int(idx[k % idx.size]); k += 1
            r0, r1, v0, v1 = b.row_offset[i], b.row_offset[i + 1], b.vis_offset[i], b.vis_offset[i + 1]
            nc, rows = int(b.n_chan[i]), int(r1 - r0)
            P = O.OracleProblem(b.data[v0:v1].cpu().numpy().reshape(rows, nc, 4),
                                b.model[v0:v1].cpu().numpy().reshape(rows, nc, 4),
                                b.weight[v0:v1].cpu().numpy().reshape(rows, nc, 4),
                                b.flag[v0:v1].cpu().numpy().reshape(rows, nc), b.ant1[r0:r1], b.ant2[r0:r1],
                                np.zeros(rows, np.int32), int(b.n_ant[i]), 1)
            T = O.OracleTerm("diag", np.zeros(1, np.int32), np.zeros(nc, np.int32), 1, 1, int(b.n_ant[i]))
            it = O.solve(P, [T], damping_mode=1)[0]
            vi += rows * nc * int(it[0, 0])
        dt = time.perf_counter() - t0
        cpu = {"value": vi / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{k} of the {b.n_prob} problems solved one by one, {dt:.1f} s single-threaded FP64 C"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": f"batched: {args.n_prob} independent diagonal-gain intervals, ant U{{7..64}}, "
                                   "times U{1..16}, chans U{1..64}, flags U(0,0.5), one persistent launch",
                       "n_vis": b.n_vis, "input_bytes_per_gpu": int(b.n_vis * 81),
                       "l2": "inputs larger than L2 (129 MB); a small problem may stay in L2 across its iterations",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU", "gen_s": round(t_gen, 1)},
            "autotune": {"threads": best.threads, "ctas_per_sm": best.ctas_per_sm, "schedule": best.schedule,
                         "candidates": n_tried, "best_ms": best.ms},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": "batch_kernel (persistent, whole solve)",
                         "bytes_per_vis_iteration": 81, "unflagged_read_bytes": byts,
                         "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)",
                         "mean_iters": stats[-1].mean_iters},
            "looped_plain": {"problems": int(idx.size), "value": loop_value, "unit": UNIT, "seconds": dt_loop,
                             "speedup_of_batched": value / loop_value},
            "moments": moments,
            "cpu_baseline": cpu, "e2e": None, "clocks": clock_info,
            "gpu_launches": args.steps, "vis_iters": int(vis_all)}), flush=True)
    S.close()
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# learned warm start at 64 antennas, and time to tolerance against looped plain solves
# ---------------------------------------------------------------------------

def run_warmstart(args):
    import numpy as np
    import torch
    from paper_2412_10072_gb300 import qc, synth
    from paper_2412_10072_gb300 import warmstart as ws
    world, rank, local, dist = _dist_setup()
    dev = f"cuda:{local}"
    ckpt = args.checkpoint or ws.DEFAULT_CHECKPOINT
    net = ws.MLP.load(ckpt, device=dev)
    shapes = synth.batch_shapes(args.n_prob, seed_base=50000 + rank * args.n_prob, ant=(64, 64))
    offs = np.concatenate([[0], np.cumsum([s_[1] for s_ in shapes])])
    # previous intervals: solved untimed, only their gains are kept
    t_gen = time.perf_counter()
    prev_b, _ = synth.make_pair_batches(shapes, device=dev, which=(0,))
    Sp = qc.BatchSolver(prev_b.data, prev_b.model, prev_b.weight, prev_b.flag, prev_b.ant1, prev_b.ant2,
                        prev_b.row_offset, prev_b.vis_offset, prev_b.n_chan, prev_b.n_ant)
    gp, _, _, _ = Sp.solve(torch.ones((Sp.total_ant, 2), dtype=torch.complex64, device=dev), max_iter=50, tol=1e-8)
    Sp.close()
    del prev_b, Sp
    torch.cuda.empty_cache()
    _, b = synth.make_pair_batches(shapes, device=dev, which=(1,))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    S = qc.BatchSolver(b.data, b.model, b.weight, b.flag, b.ant1, b.ant2, b.row_offset, b.vis_offset, b.n_chan,
                       b.n_ant)
    S16 = qc.BatchSolver(b.data, b.model, b.weight, b.flag, b.ant1, b.ant2, b.row_offset, b.vis_offset, b.n_chan,
                         b.n_ant, model_fp16=True)
    stream = torch.cuda.Stream()
    S.autotune(stream=stream)
    S16.autotune(stream=stream)
    unit = torch.ones((S.total_ant, 2), dtype=torch.complex64, device=dev)
    ref, _, _, _ = S.solve(gp.clone(), max_iter=200, tol=1e-10, stream=stream)
    ref_h = ref.cpu().numpy()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    # time to tolerance: each arm is run with a ladder of stopping tolerances (relative gain
    # change); its time to tolerance is its fastest run that leaves >= 99% of the intervals
    # within 1e-4 (relative, referenced) of the converged solution
    ladder = (1e-4, 3e-5, 1e-5, 3e-6, 1e-6)
    goal, quorum = 1e-4, 0.99

    def pick(res):
        ok = [(v["ms"], k) for k, v in res.items() if v["frac_within_1e-4"] >= quorum]
        return min(ok) if ok else (None, None)

    arms = {}
    # the sample-based batched solve, and the same from per-baseline sums (qc_batch_solve_moments;
    # its network arms take the fallback rule from the sums)
    for name, solver, start, mom in (("cold", S, "unit", False), ("prev", S, "prev", False), ("mlp", S, "mlp", False),
                                     ("mlp_fp16", S16, "mlp", False), ("prev_moments", S, "prev", True),
                                     ("mlp_moments", S, "mlp", True), ("mlp_fp16_moments", S16, "mlp", True)):
        res = {}
        for tol in ladder:
            for _ in range(max(1, args.warmup)):       # warm the launch path
                solver.solve(unit.clone(), max_iter=20, tol=tol, stream=stream, moments=mom)

            def run():
                if start == "mlp":
                    return ws.warm_solve(solver, net, gp, max_iter=40, tol=tol, stream=stream, moments=mom)
                g0 = unit.clone() if start == "unit" else gp.clone()
                g, _, it, st = solver.solve(g0, max_iter=40, tol=tol, stream=stream, moments=mom)
                return g, it, st, 0

            (g, it, st, n_fb), ms = timed(run)
            err = _per_problem_err(g.cpu().numpy(), ref_h, offs)
            res[f"tol{tol:g}"] = {"ms": ms, "mean_iters": float(it.float().mean()), "max_iters": int(it.max()),
                                  "median_err": float(np.median(err)), "frac_within_1e-4": float(np.mean(err <= goal)),
                                  "fallbacks": int(n_fb)}
        ms_best, tol_best = pick(res)
        arms[name] = {"time_to_tol_ms": ms_best, "stop_tol": tol_best, "runs": res}
    # the plain GPU solve: config-0-style single-problem launches, looped, on a sample of the problems
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(b.n_prob, size=min(args.looped, b.n_prob), replace=False))
    sub_offs = np.concatenate([[0], np.cumsum(b.n_ant[idx])])
    ref_sub = np.concatenate([ref_h[offs[i]:offs[i + 1]] for i in idx])
    loop_res = {}
    for tol in ladder:
        dt_loop, vi_loop, g_loop = _looped_plain(b, idx, tol, 40)
        err_loop = _per_problem_err(g_loop, ref_sub, sub_offs)
        loop_res[f"tol{tol:g}"] = {"ms": dt_loop * 1e3 * b.n_prob / idx.size, "sample_seconds": dt_loop,
                                   "median_err": float(np.median(err_loop)),
                                   "frac_within_1e-4": float(np.mean(err_loop <= goal))}
    plain_ms, plain_tol = pick(loop_res)
    # batched + warm start + FP16 model: the faster of the sample-based and the sums-based solve
    fast = [k for k in ("mlp_fp16", "mlp_fp16_moments") if arms[k]["time_to_tol_ms"]]
    fast_arm = min(fast, key=lambda k: arms[k]["time_to_tol_ms"]) if fast else None
    fast_ms = arms[fast_arm]["time_to_tol_ms"] if fast_arm else None
    value = plain_ms / fast_ms if (plain_ms and fast_ms) else None
    out = {"metric": "time to 1e-4 gain tolerance (batched + warm start + FP16 model vs looped plain solves)",
           "value": value, "unit": "x speed-up", "n_gpus": world, "steps": 1, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f16", "data": "synthetic",
           "config": {"workload": f"warm start: {args.n_prob} intervals of 64 antennas, times U{{1..16}}, chans "
                                  "U{1..64}, flags U(0,0.5); previous interval of each solved first",
                      "n_vis": b.n_vis, "gen_s": round(t_gen, 1), "checkpoint": os.path.basename(ckpt),
                      "time_to_tolerance": f">= {quorum:.0%} of intervals within {goal:g} of the converged gains "
                                           "(relative, referenced); fastest stopping tolerance of " + str(ladder)},
           "headline_arm": fast_arm, "arms": arms,
           "speedup_vs_looped_plain": {k: (plain_ms / v["time_to_tol_ms"] if plain_ms and v["time_to_tol_ms"]
                                           else None) for k, v in arms.items()},
           "looped_plain": {"problems": int(idx.size), "time_to_tol_ms_extrapolated": plain_ms, "stop_tol": plain_tol,
                            "runs": loop_res}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    S.close()
    S16.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
