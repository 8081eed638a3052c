"""Train the warm-start network on the solver's own solutions.

    python -m paper_2412_10072_gb300.train_warmstart --n-obs 21 --out warmstart_mlp.npz

Each observation is a config-1-style synthetic observation (64 antennas,
50 sources, MeerKAT L-band, 300 times x 512 channels) whose diagonal gains
drift from one time to the next; it is cut into 1-time x 16-channel
intervals (9600 per observation), solved to convergence by the batched
solver, and turned into (features, targets) pairs, the previous-interval
feature of interval (t, f) being the solution of interval (t - 1, f).
21 observations give 201,600 intervals (12.9 M antenna rows).  Seeds
20000 + k are used for training; evaluation uses other seeds.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-obs", type=int, default=21)
    ap.add_argument("--seed0", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--n-time", type=int, default=300)
    ap.add_argument("--n-chan", type=int, default=512)
    ap.add_argument("--out", default=None)
    ap.add_argument("--log", default=None)
    args = ap.parse_args(argv)

    import torch
    from . import warmstart as ws

    logf = open(args.log, "w") if args.log else None

    def log(*a):
        msg = " ".join(str(x) for x in a)
        print(msg, flush=True)
        if logf:
            logf.write(msg + "\n")
            logf.flush()

    t0 = time.time()
    X, T = ws.training_set(args.n_obs, seed0=args.seed0, n_time=args.n_time, n_chan=args.n_chan, log=log)
    t_data = time.time() - t0
    n = X.shape[0]
    n_val = min(n // 10, 200000)
    val = (X[n - n_val:].contiguous(), T[n - n_val:].contiguous())
    X, T = X[:n - n_val].contiguous(), T[:n - n_val].contiguous()
    t1 = time.time()
    net, hist = ws.train(X, T, epochs=args.epochs, batch=args.batch, lr=args.lr, log=log, val=val)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    summary = {"intervals": int(args.n_obs * (args.n_time * args.n_chan // 16)), "rows_train": int(X.shape[0]),
               "rows_val": int(n_val), "data_s": round(t_data, 1), "train_s": round(t_train, 1), "history": hist}
    log(json.dumps(summary))
    net.save(args.out or ws.DEFAULT_CHECKPOINT, history=json.dumps(hist), intervals=summary["intervals"])
    return summary


if __name__ == "__main__":
    main()
