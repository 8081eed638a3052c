"""Learned warm start for the batched solver (binding, trainer, training data).

Every numerical step runs in the library's CUDA kernels (include/qc.h):
``qc_batch_features`` (features at unit gains), ``qc_mlp_forward`` /
``qc_mlp_backward`` / ``qc_mlp_adam`` (the network), ``qc_batch_reference_gains``
(target gauge) and ``qc_batch_warmstart`` (initial gains with fallback).
PyTorch only holds device buffers and orders work on a stream.

Training data are the solver's own solutions: config-1-style observations
(64 antennas, 50 sources, MeerKAT L-band) cut into intervals of 1 time x 16
channels, solved by the batched solver; the previous-interval feature of
interval (t, f) is the solution of interval (t - 1, f).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import time
from typing import Optional

import numpy as np

from . import qc, synth

N_IN, N_HID, N_OUT, N_PARAM = 10, 128, 4, 34948


def _lib():
    lib = qc._load_batch(qc.load())
    if not getattr(lib, "_mlp_ready", False):
        vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
        lib.qc_mlp_forward.argtypes = [vp, vp, i64, vp, vp, vp]
        lib.qc_mlp_backward.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp]
        lib.qc_mlp_adam.argtypes = [vp, vp, vp, vp, f32, f32, f32, f32, i32, vp]
        lib.qc_mlp_last_error.argtypes = []
        lib.qc_mlp_last_error.restype = C.c_char_p
        lib.qc_batch_features.argtypes = [vp, vp, vp, vp, i32, vp]
        lib.qc_batch_warmstart.argtypes = [vp, vp, vp, i32, vp, C.POINTER(C.c_int32), vp]
        lib.qc_batch_reference_gains.argtypes = [vp, vp, vp, vp]
        for f in (lib.qc_mlp_forward, lib.qc_mlp_backward, lib.qc_mlp_adam, lib.qc_batch_features,
                  lib.qc_batch_warmstart, lib.qc_batch_reference_gains):
            f.restype = C.c_int
        lib._mlp_ready = True
    return lib


def _check(rc, msg):
    if rc != qc.QC_OK:
        raise qc.QCError(rc, msg)


def _stream_ptr(stream):
    return None if stream is None else (int(getattr(stream, "cuda_stream", stream)) or None)


class MLP:
    """The 10 -> 128 -> 128 -> 128 -> 4 GELU network with parameters on the device."""

    def __init__(self, params=None, device="cuda", seed: int = 0):
        import torch
        self.device = torch.device(device)
        if params is None:
            from_np = _he_init(seed)
            params = torch.from_numpy(from_np.astype(np.float32))
        self.params = params.to(self.device, torch.float32).contiguous()
        assert self.params.numel() == N_PARAM
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0

    def forward(self, x, z=None, stream=None):
        import torch
        y = torch.empty((x.shape[0], N_OUT), dtype=torch.float32, device=self.device)
        rc = _lib().qc_mlp_forward(self.params.data_ptr(), x.data_ptr(), int(x.shape[0]), y.data_ptr(),
                                   None if z is None else z.data_ptr(), _stream_ptr(stream))
        _check(rc, _lib().qc_mlp_last_error().decode())
        return y

    def train_step(self, x, t, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, stream=None):
        """One Adam step on the mean squared error of a mini-batch; returns the device loss tensor."""
        import torch
        n = int(x.shape[0])
        z = torch.empty((n, 3 * N_HID), dtype=torch.float32, device=self.device)
        y = self.forward(x, z, stream)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        lib = _lib()
        _check(lib.qc_mlp_backward(self.params.data_ptr(), x.data_ptr(), z.data_ptr(), y.data_ptr(), t.data_ptr(), n,
                                   self.grad.data_ptr(), loss.data_ptr(), _stream_ptr(stream)),
               lib.qc_mlp_last_error().decode())
        self.step += 1
        _check(lib.qc_mlp_adam(self.params.data_ptr(), self.grad.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                               lr, betas[0], betas[1], eps, self.step, _stream_ptr(stream)),
               lib.qc_mlp_last_error().decode())
        return loss

    def save(self, path: str, **meta):
        np.savez(path, params=self.params.cpu().numpy(), **{k: np.asarray(v) for k, v in meta.items()})

    @classmethod
    def load(cls, path: str, device="cuda"):
        import torch
        d = np.load(path)
        return cls(torch.from_numpy(d["params"]), device=device)


def _he_init(seed: int) -> np.ndarray:
    """He-normal hidden layers; the output layer starts at zero, so the untrained network
    returns the previous-interval gains (the skip term) unchanged."""
    rng = np.random.default_rng(seed)
    parts = []
    for out_d, in_d in ((N_HID, N_IN), (N_HID, N_HID), (N_HID, N_HID), (N_OUT, N_HID)):
        w = rng.standard_normal((out_d, in_d)).reshape(-1) * math.sqrt(2.0 / in_d)
        parts.append(w if out_d != N_OUT else np.zeros_like(w))
        parts.append(np.zeros(out_d))
    return np.concatenate(parts)


def features(bsolver: "qc.BatchSolver", prev_gains=None, stream=None, want_prev_chi2: bool = False):
    """Per-antenna features [sum n_ant][10] (device) of a batch on the device; with
    want_prev_chi2, also each problem's chi^2 at prev_gains (same data pass)."""
    import torch
    f = torch.empty((bsolver.total_ant, N_IN), dtype=torch.float32, device="cuda")
    chi = torch.empty(bsolver.n_prob, dtype=torch.float64, device="cuda") if want_prev_chi2 else None
    rc = _lib().qc_batch_features(bsolver._h, None if prev_gains is None else prev_gains.data_ptr(), f.data_ptr(),
                                  None if chi is None else chi.data_ptr(), qc.QC_MEM_DEVICE, _stream_ptr(stream))
    if rc != qc.QC_OK:
        bsolver._err(rc)
    return (f, chi) if want_prev_chi2 else f


def reference(bsolver: "qc.BatchSolver", gains, stream=None):
    import torch
    out = torch.empty_like(gains)
    rc = _lib().qc_batch_reference_gains(bsolver._h, gains.data_ptr(), out.data_ptr(), _stream_ptr(stream))
    if rc != qc.QC_OK:
        bsolver._err(rc)
    return out


def initial_gains(bsolver: "qc.BatchSolver", net: MLP, prev_gains=None, check_chi2: bool = True, stream=None):
    """Features -> network -> initial gains, falling back to prev_gains (or unit gains) per problem
    when the prediction is not finite or has a larger chi^2.  Returns (gains, n_fallback)."""
    import torch
    x = features(bsolver, prev_gains, stream)
    y = net.forward(x, stream=stream)
    fb = prev_gains if prev_gains is not None else torch.ones((bsolver.total_ant, 2), dtype=torch.complex64,
                                                                  device="cuda")
    g = torch.empty((bsolver.total_ant, 2), dtype=torch.complex64, device="cuda")
    n_fb = C.c_int32(0)
    rc = _lib().qc_batch_warmstart(bsolver._h, y.data_ptr(), fb.data_ptr(), int(check_chi2), g.data_ptr(),
                                   C.byref(n_fb), _stream_ptr(stream))
    if rc != qc.QC_OK:
        bsolver._err(rc)
    return g, n_fb.value


def warm_solve(bsolver: "qc.BatchSolver", net: MLP, prev_gains, max_iter: int = 20, tol: float = 1e-6, stream=None,
               **solve_kw):
    """The learned warm start fused ahead of the batched solve: one data pass for the features
    (and chi^2 at the previous-interval gains), the network, then the solve from the predicted
    gains; a problem whose prediction is not finite falls back at once, and one whose chi^2 at
    the prediction exceeds that at the previous gains restarts from them inside the solve's first
    pass (with moments=True: after the pass forming the sums, both chi^2 from the sums).  Returns
    (gains, iters, BatchStats, n_fallback)."""
    x, chi_prev = features(bsolver, prev_gains, stream, want_prev_chi2=True)
    y = net.forward(x, stream=stream)
    import torch
    g0 = torch.empty((bsolver.total_ant, 2), dtype=torch.complex64, device="cuda")
    n_nf = C.c_int32(0)
    rc = _lib().qc_batch_warmstart(bsolver._h, y.data_ptr(), prev_gains.data_ptr(), 0, g0.data_ptr(), C.byref(n_nf),
                                   _stream_ptr(stream))
    if rc != qc.QC_OK:
        bsolver._err(rc)
    g, _, it, st = bsolver.solve(g0, max_iter=max_iter, tol=tol, stream=stream, fallback=(prev_gains, chi_prev),
                                 **solve_kw)
    return g, it, st, n_nf.value + st.n_fallback


def targets_from_gains(bsolver, gains):
    """Network targets [sum n_ant][4]: solved gains referenced to the sum-real gauge, (re, im) per corr."""
    import torch
    r = reference(bsolver, gains)
    return torch.view_as_real(r).reshape(-1, 4).contiguous()


# ---------------------------------------------------------------------------
# training data: config-1-style observations cut into 1 x 16 intervals
# ---------------------------------------------------------------------------

def observation_batch(seed: int, n_ant=64, n_time=300, n_chan=512, f_block=16, n_src=50, noise=0.05,
                      device="cuda"):
    """One observation generated on the device and laid out as a batch of interval problems
    ordered (time, frequency block)."""
    import torch
    su = synth.warmstart_observation_setup(seed, n_ant, n_time, n_chan, f_block, n_src)
    obs = synth.make_observation_device(su, noise, seed + 12345, device)
    n_bl = n_ant * (n_ant - 1) // 2
    n_fb = n_chan // f_block
    assert n_chan % f_block == 0

    def relayout(t, tail):
        shp = (n_time, n_bl, n_fb, f_block) + tail
        return t.view(shp).permute(0, 2, 1, 3, *range(4, 4 + len(tail))).contiguous().view(-1, *tail)

    data = relayout(obs["data"], (4,))
    model = relayout(obs["model"], (4,))
    weight = relayout(obs["weight"], (4,))
    flag = relayout(obs["flag"], ())
    del obs
    n_prob = n_time * n_fb
    p, q = synth.baselines(n_ant)
    ant1 = np.tile(p, n_prob).astype(np.int32)
    ant2 = np.tile(q, n_prob).astype(np.int32)
    row_off = (np.arange(n_prob + 1) * n_bl).astype(np.int64)
    vis_off = row_off * f_block
    b = qc.BatchSolver(data, model, weight, flag, ant1, ant2, row_off, vis_off, np.full(n_prob, f_block, np.int32),
                       np.full(n_prob, n_ant, np.int32))
    b._arrays = (data, model, weight, flag)
    b.grid_shape = (n_time, n_fb)
    return b


def training_set(n_obs: int, seed0: int = 20000, max_iter: int = 50, tol: float = 1e-7, log=print, **kw):
    """Features and targets (device tensors) from n_obs observations (9600 intervals each by default)."""
    import torch
    X, T = [], []
    for k in range(n_obs):
        t0 = time.time()
        b = observation_batch(seed0 + k, **kw)
        n_time, n_fb = b.grid_shape
        n_ant = int(b.n_ant[0])
        g = torch.ones((b.total_ant, 2), dtype=torch.complex64, device="cuda")
        g, _, iters, st = b.solve(g, max_iter=max_iter, tol=tol)
        # previous interval (t - 1, f): shift the solution by one time row of problems
        sol = g.view(n_time, n_fb, n_ant, 2)
        prev = torch.ones_like(sol)
        prev[1:] = sol[:-1]
        prev = prev.reshape(-1, 2).contiguous()
        X.append(features(b, prev))
        T.append(targets_from_gains(b, g))
        torch.cuda.synchronize()
        log(f"observation {k}: {b.n_prob} intervals, mean iters {float(iters.float().mean()):.1f}, "
            f"{time.time() - t0:.1f} s")
        b.close()
        del b
    return torch.cat(X), torch.cat(T)


def train(X, T, epochs=8, batch=4096, lr=2e-3, seed=0, log=print, net: Optional[MLP] = None, val=None):
    """Adam on mini-batches of the solver's own solutions; returns the network and loss history."""
    import torch
    net = net or MLP(seed=seed)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    n = X.shape[0]
    hist = []
    if val is not None:
        # the skip term alone: previous-interval gains as the prediction
        hist.append({"epoch": -1, "val_loss_prev_gains": float(((val[0][:, 6:10] - val[1]) ** 2).mean().item())})
        log(hist[-1])
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        tot, cnt = 0.0, 0
        lr_ep = lr * (0.5 ** (ep // max(1, epochs // 3)))
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            loss = net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr=lr_ep)
            tot += float(loss.item()) if (i // batch) % 50 == 0 else 0.0
            cnt += 1 if (i // batch) % 50 == 0 else 0
        entry = {"epoch": ep, "train_loss": tot / max(1, cnt)}
        if val is not None:
            yv = net.forward(val[0])
            entry["val_loss"] = float(((yv - val[1]) ** 2).mean().item())
        hist.append(entry)
        log(entry)
    return net, hist


DEFAULT_CHECKPOINT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warmstart_mlp.npz")
