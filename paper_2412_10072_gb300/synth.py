"""Seeded synthetic interferometer observations (input generation only).

This module draws every random number the workloads need and lays the
results out in the Measurement-Set row order the solver consumes: rows are
(time, baseline) pairs sorted by time, then by baseline p < q, with
``ant1``/``ant2``/``time_idx`` per row (the paper's row-to-time mapping,
Section 4.1) and visibilities stored ``[row][chan][corr]`` with the four
correlations of each 2x2 matrix in row-major order (Eq. gvec / Eq. jones).

It holds no part of the calibration method: no Jacobians, normal equations,
block solves or iterations.  Corrupting the predicted visibilities with
"true" gains (``V = G_p M G_q^H``, the forward measurement equation of
Eq. baselinemodel) is simulation of the instrument and is written here with
``numpy.einsum`` independently of both the CPU oracle and the CUDA path,
which only ever *read* what this module writes.

Sky model: unpolarised point sources, ``M = sum_k S_k exp(-2 pi i nu/c
(u l + v m + w (n - 1))) * I``, uvw from an east-west array (the textbook
form; the paper delegates prediction to an external DFT, Section 4.7).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

C_LIGHT = 299_792_458.0
DEG = np.pi / 180.0


# ---------------------------------------------------------------------------
# geometry and sky
# ---------------------------------------------------------------------------

def ew_array(n_ant: int, max_baseline_m: float, rng: np.random.Generator) -> np.ndarray:
    """East-west antenna offsets in metres (sorted, first antenna at 0)."""
    x = np.sort(rng.uniform(0.0, max_baseline_m, size=n_ant))
    x[0] = 0.0
    x[-1] = max_baseline_m
    return np.sort(x)


def baselines(n_ant: int):
    """All p < q pairs in lexicographic order (no autocorrelations)."""
    p, q = np.triu_indices(n_ant, k=1)
    return p.astype(np.int32), q.astype(np.int32)


def hour_angles(n_time: int, span_hours: float = 4.0, centre_hours: float = 0.0) -> np.ndarray:
    """Hour angles (radians) uniform over centre +- span/2 hours across n_time samples."""
    h = np.linspace(-span_hours / 2.0, span_hours / 2.0, n_time) if n_time > 1 else np.zeros(1)
    return (h + centre_hours) * 15.0 * DEG


def ew_uvw(ant_x: np.ndarray, p: np.ndarray, q: np.ndarray, ha: np.ndarray,
           dec: float = -30.0 * DEG) -> np.ndarray:
    """uvw (metres) for every (time, baseline): shape [n_time, n_bl, 3].

    For an east-west baseline of length b: u = b cos H, v = b sin(dec) sin H,
    w = -b cos(dec) sin H.
    """
    b = (ant_x[q] - ant_x[p])[None, :]
    H = ha[:, None]
    u = b * np.cos(H)
    v = b * np.sin(dec) * np.sin(H)
    w = -b * np.cos(dec) * np.sin(H)
    return np.stack([u, v, w], axis=-1)


@dataclasses.dataclass
class Sky:
    flux: np.ndarray   # [n_src] Jy
    l: np.ndarray      # [n_src] direction cosines
    m: np.ndarray

    @property
    def n(self) -> np.ndarray:
        return np.sqrt(1.0 - self.l ** 2 - self.m ** 2)


def point_sources(n_src: int, rng: np.random.Generator, radius_deg: float = 1.0,
                  flux_lo: float = 0.1, flux_hi: float = 1.0) -> Sky:
    """Point sources with flux U(lo, hi) uniformly inside a disk of given radius."""
    flux = rng.uniform(flux_lo, flux_hi, size=n_src)
    rad = radius_deg * DEG * np.sqrt(rng.uniform(0.0, 1.0, size=n_src))
    ang = rng.uniform(0.0, 2 * np.pi, size=n_src)
    return Sky(flux=flux, l=rad * np.cos(ang), m=rad * np.sin(ang))


def predict_scalar(uvw: np.ndarray, freqs: np.ndarray, sky: Sky) -> np.ndarray:
    """Scalar (Stokes I) visibility for each uvw row and channel: [rows, chan] complex128."""
    phase = (uvw[:, 0:1] * sky.l[None, :] + uvw[:, 1:2] * sky.m[None, :]
             + uvw[:, 2:3] * (sky.n[None, :] - 1.0))            # [rows, src] metres
    out = np.zeros((uvw.shape[0], freqs.size), dtype=np.complex128)
    for ci, nu in enumerate(freqs):
        out[:, ci] = np.exp(-2j * np.pi * nu / C_LIGHT * phase) @ sky.flux
    return out


# ---------------------------------------------------------------------------
# gain truths (each returned on the term's own [n_tint][n_fint][n_ant][4] grid)
# ---------------------------------------------------------------------------

def interval_map(n: int, width: int) -> np.ndarray:
    """Map sample index -> solution-interval index for contiguous intervals."""
    return (np.arange(n) // max(1, width)).astype(np.int32)


def diag_truth(n_ant: int, n_tint: int, n_fint: int, rng: np.random.Generator,
               amp_sigma: float = 0.05, drift_cycles: float = 0.05) -> np.ndarray:
    """Diagonal complex gains: amplitude 1+N(0,amp_sigma), phase U(-pi,pi) plus a slow drift.

    The drift is sampled at each time interval's centre, so the truth is
    piecewise constant over solution intervals (noise-free data are then
    fitted exactly).
    """
    amp = 1.0 + amp_sigma * rng.standard_normal((n_ant, 2))
    ph0 = rng.uniform(-np.pi, np.pi, size=(n_ant, 2))
    rate = drift_cycles * rng.standard_normal((n_ant, 2))
    tc = (np.arange(n_tint) + 0.5) / max(1, n_tint)
    ph = ph0[None] + 2 * np.pi * rate[None] * tc[:, None, None]        # [tint, ant, 2]
    g = amp[None] * np.exp(1j * ph)
    out = np.zeros((n_tint, n_fint, n_ant, 4), dtype=np.complex128)
    out[:, :, :, 0] = g[:, None, :, 0]
    out[:, :, :, 3] = g[:, None, :, 1]
    return out


def full_truth(n_ant: int, n_tint: int, n_fint: int, rng: np.random.Generator,
               leakage: float = 0.05) -> np.ndarray:
    """Full 2x2 gains: diagonal as :func:`diag_truth` plus 0.05*CN(0,1) off-diagonal leakage."""
    out = diag_truth(n_ant, n_tint, n_fint, rng)
    cn = (rng.standard_normal((n_tint, n_ant, 2)) + 1j * rng.standard_normal((n_tint, n_ant, 2))) / np.sqrt(2)
    out[:, :, :, 1] = leakage * cn[:, None, :, 0]
    out[:, :, :, 2] = leakage * cn[:, None, :, 1]
    return out


def bandpass_truth(n_ant: int, n_tint: int, n_fint: int, rng: np.random.Generator,
                   amp_sigma: float = 0.1) -> np.ndarray:
    """Diagonal bandpass: amplitude N(1, amp_sigma) per (antenna, channel, corr) and a
    smooth phase sum_k a_k cos(pi k x + theta_k), x in [0,1], a_k ~ N(0, 0.5/k)."""
    x = np.arange(n_fint) / max(1, n_fint - 1)
    amp = 1.0 + amp_sigma * rng.standard_normal((n_fint, n_ant, 2))
    ph = np.zeros((n_fint, n_ant, 2))
    for k in range(1, 5):
        a = rng.normal(0.0, np.sqrt(0.5 / k), size=(n_ant, 2))
        th = rng.uniform(0, 2 * np.pi, size=(n_ant, 2))
        ph += a[None] * np.cos(np.pi * k * x[:, None, None] + th[None])
    g = amp * np.exp(1j * ph)
    out = np.zeros((n_tint, n_fint, n_ant, 4), dtype=np.complex128)
    out[:, :, :, 0] = g[None, :, :, 0]
    out[:, :, :, 3] = g[None, :, :, 1]
    return out


def phase_truth(n_ant: int, n_tint: int, n_fint: int, rng: np.random.Generator) -> np.ndarray:
    """Phase-only parameters [n_tint][n_fint][n_ant][2] (radians), U(-pi, pi)."""
    return rng.uniform(-np.pi, np.pi, size=(n_tint, n_fint, n_ant, 2))


def phase_to_jones(phi: np.ndarray) -> np.ndarray:
    """Phase parameters [..., 2] -> diagonal Jones [..., 4] (instrument simulation only)."""
    out = np.zeros(phi.shape[:-1] + (4,), dtype=np.complex128)
    out[..., 0] = np.exp(1j * phi[..., 0])
    out[..., 3] = np.exp(1j * phi[..., 1])
    return out


# ---------------------------------------------------------------------------
# observation container and corruption (instrument simulation)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class TermSpec:
    """One Jones term of a chain: kind in {"diag","full","phase"} and its interval maps."""
    kind: str
    t_map: np.ndarray      # [n_time] -> time interval
    f_map: np.ndarray      # [n_chan] -> freq interval
    n_tint: int
    n_fint: int
    truth: Optional[np.ndarray] = None   # complex [tint][fint][ant][4] or phase [..][2]

    def truth_jones(self) -> np.ndarray:
        if self.kind == "phase":
            return phase_to_jones(self.truth)
        return self.truth


@dataclasses.dataclass
class Observation:
    n_ant: int
    n_time: int
    n_chan: int
    data: np.ndarray        # [row][chan][4] complex
    model: np.ndarray       # [row][chan][4] complex (n_dir = 1)
    weight: np.ndarray      # [row][chan][4] float
    flag: np.ndarray        # [row][chan] uint8
    ant1: np.ndarray        # [row] int32
    ant2: np.ndarray
    time_idx: np.ndarray
    freqs: np.ndarray
    terms: List[TermSpec]
    meta: Dict

    @property
    def n_row(self) -> int:
        return int(self.ant1.size)

    @property
    def n_vis(self) -> int:
        return self.n_row * self.n_chan


def _jones_at(term: TermSpec, t: np.ndarray, c: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Gather a term's truth Jones [rows, chan, 2, 2] for row times t, channels c, antennas a."""
    J = term.truth_jones()
    it = term.t_map[t][:, None]
    jf = term.f_map[c][None, :]
    return J[it, jf, a[:, None]].reshape(t.size, c.size, 2, 2)


def corrupt(model: np.ndarray, terms: List[TermSpec], ant1, ant2, time_idx, n_chan) -> np.ndarray:
    """Apply the true Jones chain C_a = prod_j G_j,a to the model: C_p M C_q^H (simulation)."""
    chan = np.arange(n_chan)
    M = model.reshape(model.shape[0], n_chan, 2, 2)
    Cp = np.broadcast_to(np.eye(2, dtype=np.complex128), M.shape).copy()
    Cq = Cp.copy()
    for term in terms:
        Cp = np.einsum("rcij,rcjk->rcik", Cp, _jones_at(term, time_idx, chan, ant1))
        Cq = np.einsum("rcij,rcjk->rcik", Cq, _jones_at(term, time_idx, chan, ant2))
    V = np.einsum("rcij,rcjk,rclk->rcil", Cp, M, Cq.conj())
    return V.reshape(model.shape)


@dataclasses.dataclass
class Setup:
    """Everything of an observation that is drawn from the host RNG (small arrays only)."""
    n_ant: int
    n_time: int
    freqs: np.ndarray
    terms: List[TermSpec]
    ant_x: np.ndarray
    sky: Sky
    ant1: np.ndarray
    ant2: np.ndarray
    time_idx: np.ndarray
    uvw: np.ndarray            # [row, 3] metres
    flag_rows: np.ndarray      # [row] bool, whole-row flags
    rng: np.random.Generator   # continues with the noise draws of the host path
    flag_samples: Optional[np.ndarray] = None   # [row, chan] bool, per-sample flags (optional)


def draw_setup(n_ant: int, n_time: int, freqs: np.ndarray, terms: List[TermSpec], *, n_src: int,
               rng: np.random.Generator, ant_x: np.ndarray, flag_row_frac: float = 0.0,
               flag_sample_frac: float = 0.0, ha_span_hours: float = 4.0, ha_centre_hours: float = 0.0) -> Setup:
    sky = point_sources(n_src, rng)
    p, q = baselines(n_ant)
    n_bl = p.size
    ha = hour_angles(n_time, ha_span_hours, ha_centre_hours)
    uvw = ew_uvw(ant_x, p, q, ha).reshape(n_time * n_bl, 3)
    ant1 = np.tile(p, n_time).astype(np.int32)
    ant2 = np.tile(q, n_time).astype(np.int32)
    time_idx = np.repeat(np.arange(n_time, dtype=np.int32), n_bl)
    flag_rows = (rng.random(ant1.size) < flag_row_frac) if flag_row_frac > 0 else np.zeros(ant1.size, bool)
    flag_samples = (rng.random((ant1.size, len(freqs))) < flag_sample_frac) if flag_sample_frac > 0 else None
    return Setup(n_ant, n_time, np.asarray(freqs, np.float64), terms, ant_x, sky, ant1, ant2, time_idx, uvw,
                 flag_rows, rng, flag_samples)


def make_observation(n_ant: int, n_time: int, freqs: np.ndarray, terms: List[TermSpec], *,
                     n_src: int, seed: int, noise: float, flag_row_frac: float = 0.0,
                     max_baseline_m: float = 1000.0, nan_in_flagged: bool = False,
                     rng: Optional[np.random.Generator] = None,
                     ant_x: Optional[np.ndarray] = None, su: Optional[Setup] = None) -> Observation:
    """Build one observation on the host; every random draw comes from ``seed`` (or ``rng``)."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    n_chan = freqs.size
    if su is None:
        if ant_x is None:
            ant_x = ew_array(n_ant, max_baseline_m, rng)
        su = draw_setup(n_ant, n_time, freqs, terms, n_src=n_src, rng=rng, ant_x=ant_x,
                        flag_row_frac=flag_row_frac)
    else:
        rng = su.rng
        ant_x = su.ant_x
    scal = predict_scalar(su.uvw, freqs, su.sky)
    model = np.zeros((su.ant1.size, n_chan, 4), dtype=np.complex128)
    model[:, :, 0] = scal
    model[:, :, 3] = scal
    data = corrupt(model, terms, su.ant1, su.ant2, su.time_idx, n_chan)
    if noise > 0:
        data = data + noise * (rng.standard_normal(data.shape) + 1j * rng.standard_normal(data.shape))
    weight = np.ones(data.shape, dtype=np.float64)
    flag = np.zeros((su.ant1.size, n_chan), dtype=np.uint8)
    flag[su.flag_rows, :] = 1
    if su.flag_samples is not None:
        flag[su.flag_samples] = 1
    if nan_in_flagged:
        data[flag.astype(bool)] = np.nan + 1j * np.nan
    return Observation(n_ant=n_ant, n_time=n_time, n_chan=n_chan, data=data, model=model,
                       weight=weight, flag=flag, ant1=su.ant1, ant2=su.ant2, time_idx=su.time_idx,
                       freqs=freqs, terms=terms,
                       meta=dict(seed=seed, noise=noise, n_src=n_src, ant_x=ant_x,
                                 flag_row_frac=flag_row_frac, sky=su.sky))


def make_observation_device(su: Setup, noise: float, noise_seed: int, device, rows_per_chunk: int = 4096):
    """The same observation generated on a CUDA device (for sizes the host cannot produce
    quickly): complex64 data/model, float32 weights, uint8 flags, all resident on ``device``.

    The small random draws (array, sky, truths, flagged rows) come from ``su`` and are identical
    to :func:`make_observation`; the thermal noise is drawn on the device from ``noise_seed``.
    Returns a dict of tensors plus the host metadata.
    """
    import torch
    n_row, n_chan = su.ant1.size, su.freqs.size
    dev = torch.device(device)
    f64, c64 = torch.float64, torch.complex64
    data = torch.empty((n_row, n_chan, 4), dtype=c64, device=dev)
    model = torch.empty((n_row, n_chan, 4), dtype=c64, device=dev)
    weight = torch.ones((n_row, n_chan, 4), dtype=torch.float32, device=dev)
    fl = np.repeat(su.flag_rows[:, None], n_chan, axis=1)
    if su.flag_samples is not None:
        fl = fl | su.flag_samples
    flag = torch.from_numpy(fl.astype(np.uint8)).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(noise_seed))
    # -2 pi nu / c in FP64; the phase is range-reduced in FP64 and its exponential taken in FP32
    k_nu = torch.from_numpy(-2.0 * np.pi * su.freqs / C_LIGHT).to(dev, f64)
    flux = torch.from_numpy(su.sky.flux).to(dev, torch.float32).to(c64)
    lmn = torch.from_numpy(np.stack([su.sky.l, su.sky.m, su.sky.n - 1.0])).to(dev, f64)     # [3, src]
    jones = [torch.from_numpy(t.truth_jones()).to(dev, c64) for t in su.terms]
    tmaps = [torch.from_numpy(t.t_map.astype(np.int64)).to(dev) for t in su.terms]
    fmaps = [torch.from_numpy(t.f_map.astype(np.int64)).to(dev) for t in su.terms]
    chan = torch.arange(n_chan, device=dev)
    two_pi = 2.0 * np.pi
    for r0 in range(0, n_row, rows_per_chunk):
        r1 = min(n_row, r0 + rows_per_chunk)
        uvw = torch.from_numpy(su.uvw[r0:r1]).to(dev, f64)
        ph = uvw @ lmn                                                         # [R, src] metres
        ang = ph[:, :, None] * k_nu[None, None, :]                             # [R, src, C] radians
        ang = (ang - two_pi * torch.round(ang / two_pi)).to(torch.float32)
        scal = torch.einsum("k,rkc->rc", flux, torch.polar(torch.ones_like(ang), ang))   # [R, C]
        t = torch.from_numpy(su.time_idx[r0:r1].astype(np.int64)).to(dev)
        a1 = torch.from_numpy(su.ant1[r0:r1].astype(np.int64)).to(dev)
        a2 = torch.from_numpy(su.ant2[r0:r1].astype(np.int64)).to(dev)
        Cp = None
        Cq = None
        for J, tm, fm in zip(jones, tmaps, fmaps):
            it = tm[t][:, None]
            jf = fm[chan][None, :]
            Jp = J[it, jf, a1[:, None]].reshape(r1 - r0, n_chan, 2, 2)
            Jq = J[it, jf, a2[:, None]].reshape(r1 - r0, n_chan, 2, 2)
            Cp = Jp if Cp is None else Cp @ Jp
            Cq = Jq if Cq is None else Cq @ Jq
        V = scal[:, :, None, None] * (Cp @ Cq.conj().transpose(-1, -2))       # M = scal * I
        V = V.reshape(r1 - r0, n_chan, 4)
        if noise > 0:
            nz = torch.randn((r1 - r0, n_chan, 4, 2), dtype=torch.float32, device=dev, generator=gen)
            V = V + noise * torch.view_as_complex(nz)
        data[r0:r1] = V
        m = model[r0:r1]
        m.zero_()
        m[:, :, 0] = scal
        m[:, :, 3] = scal
    return dict(data=data, model=model, weight=weight, flag=flag, ant1=su.ant1, ant2=su.ant2,
                time_idx=su.time_idx, n_ant=su.n_ant, n_time=su.n_time, n_chan=n_chan, terms=su.terms)


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def plain_small(seed: int = 0, noise: float = 0.01, n_ant: int = 7, n_time: int = 60,
                n_chan: int = 16, t_int: int = 4, f_int: int = 4, n_src: int = 5) -> Observation:
    """7 antennas, 60 times x 16 channels at 1.4 GHz, 5 sources, diagonal gains
    on 4 x 4 solution intervals, sigma = 0.01, unit weights, no flags."""
    rng = np.random.default_rng(seed)
    freqs = 1.4e9 + 1.0e6 * (np.arange(n_chan) - (n_chan - 1) / 2.0)
    n_tint = -(-n_time // t_int)
    n_fint = -(-n_chan // f_int)
    term = TermSpec("diag", interval_map(n_time, t_int), interval_map(n_chan, f_int), n_tint, n_fint)
    ant_x = ew_array(n_ant, 1000.0, rng)
    term.truth = diag_truth(n_ant, n_tint, n_fint, rng)
    return make_observation(n_ant, n_time, freqs, [term], n_src=n_src, seed=seed, noise=noise,
                            rng=rng, ant_x=ant_x)


def meerkat_band(n_chan: int) -> np.ndarray:
    """n_chan channels across 856 MHz centred at 1.284 GHz (MeerKAT L-band)."""
    bw = 856e6
    return 1.284e9 + bw * ((np.arange(n_chan) + 0.5) / n_chan - 0.5)


def plain_large_terms(n_ant: int, n_time: int, n_chan: int, rng: np.random.Generator):
    """Two-term chain: G full 2x2 per (1 time x all channels), B diagonal bandpass per
    (all times x 1 channel)."""
    G = TermSpec("full", interval_map(n_time, 1), np.zeros(n_chan, np.int32), n_time, 1)
    B = TermSpec("diag", np.zeros(n_time, np.int32), interval_map(n_chan, 1), 1, n_chan)
    G.truth = full_truth(n_ant, n_time, 1, rng)
    B.truth = bandpass_truth(n_ant, 1, n_chan, rng)
    return [G, B]


def plain_large_setup(seed: int = 1, n_ant: int = 64, n_time: int = 300, n_chan: int = 512,
                      flag_row_frac: float = 0.1, n_src: int = 50) -> Setup:
    """Host-drawn part of the large two-term workload (see :func:`plain_large`)."""
    rng = np.random.default_rng(seed)
    freqs = meerkat_band(n_chan)
    ant_x = ew_array(n_ant, 8000.0, rng)
    terms = plain_large_terms(n_ant, n_time, n_chan, rng)
    return draw_setup(n_ant, n_time, freqs, terms, n_src=n_src, rng=rng, ant_x=ant_x, flag_row_frac=flag_row_frac)


def plain_large(seed: int = 1, n_ant: int = 64, n_time: int = 300, n_chan: int = 512,
                noise: float = 0.05, flag_row_frac: float = 0.1, n_src: int = 50,
                nan_in_flagged: bool = False) -> Observation:
    """The large two-term workload on host memory (use reduced sizes on the CPU).

    64 antennas, 300 times x 512 channels over 856 MHz, 50 sources, G (full) then
    B (diagonal bandpass), sigma = 0.05, 10% of rows flagged.
    """
    rng = np.random.default_rng(seed)
    freqs = meerkat_band(n_chan)
    ant_x = ew_array(n_ant, 8000.0, rng)
    terms = plain_large_terms(n_ant, n_time, n_chan, rng)
    return make_observation(n_ant, n_time, freqs, terms, n_src=n_src, seed=seed, noise=noise,
                            flag_row_frac=flag_row_frac, rng=rng, ant_x=ant_x,
                            nan_in_flagged=nan_in_flagged)


# ---------------------------------------------------------------------------
# batches of independent one-interval problems
# ---------------------------------------------------------------------------

def interval_problem_setup(seed: int, n_ant: int, n_time: int, n_chan: int, flag_frac: float,
                           n_src: int = 5, integration_s: float = 8.0) -> Setup:
    """One diagonal-gain solution interval drawn like the small plain workload: an east-west array,
    5 sources at 1.4 GHz (1 MHz channels), gains with amplitude 1+N(0,0.05) and phase U(-pi,pi),
    n_time integrations of 8 s at a random hour angle, per-sample flags with probability flag_frac."""
    rng = np.random.default_rng(seed)
    freqs = 1.4e9 + 1.0e6 * (np.arange(n_chan) - (n_chan - 1) / 2.0)
    ant_x = ew_array(n_ant, 1000.0, rng)
    term = TermSpec("diag", np.zeros(n_time, np.int32), np.zeros(n_chan, np.int32), 1, 1)
    term.truth = diag_truth(n_ant, 1, 1, rng)
    centre = rng.uniform(-2.0, 2.0)
    return draw_setup(n_ant, n_time, freqs, [term], n_src=n_src, rng=rng, ant_x=ant_x,
                      flag_sample_frac=flag_frac, ha_span_hours=n_time * integration_s / 3600.0,
                      ha_centre_hours=centre)


def batch_shapes(n_prob: int, seed_base: int = 1000, ant=(7, 64), times=(1, 16), chans=(1, 64), flag_max=0.5):
    """Per-problem (seed, n_ant, n_time, n_chan, flag fraction), each drawn from its own seed."""
    out = []
    for i in range(n_prob):
        r = np.random.default_rng(seed_base + i)
        out.append((seed_base + i, int(r.integers(ant[0], ant[1] + 1)), int(r.integers(times[0], times[1] + 1)),
                    int(r.integers(chans[0], chans[1] + 1)), float(r.uniform(0.0, flag_max))))
    return out


@dataclasses.dataclass
class Batch:
    shapes: list
    data: object
    model: object
    weight: object
    flag: object
    ant1: np.ndarray
    ant2: np.ndarray
    row_offset: np.ndarray
    vis_offset: np.ndarray
    n_chan: np.ndarray
    n_ant: np.ndarray
    truths: list                 # per problem [n_ant][2] complex (g_XX, g_YY)
    setups: list

    @property
    def n_prob(self) -> int:
        return len(self.shapes)

    @property
    def n_vis(self) -> int:
        return int(self.vis_offset[-1])


def fill_interval_problems_device(sus, noise: float, noise_seed: int, data, model, weight, flag,
                                  chunk_samples: int = 1 << 23):
    """Generate many single-interval diagonal-gain problems (``interval_problem_setup`` /
    ``pair_problem_setups``) straight into flat device arrays [sum rows x chans][4], a few
    million samples per pass over the concatenation instead of one pass per problem.

    Same arithmetic as :func:`make_observation_device` (FP64 phases range-reduced, FP32
    exponentials, complex64 output); flags are the setups' own; noise comes from one device
    generator seeded with ``noise_seed``."""
    import torch
    dev = data.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(noise_seed))
    two_pi = 2.0 * np.pi
    weight.fill_(1.0)
    i, n_p, v0 = 0, len(sus), 0
    while i < n_p:
        # group problems up to ~chunk_samples samples (at least one problem)
        j, n_s = i, 0
        while j < n_p and (j == i or n_s + sus[j].ant1.size * sus[j].freqs.size <= chunk_samples):
            n_s += sus[j].ant1.size * sus[j].freqs.size
            j += 1
        grp = sus[i:j]
        n_src = grp[0].sky.flux.size
        rows = np.array([su.ant1.size for su in grp])
        ncs = np.array([su.freqs.size for su in grp])
        max_ant = max(su.n_ant for su in grp)
        uvw = np.concatenate([su.uvw for su in grp])                                   # [R, 3]
        prob_row = np.repeat(np.arange(j - i), rows)
        a1 = np.concatenate([su.ant1 for su in grp]).astype(np.int64)
        a2 = np.concatenate([su.ant2 for su in grp]).astype(np.int64)
        nc_row = ncs[prob_row]
        lmn = np.stack([np.stack([su.sky.l, su.sky.m, su.sky.n - 1.0]) for su in grp])   # [P, 3, src]
        flux = np.stack([su.sky.flux for su in grp])                                   # [P, src]
        f0 = np.array([su.freqs[0] for su in grp])
        df = np.array([su.freqs[1] - su.freqs[0] if su.freqs.size > 1 else 0.0 for su in grp])
        gains = np.ones((j - i, max_ant, 2), np.complex128)
        for k, su in enumerate(grp):
            t = su.terms[0].truth_jones()[0, 0]
            gains[k, :su.n_ant, 0] = t[:, 0]
            gains[k, :su.n_ant, 1] = t[:, 3]
        fl = np.concatenate([(np.repeat(su.flag_rows[:, None], su.freqs.size, axis=1) |
                              (su.flag_samples if su.flag_samples is not None else False)).reshape(-1)
                             for su in grp]).astype(np.uint8)
        # per-sample indices on the device
        t_ = lambda x, dt=torch.int64: torch.from_numpy(np.ascontiguousarray(x)).to(dev, dt)
        nc_row_d = t_(nc_row)
        row_s = torch.repeat_interleave(torch.arange(rows.sum(), device=dev), nc_row_d)
        row_start = torch.cumsum(nc_row_d, 0) - nc_row_d
        chan_s = torch.arange(n_s, device=dev) - row_start[row_s]
        prob_s = t_(prob_row)[row_s]
        ph_row = torch.einsum("rk,rks->rs", t_(uvw, torch.float64), t_(lmn, torch.float64)[t_(prob_row)])  # [R, src]
        freq_s = t_(f0, torch.float64)[prob_s] + t_(df, torch.float64)[prob_s] * chan_s.to(torch.float64)
        k_nu = -two_pi * freq_s / C_LIGHT
        ang = ph_row[row_s] * k_nu[:, None]                                            # [S, src]
        ang = (ang - two_pi * torch.round(ang / two_pi)).to(torch.float32)
        scal = (torch.polar(torch.ones_like(ang), ang) *
                t_(flux, torch.float32)[prob_s].to(torch.complex64)).sum(dim=1)      # [S]
        del ang
        g = t_(gains, torch.complex128).to(torch.complex64)
        gp = g[prob_s, t_(a1)[row_s]]                                                  # [S, 2]
        gq = g[prob_s, t_(a2)[row_s]]
        out = torch.zeros((n_s, 4), dtype=torch.complex64, device=dev)
        out[:, 0] = gp[:, 0] * scal * gq[:, 0].conj()
        out[:, 3] = gp[:, 1] * scal * gq[:, 1].conj()
        if noise > 0:
            nz = torch.randn((n_s, 4, 2), dtype=torch.float32, device=dev, generator=gen)
            out += noise * torch.view_as_complex(nz)
        data[v0:v0 + n_s] = out
        m = model[v0:v0 + n_s]
        m.zero_()
        m[:, 0] = scal
        m[:, 3] = scal
        flag[v0:v0 + n_s] = t_(fl, torch.uint8)
        v0 += n_s
        i = j
    assert v0 == data.shape[0]


def make_batch(shapes, noise: float = 0.01, device=None, noise_seed: int = 7) -> Batch:
    """Concatenate problems; host complex128 arrays (device=None) or complex64 device tensors
    (generated in a few large passes by :func:`fill_interval_problems_device`)."""
    row_off, vis_off = [0], [0]
    a1, a2, truths, setups = [], [], [], []
    parts = []
    for i, (seed, na, nt, nc, ff) in enumerate(shapes):
        su = interval_problem_setup(seed, na, nt, nc, ff)
        setups.append(su)
        truths.append(su.terms[0].truth[0, 0][:, [0, 3]].copy())
        if device is None:
            obs = make_observation(na, nt, su.freqs, su.terms, n_src=5, seed=seed, noise=noise, su=su)
            parts.append((obs.data, obs.model, obs.weight, obs.flag))
        a1.append(su.ant1)
        a2.append(su.ant2)
        row_off.append(row_off[-1] + su.ant1.size)
        vis_off.append(vis_off[-1] + su.ant1.size * nc)
    if device is None:
        data = np.concatenate([p_[0].reshape(-1, 4) for p_ in parts])
        model = np.concatenate([p_[1].reshape(-1, 4) for p_ in parts])
        weight = np.concatenate([p_[2].reshape(-1, 4) for p_ in parts])
        flag = np.concatenate([p_[3].reshape(-1) for p_ in parts])
    else:
        import torch
        n_vis = vis_off[-1]
        data = torch.empty((n_vis, 4), dtype=torch.complex64, device=device)
        model = torch.empty((n_vis, 4), dtype=torch.complex64, device=device)
        weight = torch.empty((n_vis, 4), dtype=torch.float32, device=device)
        flag = torch.empty(n_vis, dtype=torch.uint8, device=device)
        fill_interval_problems_device(setups, noise, noise_seed, data, model, weight, flag)
    return Batch(list(shapes), data, model, weight, flag, np.concatenate(a1).astype(np.int32),
                 np.concatenate(a2).astype(np.int32), np.array(row_off, np.int64), np.array(vis_off, np.int64),
                 np.array([s_[3] for s_ in shapes], np.int32), np.array([s_[1] for s_ in shapes], np.int32),
                 truths, setups)


# ---------------------------------------------------------------------------
# streams of consecutive intervals for the learned warm start
# ---------------------------------------------------------------------------

def drifting_diag_truth(n_ant: int, n_tint: int, n_fint: int, rng: np.random.Generator, amp_sigma: float = 0.05,
                        phase_step: float = 0.08, amp_step: float = 0.01) -> np.ndarray:
    """Diagonal gains per (time interval, frequency interval): amplitude 1+N(0,amp_sigma), phase
    U(-pi,pi) plus a smooth frequency slope, then a random walk from one time interval to the
    next (phase steps N(0, phase_step) rad, amplitude steps N(0, amp_step))."""
    amp0 = 1.0 + amp_sigma * rng.standard_normal((n_ant, 2))
    ph0 = rng.uniform(-np.pi, np.pi, size=(n_ant, 2))
    slope = 0.5 * rng.standard_normal((n_ant, 2))
    x = (np.arange(n_fint) + 0.5) / max(1, n_fint) - 0.5
    dph = np.cumsum(phase_step * rng.standard_normal((n_tint, n_ant, 2)), axis=0)
    damp = np.cumsum(amp_step * rng.standard_normal((n_tint, n_ant, 2)), axis=0)
    ph = ph0[None, None] + slope[None, None] * x[None, :, None, None] + dph[:, None]
    amp = amp0[None, None] + damp[:, None]
    g = amp * np.exp(1j * ph)                                   # [tint, fint, ant, 2]
    out = np.zeros((n_tint, n_fint, n_ant, 4), dtype=np.complex128)
    out[..., 0] = g[..., 0]
    out[..., 3] = g[..., 1]
    return out


def warmstart_observation_setup(seed: int, n_ant: int = 64, n_time: int = 300, n_chan: int = 512,
                                f_block: int = 16, n_src: int = 50) -> Setup:
    """Config-1-style observation (8 km east-west array, 50 sources, MeerKAT L-band) with one diagonal
    term on intervals of 1 time x f_block channels whose gains drift from one time to the next."""
    rng = np.random.default_rng(seed)
    freqs = meerkat_band(n_chan)
    ant_x = ew_array(n_ant, 8000.0, rng)
    n_fb = -(-n_chan // f_block)
    term = TermSpec("diag", interval_map(n_time, 1), interval_map(n_chan, f_block), n_time, n_fb)
    term.truth = drifting_diag_truth(n_ant, n_time, n_fb, rng)
    return draw_setup(n_ant, n_time, freqs, [term], n_src=n_src, rng=rng, ant_x=ant_x, flag_row_frac=0.05)


def pair_problem_setups(seed: int, n_ant: int, n_time: int, n_chan: int, flag_frac: float, n_src: int = 5):
    """Two consecutive solution intervals of one stream (same array and sky): the previous interval
    and the current one, n_time integrations of 8 s each, with the gains drifted in between."""
    rng = np.random.default_rng(seed)
    freqs = 1.4e9 + 1.0e6 * (np.arange(n_chan) - (n_chan - 1) / 2.0)
    ant_x = ew_array(n_ant, 1000.0, rng)
    truth = drifting_diag_truth(n_ant, 2, 1, rng)
    centre = rng.uniform(-2.0, 2.0)
    span = n_time * 8.0 / 3600.0
    sky_seed = int(rng.integers(1 << 31))
    out = []
    for k, c in enumerate((centre - span, centre)):
        term = TermSpec("diag", np.zeros(n_time, np.int32), np.zeros(n_chan, np.int32), 1, 1)
        term.truth = truth[k:k + 1]
        r = np.random.default_rng(sky_seed)          # same sky for both intervals
        su = draw_setup(n_ant, n_time, freqs, [term], n_src=n_src, rng=r, ant_x=ant_x, flag_sample_frac=flag_frac,
                        ha_span_hours=span, ha_centre_hours=c)
        su.rng = np.random.default_rng(seed * 7 + k + 1)
        out.append(su)
    return out


def make_pair_batches(shapes, noise: float = 0.01, device=None, noise_seed: int = 11, which=(0, 1)):
    """(previous-interval batch, current-interval batch) for problems of the given shapes, written
    straight into preallocated arrays (no concatenation copies).  ``which`` selects the batches to
    build (0: previous, 1: current); the others are returned as None."""
    setups = [pair_problem_setups(seed, na, nt, nc, ff) for (seed, na, nt, nc, ff) in shapes]
    batches = [None, None]
    for k in which:
        sus = [s_[k] for s_ in setups]
        row_off = np.concatenate([[0], np.cumsum([su.ant1.size for su in sus])]).astype(np.int64)
        vis_off = np.concatenate([[0], np.cumsum([su.ant1.size * su.freqs.size for su in sus])]).astype(np.int64)
        n_vis = int(vis_off[-1])
        if device is None:
            data = np.zeros((n_vis, 4), np.complex128)
            model = np.zeros((n_vis, 4), np.complex128)
            weight = np.zeros((n_vis, 4))
            flag = np.zeros(n_vis, np.uint8)
        else:
            import torch
            data = torch.empty((n_vis, 4), dtype=torch.complex64, device=device)
            model = torch.empty((n_vis, 4), dtype=torch.complex64, device=device)
            weight = torch.empty((n_vis, 4), dtype=torch.float32, device=device)
            flag = torch.empty(n_vis, dtype=torch.uint8, device=device)
        if device is None:
            for i, su in enumerate(sus):
                v0, v1 = vis_off[i], vis_off[i + 1]
                o = make_observation(su.n_ant, su.n_time, su.freqs, su.terms, n_src=5, seed=0, noise=noise, su=su)
                data[v0:v1] = o.data.reshape(-1, 4)
                model[v0:v1] = o.model.reshape(-1, 4)
                weight[v0:v1] = o.weight.reshape(-1, 4)
                flag[v0:v1] = o.flag.reshape(-1)
        else:
            fill_interval_problems_device(sus, noise, noise_seed + k, data, model, weight, flag)
        truths = [su.terms[0].truth[0, 0][:, [0, 3]].copy() for su in sus]
        batches[k] = (Batch(list(shapes), data, model, weight, flag,
                             np.concatenate([su.ant1 for su in sus]).astype(np.int32),
                             np.concatenate([su.ant2 for su in sus]).astype(np.int32), row_off, vis_off,
                             np.array([s_[3] for s_ in shapes], np.int32), np.array([s_[1] for s_ in shapes], np.int32),
                             truths, sus))
    return batches[0], batches[1]


# ---------------------------------------------------------------------------
# the KdE workload: two directions, a delay term K and a direction-dependent dE
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class KdESetup:
    """Host-drawn part of the KdE workload (Section 5: K per integration over all channels; dE,
    direction-dependent diagonal, over 16 integrations x 128 channels; two directions: the
    field and one bright source away from it)."""
    base: Setup                # array, rows, uvw, flagged rows, field sky (direction 0)
    off: Sky                   # direction 1: the off-axis source
    freqs_ghz: np.ndarray      # channel frequencies in GHz (the delay term's frequency axis)
    k_truth: np.ndarray        # float [n_time][1][n_ant][4] (phi_X, tau_X ns, phi_Y, tau_Y ns)
    k_tmap: np.ndarray
    de_truth: np.ndarray       # complex [n_tint][n_fint][n_ant][2][4]
    de_tmap: np.ndarray
    de_fmap: np.ndarray


def kde_setup(seed: int = 3, n_ant: int = 64, n_time: int = 300, n_chan: int = 512, n_src: int = 50,
              flag_row_frac: float = 0.1, de_times: int = 16, de_chans: int = 128) -> KdESetup:
    rng = np.random.default_rng(seed)
    freqs = meerkat_band(n_chan)
    ant_x = ew_array(n_ant, 8000.0, rng)
    base = draw_setup(n_ant, n_time, freqs, [], n_src=n_src - 1, rng=rng, ant_x=ant_x, flag_row_frac=flag_row_frac)
    # the off-axis source: 5 Jy at 1.5 degrees
    ang = rng.uniform(0, 2 * np.pi)
    l, m = np.deg2rad(1.5) * np.cos(ang), np.deg2rad(1.5) * np.sin(ang)
    off = Sky(flux=np.array([5.0]), l=np.array([l]), m=np.array([m]))
    k = np.zeros((n_time, 1, n_ant, 4))
    k[..., 0] = rng.uniform(-np.pi, np.pi, (n_time, 1, n_ant))
    k[..., 2] = rng.uniform(-np.pi, np.pi, (n_time, 1, n_ant))
    tau = rng.normal(0.0, 1.0, (1, 1, n_ant, 2)) + 0.05 * np.cumsum(rng.normal(0, 1, (n_time, 1, n_ant, 2)), axis=0)
    k[..., 1], k[..., 3] = tau[..., 0], tau[..., 1]
    nt, nf = -(-n_time // de_times), -(-n_chan // de_chans)
    de = np.zeros((nt, nf, n_ant, 2, 4), dtype=np.complex128)
    amp = np.stack([1 + 0.02 * rng.standard_normal((nt, nf, n_ant, 2)),
                    1 + 0.1 * rng.standard_normal((nt, nf, n_ant, 2))], axis=3)
    ph = np.stack([0.05 * rng.standard_normal((nt, nf, n_ant, 2)),
                   rng.uniform(-np.pi, np.pi, (nt, nf, n_ant, 2))], axis=3)
    g = amp * np.exp(1j * ph)                                              # [nt, nf, ant, dir, corr]
    de[..., 0], de[..., 3] = g[..., 0], g[..., 1]
    return KdESetup(base, off, freqs / 1e9, k, interval_map(n_time, 1), de, interval_map(n_time, de_times),
                    interval_map(n_chan, de_chans))


def make_kde_device(ks: KdESetup, noise: float, noise_seed: int, device, rows_per_chunk: int = 2048):
    """The KdE observation on a CUDA device: data complex64 [row][chan][4], model complex64
    [row][chan][2][4] (direction 0: the field, 1: the off-axis source), float32 weights, uint8
    flags.  data = sum_d K_p dE_{p,d} M_d dE_{q,d}^H K_q^H + noise (complex Gaussian, re and im
    each N(0, noise^2))."""
    import torch
    su = ks.base
    n_row, n_chan = su.ant1.size, su.freqs.size
    dev = torch.device(device)
    f64, c64 = torch.float64, torch.complex64
    data = torch.empty((n_row, n_chan, 4), dtype=c64, device=dev)
    model = torch.zeros((n_row, n_chan, 2, 4), dtype=c64, device=dev)
    weight = torch.ones((n_row, n_chan, 4), dtype=torch.float32, device=dev)
    flag = torch.from_numpy(np.repeat(su.flag_rows[:, None], n_chan, axis=1).astype(np.uint8)).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(noise_seed))
    k_nu = torch.from_numpy(-2.0 * np.pi * su.freqs / C_LIGHT).to(dev, f64)
    skies = [su.sky, ks.off]
    flux = [torch.from_numpy(s.flux).to(dev, torch.float32).to(c64) for s in skies]
    lmn = [torch.from_numpy(np.stack([s.l, s.m, s.n - 1.0])).to(dev, f64) for s in skies]
    nu = torch.from_numpy(ks.freqs_ghz).to(dev, f64)
    kt = torch.from_numpy(ks.k_truth[:, 0]).to(dev, f64)                    # [time, ant, 4]
    de = torch.from_numpy(ks.de_truth).to(dev, c64)                         # [nt, nf, ant, dir, 4]
    de_t = torch.from_numpy(ks.de_tmap.astype(np.int64)).to(dev)
    de_f = torch.from_numpy(ks.de_fmap.astype(np.int64)).to(dev)
    two_pi = 2.0 * np.pi

    def k_gain(t, a):                                                        # [R, C, 2] complex64
        u = kt[t, a]                                                         # [R, 4]
        px = u[:, 0:1] + two_pi * u[:, 1:2] * nu[None, :]
        py = u[:, 2:3] + two_pi * u[:, 3:4] * nu[None, :]
        return torch.stack([torch.polar(torch.ones_like(px), px), torch.polar(torch.ones_like(py), py)], -1).to(c64)

    for r0 in range(0, n_row, rows_per_chunk):
        r1 = min(n_row, r0 + rows_per_chunk)
        uvw = torch.from_numpy(su.uvw[r0:r1]).to(dev, f64)
        t = torch.from_numpy(su.time_idx[r0:r1].astype(np.int64)).to(dev)
        a1 = torch.from_numpy(su.ant1[r0:r1].astype(np.int64)).to(dev)
        a2 = torch.from_numpy(su.ant2[r0:r1].astype(np.int64)).to(dev)
        kp, kq = k_gain(t, a1), k_gain(t, a2)
        it = de_t[t][:, None]
        jf = de_f[None, :]
        V = torch.zeros((r1 - r0, n_chan, 2), dtype=c64, device=dev)        # parallel hands (diagonal chain)
        for d in range(2):
            ang = (uvw @ lmn[d])[:, :, None] * k_nu[None, None, :]
            ang = (ang - two_pi * torch.round(ang / two_pi)).to(torch.float32)
            scal = torch.einsum("k,rkc->rc", flux[d], torch.polar(torch.ones_like(ang), ang))
            model[r0:r1, :, d, 0] = scal
            model[r0:r1, :, d, 3] = scal
            ep = de[it, jf, a1[:, None], d][..., [0, 3]]                        # [R, C, 2]
            eq = de[it, jf, a2[:, None], d][..., [0, 3]]
            V += (kp * ep) * scal[:, :, None] * (kq * eq).conj()
        out = torch.zeros((r1 - r0, n_chan, 4), dtype=c64, device=dev)
        out[..., 0], out[..., 3] = V[..., 0], V[..., 1]
        if noise > 0:
            nz = torch.randn((r1 - r0, n_chan, 4, 2), dtype=torch.float32, device=dev, generator=gen)
            out = out + noise * torch.view_as_complex(nz)
        data[r0:r1] = out
    return dict(data=data, model=model, weight=weight, flag=flag, ant1=su.ant1, ant2=su.ant2,
                time_idx=su.time_idx, n_ant=su.n_ant, n_time=su.n_time, n_chan=n_chan)
