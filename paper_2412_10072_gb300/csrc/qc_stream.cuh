// qc_stream.cuh -- streaming accumulate kernel for chains of one or two terms.
//
// Same arithmetic as acc_kernel (the residual r = D - L_p G_p R_p M C_q^H of every
// sample and its contributions to the per-(interval, antenna) blocks of J^H W J and
// J^H W r of both antennas, Eq. jhj_entry_simplified, Eq. jhr_entry_simplified),
// organised so that nothing on a warp's critical path waits for a dependent load:
//
//  * the rows are visited through a step-major row table rt[k] = {row, p | q << 16,
//    t_int of the solved term (-1: nothing to read), t_int of the other term},
//    built once per term solve in the order of the tiles (row tiles: row order;
//    strip tiles: the rows of each baseline in time order), so a warp step --
//    one row x 32 channels -- has its antennas and interval indices in one entry;
//  * flags are folded into the weights when the problem is created (w = 0 for a
//    flagged sample or an autocorrelation), so a step reads d, m and w only, and a
//    sample whose four weights are zero is skipped (a select, so non-finite data in
//    flagged cells does not propagate);
//  * d, m, w of each step are copied DEPTH - 1 steps ahead into the warp's ring in
//    shared memory (16-byte cp.async per lane, zero-filled for lanes with nothing to
//    read), and lane 0 writes the step's row-table entry beside them;
//  * the J^H W r slots receive J^H W d: the model V = E g is linear in the solved gains of
//    either side, so J^H W r = J^H W d - JHJ g per (interval, antenna) block, formed in FP64
//    by the update; a sample forms neither V nor the residual;
//  * the lane's channel interval indices are read two steps ahead; the solved term's
//    gain entries stay in registers while their table index is unchanged (a row of a
//    row tile, a strip of a strip tile), and the gain loads of a step are issued at
//    its top, before the next copy is issued, which covers their latency (the gain
//    tables are small and stay in L2; an L1 prefetch a step ahead cost more issue
//    slots than it saved).
//
// Work decomposition as in acc_kernel: a unit is a row (row tiles: its 32-channel
// chunks are the steps) or a baseline strip x 32 channels (strip tiles: its rows
// are the steps).  Row tiles go to warps with a grid stride; strip tiles, a few hundred
// steps each, are handed out one at a time by an atomic counter as warps finish, so the
// launch does not wait on warps that drew one unit more than the rest.  Register sums are flushed
// (segmented warp reduction + FP64 atomics) when the antenna pair or any lane's
// interval bin changes.
#pragma once
#include "qc_kernels.cuh"

namespace qc {

struct StreamArgs {
    const float4 *vis;          // [n_row][n_chan] x 2
    const float4 *model;        // [n_row][n_chan] x 2, or null (FP16 model)
    const uint4 *model16;       // [n_row][n_chan] (4 half2), or null
    const float4 *wf;           // [n_row][n_chan] weights with flags folded in
    int n_chan, n_ant;
    const int4 *rt;             // step-major row table (see above)
    const float *rt_scale;      // [rt] FP16 model scale of the entry's baseline, or null
    const int *unit_off;        // strip tiles: [n_strips + 1] offsets into rt
    int order;                  // 0 row tiles, 1 strip tiles
    int n_units, n_chunks;
    DevTerm tn, to;             // solved term, other term (a copy of tn when there is none)
    const int2 *fmap2;          // [n_chan] {f_map of the solved term, f_map of the other term}
    const uint8_t *chunk_active;// [tn.n_tint][n_chunks]
    const uint8_t *active;      // [bins of the solved term]
    const int *n_active;        // nonzero: some interval still iterating
    double *acc;                // [bins][n_ant][KG]
    int *unit_counter;          // strip tiles: next unit to hand out (zero before the launch), or null
};

constexpr int STREAM_END = -2;  // row-table field marking the end of a warp's stream


__host__ __device__ constexpr int next_pow2(int n) { return n <= 1 ? 1 : 2 * next_pow2((n + 1) / 2); }

// Transposed reduction of one side's register sums when the whole warp is in one bin:
// every exchange halves the values a lane holds, so KR values take about KR shuffles
// (instead of 5 per value) and end as one total per lane, added with one atomic instruction.
template <int KR, int KG, typename Lay>
__device__ __forceinline__ void flush_side_warp(Acc<KR, false> &A, int key, int ant, int lane, bool live,
                                                double *__restrict__ acc, int n_ant)
{
    constexpr int NP = next_pow2(KR), R = NP >= 32 ? NP / 32 : 1;
    float v[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) v[i] = i < KR ? A.s[i] : 0.f;
    int idx = 0;
#pragma unroll
    for (int lev = 0; lev < 5; ++lev) {
        const int d = 16 >> lev;
        const int h = NP >> (lev + 1);
        const bool up = (lane & d) != 0;
        if (h >= 1) {
#pragma unroll
            for (int i = 0; i < NP / 2; ++i) {
                if (i < h) {
                    const float send = up ? v[i] : v[i + h];
                    const float keep = up ? v[i + h] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, d);
                }
            }
            if (up) idx += h;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], d);
        }
    }
    // lanes holding the same total after the plain butterfly levels: the lowest writes
    const bool writer = NP >= 32 || (lane & (32 / NP - 1)) == 0;
    if (writer && live) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = idx + r;
            if (j < KR) atomicAdd(acc + ((size_t)key * n_ant + ant) * KG + Lay::g(j), (double)v[r]);
        }
    }
    A.zero();
}

// Flush both sides' register sums (antennas p and q of the warp's current step) to the
// FP64 accumulators of bin `key` (per lane; -1 for lanes without a sample):
//  * one bin for the whole warp (row tiles of an interval wider than 32 channels): the
//    transposed reduction above, one side at a time;
//  * a different bin in every lane: no reduction, each lane adds its own sums;
//  * otherwise a segmented reduction over runs of lanes with equal bins (flush_side).
// The first two are compiled only where they fit the kernel's 128 registers without
// spilling (up to 16 sums per side, and up to 8 for the per-lane path).
template <int KR, int KG, typename Lay>
__device__ __forceinline__ void flush_pair(Acc<KR, false> &Ap, Acc<KR, false> &Aq, int key, int pq, int lane,
                                           const uint8_t *__restrict__ active, double *__restrict__ acc, int n_ant)
{
    const int p = pq & 0xffff, q = pq >> 16;
    if constexpr (KR <= 16) {
        const int k0 = __shfl_sync(0xffffffffu, key, 0);
        if (__all_sync(0xffffffffu, key == k0)) {
            const bool live = k0 >= 0 && __ldg(active + k0);
            flush_side_warp<KR, KG, Lay>(Ap, k0, p, lane, live, acc, n_ant);
            flush_side_warp<KR, KG, Lay>(Aq, k0, q, lane, live, acc, n_ant);
            return;
        }
    }
    const unsigned m = __match_any_sync(0xffffffffu, key);
    const bool live = key >= 0 && __ldg(active + key);
    if (KR <= 8 && __all_sync(0xffffffffu, m == (1u << lane))) {
        if (live) {
#pragma unroll
            for (int i = 0; i < KR; ++i) {
                atomicAdd(acc + ((size_t)key * n_ant + p) * KG + Lay::g(i), (double)Ap.s[i]);
                atomicAdd(acc + ((size_t)key * n_ant + q) * KG + Lay::g(i), (double)Aq.s[i]);
            }
        }
        Ap.zero();
        Aq.zero();
        return;
    }
    const unsigned seg_end = 32 - __clz(m);
    const bool head = lane == __ffs(m) - 1;
    flush_side<KR, KG, false, Lay>(Ap, key, p, lane, seg_end, head, live, acc, n_ant);
    flush_side<KR, KG, false, Lay>(Aq, key, q, lane, seg_end, head, live, acc, n_ant);
}

// Issue side of a warp's stream: walks the warp's units (grid stride W, or the unit
// counter) and their
// steps, and for each step copies the 32 lanes' d, m, w into a ring stage
// (16-byte cp.async per lane, zero-filled where there is nothing to read) and
// writes the step's row-table entry and channel offset beside them (lane 0).
template <bool M16> struct StreamCursor {
    static constexpr int V4 = M16 ? 4 : 5;
    int iu, W;                   // unit, grid stride in units
    int ii = 0, ilen = 0;        // step within the unit, steps in the unit
    int ikb = 0, ic0 = 0;        // strip tiles: first rt entry of the unit, first channel of its chunk
    int4 irt = make_int4(0, 0, -1, 0);   // row tiles: the unit's row-table entry
    float isc = 0.f;
    unsigned imask = 0;          // row tiles: active 32-channel chunks of the row (bit per chunk)
    int4 blk = make_int4(0, 0, -1, 0);   // strip tiles: entries of the current 32-step block, one per lane
    float blks = 0.f;
    unsigned blkact = 0;
    int blk_base = -1;

    // find the next unit with something to read (sets ilen > 0) or run out (iu >= n_units)
    __device__ __forceinline__ void unit_start(const StreamArgs &a, int lane)
    {
        const int nch = a.n_chunks;
        ii = 0;
        ilen = 0;
        while (iu < a.n_units) {
            if (a.order == 0) {
                irt = __ldg(a.rt + iu);
                if (irt.z >= 0) {
                    unsigned m = 0;
                    for (int c0 = 0; c0 < nch; c0 += 32) {
                        const bool act = c0 + lane < nch && __ldg(a.chunk_active + (size_t)irt.z * nch + c0 + lane);
                        const unsigned b = __ballot_sync(0xffffffffu, act);
                        if (c0 == 0) m = b;
                        else if (b) m |= 0x80000000u;    // chunks >= 32: read (activity checked per lane)
                    }
                    imask = m;
                    if (m) {
                        isc = M16 ? __ldg(a.rt_scale + iu) : 0.f;
                        ilen = nch;
                        return;
                    }
                }
            } else {
                const int s = iu / nch;
                ic0 = (iu - s * nch) * 32;
                ikb = __ldg(a.unit_off + s);
                ilen = __ldg(a.unit_off + s + 1) - ikb;
                blk_base = -1;
                if (ilen > 0) return;
            }
            next_unit(a, lane);
        }
    }

    // next unit of this warp: a grid stride (row tiles), or the next one handed out by the
    // launch's counter (strip tiles: units of a few hundred steps, taken as warps free up so
    // that no warp is left with a last unit while the others idle)
    __device__ __forceinline__ void next_unit(const StreamArgs &a, int lane)
    {
        if (a.unit_counter) {
            int u = 0;
            if (lane == 0) u = atomicAdd(a.unit_counter, 1);
            iu = __shfl_sync(0xffffffffu, u, 0);
        } else {
            iu += W;
        }
    }

    __device__ __forceinline__ void start(const StreamArgs &a, int lane, int first_unit, int stride)
    {
        W = stride;
        if (a.unit_counter) {
            iu = 0;
            W = 0;
            int u = 0;
            if (lane == 0) u = atomicAdd(a.unit_counter, 1);
            iu = __shfl_sync(0xffffffffu, u, 0);
        } else {
            iu = first_unit;
        }
        unit_start(a, lane);
    }

    // copy the next step into ring stage `stage` (one commit group) and advance
    __device__ __forceinline__ void issue(const StreamArgs &a, int lane, float4 *ring, int4 *meta, int stage)
    {
        int4 e = make_int4(STREAM_END, 0, -1, 0);
        float sc = 0.f;
        int c0 = 0;
        bool live = false;
        if (iu < a.n_units) {
            if (a.order == 0) {
                e = irt;
                sc = isc;
                c0 = ii * 32;
                live = ii >= 31 ? ((imask >> 31) & 1) : ((imask >> ii) & 1);
            } else {
                const int b = ii >> 5, l = ii & 31;
                if (b != blk_base) {
                    blk_base = b;
                    const int j = b * 32 + lane;
                    const bool in = j < ilen;
                    blk = in ? __ldg(a.rt + ikb + j) : make_int4(0, 0, -1, 0);
                    blks = (M16 && in) ? __ldg(a.rt_scale + ikb + j) : 0.f;
                    const bool act = in && blk.z >= 0 && __ldg(a.chunk_active + (size_t)blk.z * a.n_chunks + (ic0 >> 5));
                    blkact = __ballot_sync(0xffffffffu, act);
                }
                e.x = __shfl_sync(0xffffffffu, blk.x, l);
                e.y = __shfl_sync(0xffffffffu, blk.y, l);
                e.z = __shfl_sync(0xffffffffu, blk.z, l);
                e.w = __shfl_sync(0xffffffffu, blk.w, l);
                sc = __shfl_sync(0xffffffffu, blks, l);
                c0 = ic0;
                live = (blkact >> l) & 1;
            }
            if (!live) e.z = -1;
        }
        const int c = c0 + lane;
        const bool rd = live && c < a.n_chan;
        const size_t s = rd ? (size_t)e.x * a.n_chan + c : 0;
        const uint32_t nb = rd ? 16u : 0u;
        float4 *slot = ring + (size_t)stage * V4 * 32 + lane;
        cp_async16(slot, a.vis + 2 * s, nb);
        cp_async16(slot + 32, a.vis + 2 * s + 1, nb);
        if constexpr (M16) {
            cp_async16(slot + 64, a.model16 + s, nb);
            cp_async16(slot + 96, a.wf + s, nb);
        } else {
            cp_async16(slot + 64, a.model + 2 * s, nb);
            cp_async16(slot + 96, a.model + 2 * s + 1, nb);
            cp_async16(slot + 128, a.wf + s, nb);
        }
        cp_async_commit();
        if (lane == 0) {
            meta[2 * stage] = e;
            meta[2 * stage + 1] = make_int4(c0, __float_as_int(sc), 0, 0);
        }
        if (iu < a.n_units && ++ii == ilen) {
            next_unit(a, lane);
            unit_start(a, lane);
        }
    }

    // row tiles of a model with a direction axis: d, w and the sample's n_mw model words
    // (contiguous, [dir][2] float4) into a stage laid out [d0][d1][w][m_0] .. [m_{n_mw-1}]
    __device__ __forceinline__ void issue_dd(const StreamArgs &a, int lane, float4 *ring, int4 *meta, int stage,
                                             int n_mw)
    {
        int4 e = make_int4(STREAM_END, 0, -1, 0);
        int c0 = 0;
        bool live = false;
        if (iu < a.n_units) {
            e = irt;
            c0 = ii * 32;
            live = ii >= 31 ? ((imask >> 31) & 1) : ((imask >> ii) & 1);
            if (!live) e.z = -1;
        }
        const int c = c0 + lane;
        const bool rd = live && c < a.n_chan;
        const size_t s = rd ? (size_t)e.x * a.n_chan + c : 0;
        const uint32_t nb = rd ? 16u : 0u;
        float4 *slot = ring + (size_t)stage * (3 + n_mw) * 32 + lane;
        cp_async16(slot, a.vis + 2 * s, nb);
        cp_async16(slot + 32, a.vis + 2 * s + 1, nb);
        cp_async16(slot + 64, a.wf + s, nb);
        const float4 *ms = a.model + s * n_mw;
        for (int i = 0; i < n_mw; ++i) cp_async16(slot + 96 + 32 * i, ms + i, nb);
        cp_async_commit();
        if (lane == 0) {
            meta[2 * stage] = e;
            meta[2 * stage + 1] = make_int4(c0, 0, 0, 0);
        }
        if (iu < a.n_units && ++ii == ilen) {
            next_unit(a, lane);
            unit_start(a, lane);
        }
    }
};

template <int TS, int LK, int RK, bool M16, int DEPTH>
__global__ void __launch_bounds__(256, 2) acc_stream_kernel(const StreamArgs a)
{
    if (__ldg(a.n_active) == 0) return;
    constexpr bool HAS_L = LK != KIND_NONE;
    constexpr int GK = TS == TS_FULL ? KIND_FULL : KIND_DIAG;
    // FP16 model: instead of a compensated add per sample, the lane sums go to the FP64
    // accumulators at least every FLUSH_EVERY steps, so FP32 rounding is confined to
    // partial sums of at most FLUSH_EVERY samples per lane and everything beyond is FP64
    constexpr bool KAHAN = false;
    constexpr int FLUSH_EVERY = M16 ? 16 : (1 << 30);
    using Lay = AccLayout<TS, HAS_L>;
    constexpr int KR = Lay::KR, KG = Lay::KG;
    constexpr int V4 = M16 ? 4 : 5;                         // 16-byte words per sample: d (2), m (2 or 1), w (1)
    static_assert(DEPTH >= 3, "the entry of the next step must be in the ring");
    extern __shared__ float4 s_stream[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float4 *ring = s_stream + (size_t)wib * DEPTH * V4 * 32;                          // [DEPTH][V4][32]
    int4 *meta = reinterpret_cast<int4 *>(s_stream + (size_t)nw * DEPTH * V4 * 32) + (size_t)wib * DEPTH * 2;
    const int W = (int)((gridDim.x * blockDim.x) >> 5);
    const int n_chan = a.n_chan, n_ant = a.n_ant;

    // ---------------- issue side: the step DEPTH - 1 ahead of the arithmetic ----------------
    StreamCursor<M16> cur;
    cur.start(a, lane, (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), W);
    int stage_i = 0;
    auto issue = [&]() {
        cur.issue(a, lane, ring, meta, stage_i);
        if (++stage_i == DEPTH) stage_i = 0;
    };

#pragma unroll
    for (int d = 0; d < DEPTH - 1; ++d) issue();
    __syncwarp();

    // ---------------- arithmetic side ----------------
    Acc<KR, KAHAN> Ap, Aq;
    Ap.zero();
    Aq.zero();
    int stage = 0, cur_key = -1, cur_pq = -1;
    // the ring entry of the current step (A) and the lane's channel interval maps are carried
    // in registers; each step reads the next step's (B) entry from shared memory and its maps
    // from global memory, one step ahead of their use
    auto read_map = [&](const int4 &m0, const int4 &m1) {
        const int c = m1.x + lane;
        return (m0.x != STREAM_END && m0.z >= 0 && c < n_chan) ? __ldg(a.fmap2 + c) : make_int2(0, 0);
    };
    int4 eA0 = meta[0], eA1 = meta[1];
    int2 fmA = read_map(eA0, eA1);
    int ci_p = -1, ci_q = -1, act_key = -1, since_flush = 0;
    bool act_val = false;
    J2 cGp = j_identity(), cGq = j_identity();
    // a step in two parts: (A) its entries, the other term's and the solved term's gain entries,
    // the issue of the copy DEPTH - 1 steps ahead, the wait and the lane's key; (B) the sample's
    // arithmetic and the advance.  Runs of steps that need no flush stay in an inner loop that
    // only adds; a flush leaves it (keeping the register sums out of the flush's code path in
    // the loop that runs every step), then the step's part B follows.
    int4 e = eA0, e1 = eA1, eB0 = eA0, eB1 = eA1;
    int2 fm = fmA, fmB = fmA;
    int nst = 0, key = -1;
    bool in = false, live = false;
    J2 Lp, Lq, Rp, Rq;
    auto part_a = [&]() -> bool {
        e = eA0;
        e1 = eA1;
        if (e.x == STREAM_END) return false;
        fm = fmA;
        nst = stage + 1 == DEPTH ? 0 : stage + 1;
        // the next step: its entry and channel maps
        eB0 = meta[2 * nst];
        eB1 = meta[2 * nst + 1];
        fmB = read_map(eB0, eB1);
        // this step's entries of the other term, loaded here so that the issue below covers
        // their latency
        if (e.z >= 0) {
            const int p = e.y & 0xffff, q = e.y >> 16;
            if constexpr (LK != KIND_NONE) {
                Lp = fetch_k<LK>(a.to, n_ant, e.w, fm.y, p);
                Lq = fetch_k<LK>(a.to, n_ant, e.w, fm.y, q);
            }
            if constexpr (RK != KIND_NONE) {
                Rp = fetch_k<RK>(a.to, n_ant, e.w, fm.y, p);
                Rq = fetch_k<RK>(a.to, n_ant, e.w, fm.y, q);
            }
            // the solved term's entries stay in registers while the lane's table index is unchanged
            const bool inr = e1.x + lane < n_chan;
            const int ip = inr ? (e.z * n_ant + p) * a.tn.n_fint + fm.x : ci_p;
            const int iq = inr ? (e.z * n_ant + q) * a.tn.n_fint + fm.x : ci_q;
            if (__any_sync(0xffffffffu, ip != ci_p || iq != ci_q)) {
                if (ip != ci_p) { cGp = fetch_k<GK>(a.tn, n_ant, e.z, fm.x, p); ci_p = ip; }
                if (iq != ci_q) { cGq = fetch_k<GK>(a.tn, n_ant, e.z, fm.x, q); ci_q = iq; }
            }
        }
        issue();
        cp_async_wait<DEPTH - 1>();
        __syncwarp();
        live = e.z >= 0;                            // warp-uniform
        const int c = e1.x + lane;
        in = live && c < n_chan;
        key = in ? e.z * a.tn.n_fint + fm.x : -1;
        return true;
    };
    auto part_b = [&]() {
        const float4 *slot = ring + (size_t)stage * V4 * 32 + lane;
        const float4 w = slot[M16 ? 96 : 128];
        bool ok = in && (w.x != 0.f || w.y != 0.f || w.z != 0.f || w.w != 0.f);
        if (ok && key != act_key) {          // activity of the lane's bin, read when the bin changes
            act_key = key;
            act_val = __ldg(a.active + key) != 0;
        }
        ok = ok && act_val;
        if (ok) {
            const J2 Dm = j_from(slot[0], slot[32]);
            J2 M;
            if constexpr (M16) M = load_model16(*reinterpret_cast<const uint4 *>(slot + 64), __int_as_float(e1.y));
            else M = j_from(slot[64], slot[96]);
            const J2 Gp = cGp, Gq = cGq;
            sample_math<TS, LK, RK, KAHAN, true>(Lp, Gp, Rp, Lq, Gq, Rq, Dm, M, w, Ap, Aq);
        }
        fmA = fmB;
        eA0 = eB0;
        eA1 = eB1;
        stage = nst;
    };
    for (;;) {
        bool ended = false;
        for (;;) {
            if (!part_a()) { ended = true; break; }
            if (live) {
                bool change = e.y != cur_pq || key != cur_key;
                if constexpr (M16) change = change || since_flush >= FLUSH_EVERY;
                if constexpr (M16) ++since_flush;
                if (__any_sync(0xffffffffu, change && cur_key >= 0)) break;
                cur_key = key;
                cur_pq = e.y;
            }
            part_b();
        }
        if (ended) break;
        if constexpr (M16) since_flush = 1;
        flush_pair<KR, KG, Lay>(Ap, Aq, cur_key, cur_pq, lane, a.active, a.acc, n_ant);
        cur_key = key;
        cur_pq = e.y;
        part_b();
    }
    if (__any_sync(0xffffffffu, cur_key >= 0)) flush_pair<KR, KG, Lay>(Ap, Aq, cur_key, cur_pq, lane, a.active, a.acc, n_ant);
    cp_async_wait<0>();
}

// Step-major row table of a term solve: entry k of the tile order (row tiles: row k;
// strip tiles: the k-th row of the strip order) -> {row, p | q << 16, t_int of the
// solved term or -1 (no usable data), t_int of the other term}; for the FP16 model
// also the scale of the row's baseline.
static __global__ void row_table_kernel(int n, const int *order_rows, const int4 *row_info, const int4 *rows,
                                        const float *bl_scale, int4 *rt, float *rt_scale)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int row = order_rows ? order_rows[k] : (int)k;
    const int4 ri = row_info[row];
    rt[k] = make_int4(row, ri.x | (ri.y << 16), ri.z, ri.w);
    if (rt_scale) rt_scale[k] = bl_scale[rows[row].w];
}

// w_f = w where the sample is usable (unflagged cross-correlation), else 0
static __global__ void fold_flags_kernel(const float4 *w, const uint8_t *flag, const int4 *rows, long n_row, int n_chan,
                                         float4 *wf)
{
    const long n = n_row * n_chan;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int4 r = rows[i / n_chan];
        const bool use = r.x != r.y && !(flag && flag[i]);
        wf[i] = use ? w[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

} // namespace qc
