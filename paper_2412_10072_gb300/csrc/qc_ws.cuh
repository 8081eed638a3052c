// qc_ws.cuh -- warp-specialised accumulate kernel for chains of one or two terms.
//
// Same arithmetic as acc_stream_kernel: the residual r = D - L_p G_p R_p M C_q^H of every
// sample and its contributions to the per-(interval, antenna) blocks of J^H W J and J^H W r
// of both antennas of the baseline (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified; the
// q side through the conjugate baseline), for every solution interval at once.  What
// differs is who moves the data:
//
//  * warp 0 of a CTA is the producer; warps 1..NC are consumers.  Lane i of the producer
//    drives consumer warp i: it walks that warp's stream of steps (one row x 32 channels
//    each) and, for every step, issues 1-D cp.async.bulk copies of the contiguous spans of
//    d, m and the folded weights, of the step's 32 channel maps and of the other term's
//    Jones entries for antennas p and q, all completing the transaction count of one
//    stage's "full" mbarrier in the consumer's DEPTH-deep ring in shared memory.  The
//    step's antennas, interval indices and first channel go in the stage's header.
//  * consumer warps wait on "full", read the stage from shared memory, do the sample
//    arithmetic into register sums (flushed to FP64 accumulators when the antenna pair or
//    a lane's interval bin changes, exactly as in the streaming kernel) and release the
//    stage through its "empty" mbarrier.  They issue no copies, keep no cursor and load
//    nothing from global memory but the solved term's entries (kept in registers while
//    their index is unchanged) and the activity of their bins.
//  * which steps to copy is decided per launch by a small preparation kernel from the
//    intervals still active: row tiles get a compacted list of rows with an active
//    32-channel chunk and a bit per chunk, strip tiles a bit per (chunk, row-table entry).
//    The producer finds the next step with bit operations and loads its row-table entry
//    one step ahead, so none of its loads is on the critical path of a copy.
//
// Every wait is bounded in wall time.  A wait that gives up sets *err and the CTA-wide
// abort flag; the other warps leave their loops, each consumer waits (bounded) for the
// copies still in flight into its ring, and the kernel returns.
#pragma once
#include "qc_stream.cuh"

namespace qc {

struct WsArgs {
    const float4 *vis;            // [n_row][n_chan] x 2
    const float4 *model;          // [n_row][n_chan] x 2, or null (FP16 model)
    const uint4 *model16;         // [n_row][n_chan] (4 half2), or null
    const float4 *wf;             // [n_row][n_chan] weights with flags folded in
    int n_chan, n_ant;
    int order;                    // 0 row tiles, 1 strip tiles
    int n_chunks;                 // ceil(n_chan / 32)
    // row tiles: the rows with an active chunk in this launch (compacted by the preparation
    // kernel) -- entry {row, p | q << 16, t_int solved, t_int other}, FP16 scale, chunk bits
    const int4 *rl;               // [n_row]
    const float *rl_scale;        // [n_row] or null
    const unsigned *rl_bits;      // [n_row][nwr]: bit c of word w: chunk 32 w + c is active
    const int *n_rl;              // number of listed rows
    int nwr;                      // words per row
    // strip tiles: the strip-order row table and a bit per (chunk, entry)
    const int4 *rt;               // [n_rt]
    const float *rt_scale;        // [n_rt] or null
    const int *unit_off;          // [n_strips + 1] offsets of the strips in rt
    int n_strips;
    const unsigned *sbits;        // [n_chunks][nwk]: bit j of word w: entry 32 w + j is active in the chunk
    int nwk;                      // words per chunk
    int *unit_counter;            // next strip unit to hand out (zero before the launch)
    DevTerm tn, to;               // solved term, other term (a copy of tn when there is none)
    const int2 *fmap2;            // [32 n_chunks] {f_map of the solved term, f_map of the other} (padded)
    const int4 *chunk_info;       // [n_chunks] {., ., first other-term f_int, other-term f_int count}
    const uint8_t *active;        // [bins of the solved term]
    const int *n_active;          // nonzero: some interval still iterating
    double *acc;                  // [bins][n_ant][KG]
    int *err;                     // set to 1 when a bounded wait gives up
    unsigned long long wait_ns;   // wall-time limit of every wait
    int stall_fill;               // tests: every producer lane leaves its n-th stage unfilled (-1: none)
    // shared-memory layout (bytes)
    int depth;                    // stages per consumer ring
    int stage_bytes;              // one stage
    int off_m, off_w, off_fm, off_jp, off_jq, off_h;
};

// Per-launch preparation, row tiles: the rows with an active 32-channel chunk, compacted
// (warp-aggregated, so rows keep their order within a warp), and the bits of their chunks.
static __global__ void ws_rows_kernel(int n_row, const int4 *rt, const float *rt_scale, const uint8_t *chunk_active,
                                      int n_chunks, int nwr, const int *n_active, int4 *rl, float *rl_scale,
                                      unsigned *rl_bits, int *n_rl)
{
    if (__ldg(n_active) == 0) return;
    const int lane = threadIdx.x & 31;
    const long u = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int4 e = make_int4(0, 0, -1, 0);
    if (u < n_row) e = __ldg(rt + u);
    const uint8_t *ca = chunk_active + (size_t)max(e.z, 0) * n_chunks;
    bool live = false;
    if (e.z >= 0)
        for (int ch = 0; ch < n_chunks && !live; ++ch) live = __ldg(ca + ch) != 0;
    const unsigned m = __ballot_sync(0xffffffffu, live);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(n_rl, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!live) return;
    const int i = base + __popc(m & ((1u << lane) - 1u));
    rl[i] = e;
    if (rl_scale) rl_scale[i] = __ldg(rt_scale + u);
    for (int w = 0; w < nwr; ++w) {
        unsigned b = 0;
        for (int j = 0; j < 32; ++j) {
            const int ch = 32 * w + j;
            if (ch < n_chunks && __ldg(ca + ch)) b |= 1u << j;
        }
        rl_bits[(size_t)i * nwr + w] = b;
    }
}

// Per-launch preparation, strip tiles: bit j of word (ch, w) is set when row-table entry
// 32 w + j has usable data and an active bin in chunk ch.
static __global__ void ws_strip_bits_kernel(long n_rt, const int4 *rt, const uint8_t *chunk_active, int n_chunks,
                                            int nwk, const int *n_active, unsigned *sbits)
{
    if (__ldg(n_active) == 0) return;
    const int lane = threadIdx.x & 31;
    const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nwk) return;
    const long k = 32 * w + lane;
    const int tn = k < n_rt ? __ldg(rt + k).z : -1;
    const uint8_t *ca = chunk_active + (size_t)max(tn, 0) * n_chunks;
    for (int ch = 0; ch < n_chunks; ++ch) {
        const unsigned b = __ballot_sync(0xffffffffu, tn >= 0 && __ldg(ca + ch) != 0);
        if (lane == 0) sbits[(size_t)ch * nwk + w] = b;
    }
}

// Wait for a consumer's "full" barrier; gives up on the wall-time limit or when another
// warp has aborted the CTA.
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, unsigned long long limit,
                                        const volatile int *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 15) == 15) {
            if (abort_flag && *abort_flag) return false;
            if (global_timer_ns() - t0 > limit) return false;
        }
    }
}

// The walk over one stream of steps: by one producer lane (UNI = false), or by a whole warp
// that feeds itself (UNI = true: every lane holds the same cursor; strip units are claimed
// by lane 0 and broadcast).
template <bool UNI> struct WsCursorT {
    // the step to copy next: row-table entry, FP16 scale, chunk (have = false: none left)
    int4 e;
    float sc;
    int ch;
    bool have;
    // row tiles: list position, stride, length; the current row's remaining chunk bits
    int li, S, L, wi;
    unsigned bits;
    int4 ne;                      // the next listed row, loaded a row ahead
    float nsc;
    unsigned nbits;
    // strip tiles: the current unit's chunk, its range of entries, the bits still to scan
    int uch, k, kend;
    unsigned wb;                  // bits of the word holding entries [k & ~31, ...), below k cleared
    int nu;                       // the next unit, claimed a unit ahead (-1: none)
    int nk0, nk1;                 // its range of entries
    int kn;                       // the next active entry found ahead (-1: none), its entry loaded
    int4 en;
    float scn;

    __device__ __forceinline__ void claim(const WsArgs &a)
    {
        if constexpr (UNI) {
            int u = 0;
            if ((threadIdx.x & 31) == 0) u = atomicAdd(a.unit_counter, 1);
            nu = __shfl_sync(0xffffffffu, u, 0);
        } else {
            nu = atomicAdd(a.unit_counter, 1);
        }
        if (nu < a.n_strips * a.n_chunks) {
            const int s = nu / a.n_chunks;
            nk0 = __ldg(a.unit_off + s);
            nk1 = __ldg(a.unit_off + s + 1);
        } else {
            nu = -1;
        }
    }

    // strip tiles: the next active entry after the current position (or -1), walking units
    __device__ __forceinline__ int scan(const WsArgs &a)
    {
        for (;;) {
            if (wb) {
                const int j = __ffs(wb) - 1;
                wb &= wb - 1;
                const int kk = (k & ~31) + j;
                if (kk < kend) return kk;
                wb = 0;
            }
            const int nxt = (k & ~31) + 32;
            if (nxt < kend) {
                k = nxt;
                wb = __ldg(a.sbits + (size_t)uch * a.nwk + (k >> 5));
                continue;
            }
            // unit finished: start the one claimed ahead and claim the following one
            if (nu < 0) return -1;
            uch = nu % a.n_chunks;
            k = nk0;
            kend = nk1;
            claim(a);
            if (k >= kend) { wb = 0; k = kend; continue; }
            wb = __ldg(a.sbits + (size_t)uch * a.nwk + (k >> 5)) & (0xffffffffu << (k & 31));
        }
    }

    __device__ __forceinline__ void start(const WsArgs &a, int gl, int n_lanes)
    {
        have = false;
        if (a.order == 0) {
            S = n_lanes;
            L = __ldg(a.n_rl);
            li = gl;
            wi = 0;
            bits = 0;
            if (li < L) {
                e = __ldg(a.rl + li);
                sc = a.rl_scale ? __ldg(a.rl_scale + li) : 0.f;
                bits = __ldg(a.rl_bits + (size_t)li * a.nwr);
            }
            if (li + S < L) {
                ne = __ldg(a.rl + li + S);
                nsc = a.rl_scale ? __ldg(a.rl_scale + li + S) : 0.f;
                nbits = __ldg(a.rl_bits + (size_t)(li + S) * a.nwr);
            }
        } else {
            kend = 0;
            k = 0;
            wb = 0;
            uch = 0;
            claim(a);
            kn = scan(a);
            if (kn >= 0) {
                en = __ldg(a.rt + kn);
                scn = a.rt_scale ? __ldg(a.rt_scale + kn) : 0.f;
            }
        }
        advance(a);
    }

    // make the next step current (have = false when the stream has ended)
    __device__ __forceinline__ void advance(const WsArgs &a)
    {
        if (a.order == 0) {
            for (;;) {
                if (li >= L) { have = false; return; }
                if (bits) {
                    const int j = __ffs(bits) - 1;
                    bits &= bits - 1;
                    ch = 32 * wi + j;
                    have = true;
                    return;
                }
                if (++wi < a.nwr) {
                    bits = __ldg(a.rl_bits + (size_t)li * a.nwr + wi);
                    continue;
                }
                li += S;
                wi = 0;
                e = ne;
                sc = nsc;
                bits = nbits;
                if (li + S < L) {
                    ne = __ldg(a.rl + li + S);
                    nsc = a.rl_scale ? __ldg(a.rl_scale + li + S) : 0.f;
                    nbits = __ldg(a.rl_bits + (size_t)(li + S) * a.nwr);
                }
            }
        } else {
            if (kn < 0) { have = false; return; }
            e = en;
            sc = scn;
            ch = uch;
            have = true;
            kn = scan(a);
            if (kn >= 0) {
                en = __ldg(a.rt + kn);
                scn = a.rt_scale ? __ldg(a.rt_scale + kn) : 0.f;
            }
        }
    }
};

template <int TS, int LK, int RK, bool M16, int NC>
__global__ void __launch_bounds__((NC + 1) * 32, NC <= 7 ? 2 : 1) acc_ws_kernel(const WsArgs a)
{
    if (__ldg(a.n_active) == 0) return;
    constexpr bool HAS_L = LK != KIND_NONE;
    constexpr int GK = TS == TS_FULL ? KIND_FULL : KIND_DIAG;
    constexpr int OK_ = HAS_L ? LK : RK;                    // kind of the other term (NONE: single term)
    constexpr bool HAS_O = OK_ != KIND_NONE;
    constexpr int ESO = OK_ == KIND_FULL ? 32 : 16;         // bytes per table entry of the other term
    constexpr int MB = M16 ? 16 : 32;                       // model bytes per sample
    constexpr int FLUSH_EVERY = M16 ? 16 : (1 << 30);       // FP16 model: FP32 partial sums of <= 16 samples
    using Lay = AccLayout<TS, HAS_L>;
    constexpr int KR = Lay::KR, KG = Lay::KG;
    extern __shared__ __align__(128) unsigned char ws_smem[];
    __shared__ int s_abort;
    __shared__ int s_fills[NC];
    constexpr int MAX_SCHUNK = 256;               // chunk table kept in shared memory up to 8192 channels
    __shared__ int2 s_chunk_tab[HAS_O ? MAX_SCHUNK : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int D = a.depth, SB = a.stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(ws_smem + (size_t)NC * D * SB);   // full [NC][D], empty [NC][D]
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int i = 0; i < 2 * NC * D; ++i) mbar_init(bars + i, 1);
        fence_barrier_init();
    }
    if (threadIdx.x < NC) s_fills[threadIdx.x] = 0;
    const int2 *s_chunk = nullptr;
    if constexpr (HAS_O) {
        if (a.n_chunks <= MAX_SCHUNK) {
            for (int i = threadIdx.x; i < a.n_chunks; i += blockDim.x) {
                const int4 ci = __ldg(a.chunk_info + i);
                s_chunk_tab[i] = make_int2(ci.z, ci.w);
            }
            s_chunk = s_chunk_tab;
        }
    }
    __syncthreads();
    volatile int *abort_flag = &s_abort;
    // a consumer's ring position, kept for the drain after the main loops
    int c_s = 0, c_consumed = 0;
    uint32_t c_ph = 0;

    if (warp == 0) {
        // ------------------------------ producer ------------------------------
        const bool mine = lane < NC;
        WsCursorT<false> cur;
        if (mine) cur.start(a, blockIdx.x * NC + lane, gridDim.x * NC);
        unsigned char *ring = ws_smem + (size_t)lane * D * SB;
        uint64_t *full = bars + lane * D, *empty = bars + (NC + lane) * D;
        int s = 0, fills = 0;
        uint32_t eph = 1;             // the first pass over the ring finds every stage free
        bool ended = !mine;
        uint32_t idle = 0;
        uint64_t t_idle = 0;
        while (__any_sync(0xffffffffu, !ended)) {
            bool prog = false;
            // fill every free stage of this lane's consumer
            while (!ended && mbar_test_wait(empty + s, eph)) {
                unsigned char *st = ring + (size_t)s * SB;
                const bool stalled = fills == a.stall_fill;
                if (cur.have) {
                    const int4 e = cur.e;
                    const int c0 = cur.ch * 32;
                    const int nch = min(32, a.n_chan - c0);
                    const size_t sidx = (size_t)e.x * a.n_chan + c0;
                    int fo0 = 0, fcnt = 0;
                    if constexpr (HAS_O) {
                        const int2 ci = s_chunk ? s_chunk[cur.ch] : make_int2(__ldg(a.chunk_info + cur.ch).z,
                                                                             __ldg(a.chunk_info + cur.ch).w);
                        fo0 = ci.x;
                        fcnt = ci.y;
                    }
                    uint32_t bytes = (uint32_t)nch * (32u + MB + 16u) + 256u;
                    if constexpr (HAS_O) bytes += 2u * fcnt * ESO;
                    *reinterpret_cast<int4 *>(st + a.off_h) = make_int4(e.y, e.z, e.w, c0);
                    *reinterpret_cast<int4 *>(st + a.off_h + 16) = make_int4(__float_as_int(cur.sc), fo0, 0, 0);
                    if (!stalled) {
                        mbar_arrive_expect_tx(full + s, bytes);
                        bulk_copy_g2s(st, a.vis + 2 * sidx, nch * 32u, full + s);
                        if constexpr (M16) bulk_copy_g2s(st + a.off_m, a.model16 + sidx, nch * 16u, full + s);
                        else bulk_copy_g2s(st + a.off_m, a.model + 2 * sidx, nch * 32u, full + s);
                        bulk_copy_g2s(st + a.off_w, a.wf + sidx, nch * 16u, full + s);
                        bulk_copy_g2s(st + a.off_fm, a.fmap2 + c0, 256u, full + s);
                        if constexpr (HAS_O) {
                            const int p = e.y & 0xffff, q = e.y >> 16;
                            const unsigned char *tb = reinterpret_cast<const unsigned char *>(a.to.tab);
                            const size_t rp = ((size_t)e.w * a.n_ant + p) * a.to.n_fint + fo0;
                            const size_t rq = ((size_t)e.w * a.n_ant + q) * a.to.n_fint + fo0;
                            bulk_copy_g2s(st + a.off_jp, tb + rp * ESO, fcnt * ESO, full + s);
                            bulk_copy_g2s(st + a.off_jq, tb + rq * ESO, fcnt * ESO, full + s);
                        }
                    }
                    cur.advance(a);
                } else {
                    *reinterpret_cast<int4 *>(st + a.off_h) = make_int4(0, STREAM_END, 0, 0);
                    if (!stalled) mbar_arrive(full + s);
                    ended = true;
                }
                ++fills;
                if (++s == D) { s = 0; eph ^= 1u; }
                prog = true;
            }
            if (__any_sync(0xffffffffu, prog)) {
                idle = 0;
            } else {
                // nothing to fill: back off; every 256 idle trips, check the abort flag and the
                // wall-time limit (a consumer that frees no stage for that long has failed)
                if (*abort_flag) break;
                if ((idle & 255) == 0) {
                    const uint64_t now = global_timer_ns();
                    if (idle == 0) t_idle = now;
                    else if (now - t_idle > a.wait_ns) {
                        if (!ended) atomicExch(a.err, 1);
                        *abort_flag = 1;
                        break;
                    }
                }
                ++idle;
                __nanosleep(32);
            }
        }
        if (mine) s_fills[lane] = fills;
    } else {
        // ------------------------------ consumer ------------------------------
        const int c = warp - 1;
        const unsigned char *ring = ws_smem + (size_t)c * D * SB;
        uint64_t *full = bars + c * D, *empty = bars + (NC + c) * D;
        const int n_chan = a.n_chan, n_ant = a.n_ant;
        Acc<KR, false> Ap, Aq;
        Ap.zero();
        Aq.zero();
        int s = 0, consumed = 0, cur_key = -1, cur_pq = -1;
        uint32_t ph = 0;
        int ci_p = -1, ci_q = -1, act_key = -1, since_flush = 0;
        bool act_val = false, failed = false;
        J2 cGp = j_identity(), cGq = j_identity();
        for (;;) {
            if (!ws_wait(full + s, ph, a.wait_ns, abort_flag)) {
                failed = true;
                break;
            }
            const unsigned char *st = ring + (size_t)s * SB;
            const int4 h = *reinterpret_cast<const int4 *>(st + a.off_h);
            ++consumed;
            if (h.y == STREAM_END) break;
            const int p = h.x & 0xffff, q = h.x >> 16;
            const int cc = h.w + lane;
            const bool in = cc < n_chan;
            const int2 fm = in ? reinterpret_cast<const int2 *>(st + a.off_fm)[lane] : make_int2(0, 0);
            // the solved term's entries stay in registers while the lane's table index is unchanged
            {
                const int ip = in ? (h.y * n_ant + p) * a.tn.n_fint + fm.x : ci_p;
                const int iq = in ? (h.y * n_ant + q) * a.tn.n_fint + fm.x : ci_q;
                if (__any_sync(0xffffffffu, ip != ci_p || iq != ci_q)) {
                    if (ip != ci_p) { cGp = fetch_k<GK>(a.tn, n_ant, h.y, fm.x, p); ci_p = ip; }
                    if (iq != ci_q) { cGq = fetch_k<GK>(a.tn, n_ant, h.y, fm.x, q); ci_q = iq; }
                }
            }
            const int key = in ? h.y * a.tn.n_fint + fm.x : -1;
            {
                bool change = h.x != cur_pq || key != cur_key;
                if constexpr (M16) change = change || since_flush >= FLUSH_EVERY;
                if constexpr (M16) ++since_flush;
                if (__any_sync(0xffffffffu, change && cur_key >= 0)) {
                    if constexpr (M16) since_flush = 1;
                    flush_pair<KR, KG, Lay>(Ap, Aq, cur_key, cur_pq, lane, a.active, a.acc, n_ant);
                }
                cur_key = key;
                cur_pq = h.x;
            }
            const float4 w = reinterpret_cast<const float4 *>(st + a.off_w)[lane];
            bool ok = in && (w.x != 0.f || w.y != 0.f || w.z != 0.f || w.w != 0.f);
            if (ok && key != act_key) {          // activity of the lane's bin, read when the bin changes
                act_key = key;
                act_val = __ldg(a.active + key) != 0;
            }
            ok = ok && act_val;
            if (ok) {
                const float4 *sd = reinterpret_cast<const float4 *>(st) + 2 * lane;
                const J2 Dm = j_from(sd[0], sd[1]);
                J2 M;
                if constexpr (M16) {
                    const float sc = __int_as_float(reinterpret_cast<const int4 *>(st + a.off_h)[1].x);
                    M = load_model16(reinterpret_cast<const uint4 *>(st + a.off_m)[lane], sc);
                } else {
                    const float4 *sm = reinterpret_cast<const float4 *>(st + a.off_m) + 2 * lane;
                    M = j_from(sm[0], sm[1]);
                }
                J2 Op, Oq;
                if constexpr (HAS_O) {
                    const int j = fm.y - reinterpret_cast<const int4 *>(st + a.off_h)[1].y;
                    Op = smem_jones<OK_>(st + a.off_jp, j);
                    Oq = smem_jones<OK_>(st + a.off_jq, j);
                } else {
                    Op = j_identity();
                    Oq = Op;
                }
                sample_math<TS, LK, RK, false>(Op, cGp, Op, Oq, cGq, Oq, Dm, M, w, Ap, Aq);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + s);
            if (++s == D) { s = 0; ph ^= 1u; }
        }
        if (__any_sync(0xffffffffu, cur_key >= 0)) flush_pair<KR, KG, Lay>(Ap, Aq, cur_key, cur_pq, lane, a.active, a.acc, n_ant);
        if (failed && lane == 0) {
            atomicExch(a.err, 1);
            *abort_flag = 1;
        }
        c_s = s;
        c_ph = ph;
        c_consumed = consumed;
    }
    __syncthreads();
    if (warp > 0 && *abort_flag) {
        // a wait gave up somewhere in the CTA: wait (bounded) for the copies still in flight
        // into this warp's ring before the CTA's shared memory is released
        const int c = warp - 1;
        uint64_t *full = bars + c * D;
        for (int k = c_consumed; k < s_fills[c]; ++k) {
            ws_wait(full + c_s, c_ph, a.wait_ns, nullptr);
            if (++c_s == D) { c_s = 0; c_ph ^= 1u; }
        }
    }
}


// ---------------------------------------------------------------------------
// self-feeding variant: every warp moves its own data
// ---------------------------------------------------------------------------
//
// Each warp walks its own stream of steps (the tile order is a template parameter) and,
// D - 1 steps ahead of the step it computes, refills the ring stage it has just finished
// with: lane 0 writes the step's header and arms the stage's "full" barrier with the
// transaction count, then lanes 0..5 each issue one cp.async.bulk (d, m, folded weights,
// channel maps, the other term's entries for p and q).  The copy engine moves the data.
//
// Steps come in runs along which the antenna pair, every lane's interval bin and hence the
// solved term's entries and the bins' activity do not change: a row (row tiles, when the
// solved term has one frequency interval), or consecutive rows of a strip unit in one time
// interval (strip tiles).  The cursor marks the first step of each run in its header; only
// there does the warp flush its register sums and refresh the bins, the solved term's
// entries and the activity.  Every other step is: wait for the stage, read it from shared
// memory, accumulate, refill.  There is no cross-warp hand-off; every wait is bounded in
// time (a wait that gives up sets *err, the warp waits (bounded) for its copies in flight
// and leaves).

constexpr int RUN_NEW = 1 << 30;   // header flag: the step starts a run

// The walk over one warp's steps in tile order ORDER (every lane holds the same state).
template <int ORDER> struct RunCursor;

// row tiles: the listed rows (grid stride over the list) and their active chunks
template <> struct RunCursor<0> {
    int li, S, L, wi;
    unsigned bits;
    int4 e, ne;
    float sc, nsc;
    unsigned nbits;
    int ch;
    bool have, newrun;

    __device__ __forceinline__ void load_next(const WsArgs &a)
    {
        if (li + S < L) {
            ne = __ldg(a.rl + li + S);
            nsc = a.rl_scale ? __ldg(a.rl_scale + li + S) : 0.f;
            nbits = __ldg(a.rl_bits + (size_t)(li + S) * a.nwr);
        }
    }
    __device__ __forceinline__ void start(const WsArgs &a, int gw, int n_warps)
    {
        S = n_warps;
        L = __ldg(a.n_rl);
        li = gw;
        wi = 0;
        bits = 0;
        have = false;
        if (li < L) {
            e = __ldg(a.rl + li);
            sc = a.rl_scale ? __ldg(a.rl_scale + li) : 0.f;
            bits = __ldg(a.rl_bits + (size_t)li * a.nwr);
        }
        load_next(a);
        newrun = true;
        find(a);
    }
    // the next active chunk, moving to the next listed row when this one is done
    __device__ __forceinline__ void find(const WsArgs &a)
    {
        for (;;) {
            if (li >= L) { have = false; return; }
            if (bits) {
                ch = 32 * wi + __ffs(bits) - 1;
                bits &= bits - 1;
                have = true;
                return;
            }
            if (++wi < a.nwr) {
                bits = __ldg(a.rl_bits + (size_t)li * a.nwr + wi);
                continue;
            }
            li += S;
            wi = 0;
            e = ne;
            sc = nsc;
            bits = nbits;
            newrun = true;
            load_next(a);
        }
    }
    // the solved term's bins change along a row only when it has several frequency intervals
    __device__ __forceinline__ void advance(const WsArgs &a, bool fine_bins)
    {
        newrun = fine_bins;
        find(a);
    }
};

// strip tiles: units (strip x 32-channel chunk) from the launch's counter, and their active entries
template <> struct RunCursor<1> {
    int uch, k, kend;
    unsigned wb;
    int nu, nk0, nk1;
    int kn, kn_ch;                // the next active entry found ahead (-1: none) and its unit's chunk
    bool kn_new;                  //   ... which is the first active entry of its unit
    int4 en;
    float scn;
    int4 e;
    float sc;
    int ch;
    bool have, newrun;

    __device__ __forceinline__ void claim(const WsArgs &a)
    {
        int u = 0;
        if ((threadIdx.x & 31) == 0) u = atomicAdd(a.unit_counter, 1);
        nu = __shfl_sync(0xffffffffu, u, 0);
        if (nu < a.n_strips * a.n_chunks) {
            const int s_ = nu / a.n_chunks;
            nk0 = __ldg(a.unit_off + s_);
            nk1 = __ldg(a.unit_off + s_ + 1);
        } else {
            nu = -1;
        }
    }
    // the next active entry after the current position (-1: none), walking units
    __device__ __forceinline__ int scan(const WsArgs &a, bool &fresh)
    {
        for (;;) {
            if (wb) {
                const int j = __ffs(wb) - 1;
                wb &= wb - 1;
                const int kk = (k & ~31) + j;
                if (kk < kend) return kk;
                wb = 0;
            }
            const int nxt = (k & ~31) + 32;
            if (nxt < kend) {
                k = nxt;
                wb = __ldg(a.sbits + (size_t)uch * a.nwk + (k >> 5));
                continue;
            }
            if (nu < 0) return -1;
            uch = nu % a.n_chunks;
            k = nk0;
            kend = nk1;
            fresh = true;
            claim(a);
            if (k >= kend) { wb = 0; k = kend; continue; }
            wb = __ldg(a.sbits + (size_t)uch * a.nwk + (k >> 5)) & (0xffffffffu << (k & 31));
        }
    }
    __device__ __forceinline__ void look_ahead(const WsArgs &a)
    {
        bool fresh = false;
        kn = scan(a, fresh);
        kn_new = fresh;
        kn_ch = uch;
        if (kn >= 0) {
            en = __ldg(a.rt + kn);
            scn = a.rt_scale ? __ldg(a.rt_scale + kn) : 0.f;
        }
    }
    __device__ __forceinline__ void start(const WsArgs &a, int, int)
    {
        kend = 0;
        k = 0;
        wb = 0;
        uch = 0;
        have = false;
        claim(a);
        look_ahead(a);
        e = make_int4(0, 0, -1, 0);
        advance(a, false);
    }
    __device__ __forceinline__ void advance(const WsArgs &a, bool)
    {
        if (kn < 0) { have = false; return; }
        newrun = kn_new || en.z != e.z;
        e = en;
        sc = scn;
        ch = kn_ch;
        have = true;
        look_ahead(a);
    }
};

template <int TS, int LK, int RK, bool M16, int ORDER, int NW>
__global__ void __launch_bounds__(NW * 32, 2) acc_run_kernel(const WsArgs a)
{
    if (__ldg(a.n_active) == 0) return;
    constexpr bool HAS_L = LK != KIND_NONE;
    constexpr int GK = TS == TS_FULL ? KIND_FULL : KIND_DIAG;
    constexpr int OK_ = HAS_L ? LK : RK;
    constexpr bool HAS_O = OK_ != KIND_NONE;
    constexpr int ESO = OK_ == KIND_FULL ? 32 : 16;
    constexpr int MB = M16 ? 16 : 32;
    constexpr int FLUSH_EVERY = M16 ? 16 : (1 << 30);
    using Lay = AccLayout<TS, HAS_L>;
    constexpr int KR = Lay::KR, KG = Lay::KG;
    extern __shared__ __align__(128) unsigned char ws_smem[];
    constexpr int MAX_SCHUNK = 256;
    __shared__ int2 s_chunk_tab[HAS_O ? MAX_SCHUNK : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int D = a.depth, SB = a.stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(ws_smem + (size_t)NW * D * SB);   // full [NW][D]
    if (threadIdx.x == 0) {
        for (int i = 0; i < NW * D; ++i) mbar_init(bars + i, 1);
        fence_barrier_init();
    }
    const int2 *s_chunk = nullptr;
    if constexpr (HAS_O) {
        if (a.n_chunks <= MAX_SCHUNK) {
            for (int i = threadIdx.x; i < a.n_chunks; i += blockDim.x) {
                const int4 ci = __ldg(a.chunk_info + i);
                s_chunk_tab[i] = make_int2(ci.z, ci.w);
            }
            s_chunk = s_chunk_tab;
        }
    }
    __syncthreads();
    unsigned char *ring = ws_smem + (size_t)warp * D * SB;
    uint64_t *full = bars + warp * D;
    const int n_chan = a.n_chan, n_ant = a.n_ant;
    const bool fine_bins = ORDER == 0 && a.tn.n_fint > 1;

    // this lane's copy of every step: 0 d, 1 m, 2 folded weights, 3 channel maps, 4 / 5 the
    // other term's entries at p / q (lanes >= 6, and 4 / 5 without another term: none)
    const unsigned char *cbase = nullptr;
    uint32_t coff = 0, cesz = 0;
    switch (lane) {
    case 0: cbase = reinterpret_cast<const unsigned char *>(a.vis); coff = 0; cesz = 32; break;
    case 1: cbase = M16 ? reinterpret_cast<const unsigned char *>(a.model16) : reinterpret_cast<const unsigned char *>(a.model);
            coff = a.off_m; cesz = MB; break;
    case 2: cbase = reinterpret_cast<const unsigned char *>(a.wf); coff = a.off_w; cesz = 16; break;
    case 3: cbase = reinterpret_cast<const unsigned char *>(a.fmap2); coff = a.off_fm; cesz = 8; break;
    case 4: cbase = HAS_O ? reinterpret_cast<const unsigned char *>(a.to.tab) : nullptr; coff = a.off_jp; cesz = ESO; break;
    case 5: cbase = HAS_O ? reinterpret_cast<const unsigned char *>(a.to.tab) : nullptr; coff = a.off_jq; cesz = ESO; break;
    default: break;
    }

    RunCursor<ORDER> cur;
    cur.start(a, blockIdx.x * NW + warp, gridDim.x * NW);
    int fills = 0;
    bool fed_end = false;
    auto fill = [&](int fs) {
        unsigned char *st = ring + (size_t)fs * SB;
        uint64_t *bar = full + fs;
        const bool stalled = fills == a.stall_fill;
        if (cur.have) {
            const int4 e = cur.e;
            const int c0 = cur.ch * 32;
            const int nch = min(32, n_chan - c0);
            int fo0 = 0, fcnt = 0;
            if constexpr (HAS_O) {
                const int2 ci = s_chunk ? s_chunk[cur.ch] : make_int2(__ldg(a.chunk_info + cur.ch).z,
                                                                     __ldg(a.chunk_info + cur.ch).w);
                fo0 = ci.x;
                fcnt = ci.y;
            }
            if (lane == 0) {
                uint32_t bytes = (uint32_t)nch * (32u + MB + 16u) + 256u;
                if constexpr (HAS_O) bytes += 2u * fcnt * ESO;
                *reinterpret_cast<int4 *>(st + a.off_h) = make_int4(e.y, e.z | (cur.newrun ? RUN_NEW : 0), e.w, c0);
                *reinterpret_cast<int4 *>(st + a.off_h + 16) = make_int4(__float_as_int(cur.sc), fo0, 0, 0);
                if (!stalled) mbar_arrive_expect_tx(bar, bytes);
            }
            __syncwarp();
            // element index and count of this lane's copy
            const size_t sidx = (size_t)e.x * n_chan + c0;
            const int ant = lane == 4 ? (e.y & 0xffff) : (e.y >> 16);
            const size_t oidx = ((size_t)e.w * n_ant + ant) * a.to.n_fint + fo0;
            const size_t idx = lane < 3 ? sidx : (lane == 3 ? (size_t)c0 : oidx);
            const uint32_t cnt = lane < 3 ? (uint32_t)nch : (lane == 3 ? 32u : (uint32_t)fcnt);
            if (cbase && !stalled) bulk_copy_g2s(st + coff, cbase + idx * cesz, cnt * cesz, bar);
            cur.advance(a, fine_bins);
        } else {
            if (lane == 0) {
                *reinterpret_cast<int4 *>(st + a.off_h) = make_int4(0, STREAM_END, 0, 0);
                if (!stalled) mbar_arrive(bar);
            }
            fed_end = true;
        }
        ++fills;
    };
    for (int j = 0; j < D - 1 && !fed_end; ++j) fill(j);

    Acc<KR, false> Ap, Aq;
    Ap.zero();
    Aq.zero();
    int s = 0, consumed = 0, cur_key = -1, cur_pq = -1, since_flush = 0;
    uint32_t ph = 0;
    bool in = false, act = false, failed = false;
    int2 fm = make_int2(0, 0);
    J2 cGp = j_identity(), cGq = j_identity();
    for (;;) {
        if (!fed_end) {
            // refill the stage this warp finished with in the previous step (its reads are
            // ordered before the copy engine's writes)
            int fs = s + D - 1;
            if (fs >= D) fs -= D;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fill(fs);
        }
        if (!ws_wait(full + s, ph, a.wait_ns, nullptr)) {
            failed = true;
            break;
        }
        const unsigned char *st = ring + (size_t)s * SB;
        const int4 h = *reinterpret_cast<const int4 *>(st + a.off_h);
        ++consumed;
        if (h.y == STREAM_END) break;
        if (ORDER == 0) {
            // row tiles: the channel maps change every step
            in = h.w + lane < n_chan;
            fm = in ? reinterpret_cast<const int2 *>(st + a.off_fm)[lane] : make_int2(0, 0);
        }
        if (h.y & RUN_NEW) {
            // a new run: flush, then this run's antennas, bins, solved-term entries and activity
            const int tn = h.y & ~RUN_NEW;
            const int p = h.x & 0xffff, q = h.x >> 16;
            if (ORDER == 1) {
                in = h.w + lane < n_chan;
                fm = in ? reinterpret_cast<const int2 *>(st + a.off_fm)[lane] : make_int2(0, 0);
            }
            const int key = in ? tn * a.tn.n_fint + fm.x : -1;
            if (__any_sync(0xffffffffu, (h.x != cur_pq || key != cur_key) && cur_key >= 0)) {
                flush_pair<KR, KG, Lay>(Ap, Aq, cur_key, cur_pq, lane, a.active, a.acc, n_ant);
                since_flush = 0;
            }
            cur_key = key;
            cur_pq = h.x;
            if (in) {
                cGp = fetch_k<GK>(a.tn, n_ant, tn, fm.x, p);
                cGq = fetch_k<GK>(a.tn, n_ant, tn, fm.x, q);
            }
            act = in && __ldg(a.active + key) != 0;
        }
        if constexpr (M16) {
            // FP16 model: FP32 partial sums of at most FLUSH_EVERY samples per lane
            if (++since_flush > FLUSH_EVERY) {
                flush_pair<KR, KG, Lay>(Ap, Aq, cur_key, cur_pq, lane, a.active, a.acc, n_ant);
                since_flush = 1;
            }
        }
        const float4 w = reinterpret_cast<const float4 *>(st + a.off_w)[lane];
        const bool ok = in && act && (w.x != 0.f || w.y != 0.f || w.z != 0.f || w.w != 0.f);
        if (ok) {
            const float4 *sd = reinterpret_cast<const float4 *>(st) + 2 * lane;
            const J2 Dm = j_from(sd[0], sd[1]);
            J2 M;
            if constexpr (M16) {
                const float sc = __int_as_float(reinterpret_cast<const int4 *>(st + a.off_h)[1].x);
                M = load_model16(reinterpret_cast<const uint4 *>(st + a.off_m)[lane], sc);
            } else {
                const float4 *sm = reinterpret_cast<const float4 *>(st + a.off_m) + 2 * lane;
                M = j_from(sm[0], sm[1]);
            }
            J2 Op, Oq;
            if constexpr (HAS_O) {
                const int j = fm.y - reinterpret_cast<const int4 *>(st + a.off_h)[1].y;
                Op = smem_jones<OK_>(st + a.off_jp, j);
                Oq = smem_jones<OK_>(st + a.off_jq, j);
            } else {
                Op = j_identity();
                Oq = Op;
            }
            sample_math<TS, LK, RK, false>(Op, cGp, Op, Oq, cGq, Oq, Dm, M, w, Ap, Aq);
        }
        __syncwarp();
        if (++s == D) { s = 0; ph ^= 1u; }
    }
    if (__any_sync(0xffffffffu, cur_key >= 0)) flush_pair<KR, KG, Lay>(Ap, Aq, cur_key, cur_pq, lane, a.active, a.acc, n_ant);
    if (failed) {
        if (lane == 0) atomicExch(a.err, 1);
        // wait (bounded) for this warp's copies still in flight before it leaves
        for (int k = consumed; k < fills; ++k) {
            ws_wait(full + s, ph, a.wait_ns, nullptr);
            if (++s == D) { s = 0; ph ^= 1u; }
        }
    }
}

} // namespace qc
