// qc_batch.cu -- persistent batched solver: thousands of independent solution
// intervals (diagonal gains, one interval each) solved in one kernel launch.
//
// Each CTA takes whole problems (longest first from a shared work counter, or
// a static schedule) and runs Algorithm 1 of arxiv 2412.10072 (Section 4.3)
// on chip: per iteration one pass over the problem's samples forms the
// residual r = D - G_p M G_q^H and accumulates the per-antenna diagonal JHJ and
// JHr blocks (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified, including the
// conjugate baselines) in shared memory, then one thread per antenna solves its
// block in FP64 and updates its gain (Eq. update); the FP64 relative gain change
// of the problem decides convergence.  No grid-wide synchronisation and no
// spin-waits: the only shared state is an atomic work counter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/qc.h"
#include "qc_async.cuh"

cudaError_t qc_dev_malloc(void **p, size_t bytes);   // counted allocation (qc_api.cu)
void qc_dev_free(void *p);
#include "qc_jones.cuh"

namespace {

using namespace qc;

thread_local std::string g_batch_create_error;

struct BProb {
    long long vis_off, row_off;
    int n_rows, n_chan, n_ant, gain_off;
    long long n_unflag;          // unflagged samples (algorithmic bytes)
};

struct BatchArgs {
    const BProb *probs;
    int n_prob;
    const int *order;            // schedule order [n_prob]
    int *queue;                  // work counter (LPT)
    int schedule;                // QC_SCHED_LPT / QC_SCHED_STATIC
    const float4 *vis, *model;
    const uint4 *model16;
    const float *row_scale;      // per-row model scale (FP16 model): the scale of the row's baseline
    const float4 *weight;
    const uint8_t *flag;
    const int2 *ants;            // [rows] (p, q), local antenna indices
    float2 *gains;               // [sum n_ant][2]
    int8_t *gain_flags;          // [sum n_ant] or null
    int *iters;                  // [n_prob] or null
    int max_iter, damping_mode;
    double damping, tol;
    int max_ant;
    unsigned long long *vis_iters, *bytes;
    const float2 *fb_gains;      // [sum n_ant][2] fallback start, or null
    const double *fb_chi2;       // [n_prob] chi^2 at the fallback gains (with fb_gains)
    unsigned long long *n_fallback;
};

// Sum v over the run of equal keys that contains this lane; the run's first lane gets it.
__device__ __forceinline__ float run_sum(float v, int lane, unsigned run_end)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float o = __shfl_down_sync(0xffffffffu, v, d);
        if (lane + d < (int)run_end) v += o;
    }
    return v;
}

// Segmented flush of one side's register sums: lanes with equal consecutive keys
// are summed by shuffles and the head of each run adds the six sums into the
// problem's shared accumulators.  key < 0: nothing to add.
__device__ __forceinline__ void flush_runs(float (&s)[6], int key, int lane, float *acc)
{
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || key != prev;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned after = heads & ~((2u << lane) - 1u);
    const unsigned run_end = after ? (unsigned)(__ffs(after) - 1) : 32u;
    if (heads == 1u) {
        // one run over the whole warp: transposed reduction (each halving step
        // exchanges half of the remaining values), 9 shuffles for the 6 sums;
        // lane l ends with the total of value (l>>4&1)*4 + (l>>3&1)*2 + (l>>2&1)
        const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
        float t4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float lo = s[i], hi = i + 4 < 6 ? s[i + 4] : 0.f;
            t4[i] = (h16 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h16 ? lo : hi, 16);
        }
        float t2[2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
            t2[i] = (h8 ? t4[i + 2] : t4[i]) + __shfl_xor_sync(0xffffffffu, h8 ? t4[i] : t4[i + 2], 8);
        float t1 = (h4 ? t2[1] : t2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? t2[0] : t2[1], 4);
        t1 += __shfl_xor_sync(0xffffffffu, t1, 2);
        t1 += __shfl_xor_sync(0xffffffffu, t1, 1);
        const int idx = (h16 ? 4 : 0) + (h8 ? 2 : 0) + (h4 ? 1 : 0);
        if ((lane & 3) == 0 && idx < 6 && key >= 0) atomicAdd(acc + key * 6 + idx, t1);
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float sum = run_sum(s[i], lane, run_end);
            if (head && key >= 0) atomicAdd(acc + key * 6 + i, sum);
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = 0.f;
}

// Shared-memory layout of batch_kernel: per warp a ring of DEPTH stages, each
// stage V4 words x 32 lanes of 16 bytes (d: 2 words, m: 2 words or 1 FP16 word,
// w: 1 word) and 32 packed keys; then the per-antenna state.
template <bool M16> struct BatchRing { static constexpr int V4 = M16 ? 4 : 5; };

template <bool M16, int DEPTH>
__host__ __device__ constexpr size_t batch_ring_bytes_per_warp()
{
    return (size_t)DEPTH * 32 * (BatchRing<M16>::V4 * 16 + 8);
}

// Streams warp `warp`'s contiguous share of a problem's samples, 32 per step (sample
// index s = row * n_chan + chan, so each 16-byte word of a step is one contiguous
// 512-byte span whatever n_chan is), through its ring of DEPTH cp.async stages, and
// calls f(slot, key, scale_bits) once per step with the lane's sample in shared
// memory: d in slot[0], slot[32]; m in slot[64] (and slot[96]); w in slot[96 or 128].
// A lane with nothing to read (flagged sample, autocorrelation) sees zeros; key is
// p | q << 16 of the sample's row, -1 past the end of the problem.  The antennas and
// flags of a step are loaded three steps before its copies are issued (flags stream
// from DRAM, and one step is about as long as a DRAM round trip under load).
template <bool M16, int DEPTH, typename F>
__device__ __forceinline__ void stream_pass(const BatchArgs &a, const BProb &P, float4 *ring, int2 *meta, int lane,
                                            int warp, int n_warps, F &&f)
{
    constexpr int V4 = BatchRing<M16>::V4;
    const int nc = P.n_chan;
    const long n_samp = (long)P.n_rows * nc;
    const long n_steps = (n_samp + 31) >> 5;
    const long per_warp = (n_steps + n_warps - 1) / n_warps;
    const long st_begin = (long)warp * per_warp, st_end = st_begin + per_warp < n_steps ? st_begin + per_warp : n_steps;
    const int q32 = 32 / nc, r32 = 32 % nc;              // advance of (row, chan) per step
    const float4 *vis = a.vis + 2 * P.vis_off;
    const float4 *mod = M16 ? nullptr : a.model + 2 * P.vis_off;
    const uint4 *mod16 = M16 ? a.model16 + P.vis_off : nullptr;
    const float4 *wgt = a.weight + P.vis_off;
    const uint8_t *flg = a.flag ? a.flag + P.vis_off : nullptr;
    const int2 *ants = a.ants + P.row_off;
    const float *rsc = M16 ? a.row_scale + P.row_off : nullptr;
    // issue cursor: the step whose copies are issued next
    long is = st_begin;
    int r2, c2;                     // the lane's (row, chan) in step is + 2
    {
        const long s0 = st_begin * 32 + lane;
        r2 = (int)(s0 / nc);
        c2 = (int)(s0 - (long)r2 * nc);
    }
    // loads only: what depends on the loaded values is computed when the step is issued,
    // so that no instruction waits on them before then
    auto load_meta = [&](long step, int row, int2 &pq, int &fl, float &sc) {
        const long s = step * 32 + lane;
        const bool in = step < st_end && s < n_samp;
        pq = make_int2(-1, -1);     // past the end: p == q, nothing to read
        fl = 0;
        sc = 0.f;
        if (in) {
            pq = __ldg(ants + row);
            if (flg) fl = __ldg(flg + s);
            if (M16) sc = __ldg(rsc + row);
        }
    };
    auto advance = [&](int &row, int &c) {
        c += r32;
        row += q32;
        if (c >= nc) { c -= nc; ++row; }
    };
    int2 m1pq, m2pq, m3pq;
    int m1fl, m2fl, m3fl;           // the step's flag byte (nonzero: flagged)
    float m1sc, m2sc, m3sc;
    load_meta(is, r2, m1pq, m1fl, m1sc);
    advance(r2, c2);
    load_meta(is + 1, r2, m2pq, m2fl, m2sc);
    advance(r2, c2);
    load_meta(is + 2, r2, m3pq, m3fl, m3sc);
    int stage_i = 0;
    auto issue = [&]() {
        const long s = is * 32 + lane;
        const bool use = m1pq.x != m1pq.y && m1fl == 0;     // cross-correlation, unflagged
        const uint32_t nb = use ? 16u : 0u;
        const long so = use ? s : 0;
        float4 *slot = ring + (size_t)stage_i * V4 * 32 + lane;
        cp_async16(slot, vis + 2 * so, nb);
        cp_async16(slot + 32, vis + 2 * so + 1, nb);
        if constexpr (M16) {
            cp_async16(slot + 64, mod16 + so, nb);
            cp_async16(slot + 96, wgt + so, nb);
        } else {
            cp_async16(slot + 64, mod + 2 * so, nb);
            cp_async16(slot + 96, mod + 2 * so + 1, nb);
            cp_async16(slot + 128, wgt + so, nb);
        }
        cp_async_commit();
        int2 key;
        key.x = m1pq.x >= 0 ? (m1pq.x | (m1pq.y << 16)) : -1;
        key.y = __float_as_int(m1sc);
        meta[stage_i * 32 + lane] = key;
        if (++stage_i == DEPTH) stage_i = 0;
        // shift the metadata pipeline by one step
        ++is;
        m1pq = m2pq;
        m1fl = m2fl;
        m1sc = m2sc;
        m2pq = m3pq;
        m2fl = m3fl;
        m2sc = m3sc;
        advance(r2, c2);
        load_meta(is + 2, r2, m3pq, m3fl, m3sc);
    };
#pragma unroll
    for (int d = 0; d < DEPTH - 1; ++d) issue();
    int stage_c = 0;
    for (long t = st_begin; t < st_end; ++t) {
        cp_async_wait<DEPTH - 2>();
        const int2 key = meta[stage_c * 32 + lane];
        // refill the stage consumed last step before this step's arithmetic, so that
        // DEPTH - 1 stages are in flight while it runs
        issue();
        f(ring + (size_t)stage_c * V4 * 32 + lane, key.x, key.y);
        if (++stage_c == DEPTH) stage_c = 0;
    }
    cp_async_wait<0>();
}

__device__ __forceinline__ J2 ring_model16(const float4 *slot, int scale_bits)
{
    const float4 hw = slot[64];
    const uint4 h = *reinterpret_cast<const uint4 *>(&hw);
    const float sc = __int_as_float(scale_bits);
    J2 M;
    M.a = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.x)), sc);
    M.b = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.y)), sc);
    M.c = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.z)), sc);
    M.d = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.w)), sc);
    return M;
}

// One warp step covers 32 consecutive samples of the problem (sample index
// s = row * n_chan + chan, so each 16-byte word of a step is one contiguous
// 512-byte span whatever n_chan is).  Warps own contiguous ranges of steps.
template <bool M16, int DEPTH>
__global__ void __launch_bounds__(512) batch_kernel(const BatchArgs a)
{
    constexpr int V4 = BatchRing<M16>::V4;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n_warps = blockDim.x >> 5;
    float4 *ring = reinterpret_cast<float4 *>(smem) + (size_t)warp * DEPTH * V4 * 32;    // [DEPTH][V4][32]
    int2 *meta = reinterpret_cast<int2 *>(reinterpret_cast<float4 *>(smem) + (size_t)n_warps * DEPTH * V4 * 32) +
                 (size_t)warp * DEPTH * 32;                                                  // [DEPTH][32]
    unsigned char *tail = smem + (size_t)n_warps * batch_ring_bytes_per_warp<M16, DEPTH>();
    double2 *g64 = reinterpret_cast<double2 *>(tail);                         // [max_ant][2]
    float4 *g32 = reinterpret_cast<float4 *>(g64 + a.max_ant * 2);            // [max_ant] (g_XX, g_YY)
    float *acc = reinterpret_cast<float *>(g32 + a.max_ant);                  // [max_ant][6]
    __shared__ double red[2][32];
    __shared__ double s_chi;
    __shared__ int s_prob, s_done;
    int static_k = 0;

    for (;;) {
        if (tid == 0) {
            int idx;
            if (a.schedule == QC_SCHED_STATIC) idx = blockIdx.x + (static_k++) * gridDim.x;
            else idx = atomicAdd(a.queue, 1);
            s_prob = idx < a.n_prob ? a.order[idx] : -1;
        }
        __syncthreads();
        const int pi = s_prob;
        if (pi < 0) break;
        const BProb P = a.probs[pi];
        const int na = P.n_ant, nc = P.n_chan;
        for (int i = tid; i < na; i += blockDim.x) {
            const float2 g0 = a.gains[(size_t)(P.gain_off + i) * 2], g1 = a.gains[(size_t)(P.gain_off + i) * 2 + 1];
            g32[i] = make_float4(g0.x, g0.y, g1.x, g1.y);
            g64[2 * i] = make_double2(g0.x, g0.y);
            g64[2 * i + 1] = make_double2(g1.x, g1.y);
        }
        const long n_samp = (long)P.n_rows * nc;
        int k;
        bool fell_back = false;
        const bool check = a.fb_gains != nullptr;
        for (k = 1; k <= a.max_iter; ++k) {
            for (int i = tid; i < na * 6; i += blockDim.x) acc[i] = 0.f;
            if (tid == 0) s_chi = 0.0;
            __syncthreads();
            // the first pass also sums chi^2 at the starting gains (fallback check)
            const bool want_chi = check && k == 1 && !fell_back;
            float chi = 0.f;
            float sp[6], sq[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) sp[i] = sq[i] = 0.f;
            int kp = -1, kq = -1;
            stream_pass<M16, DEPTH>(a, P, ring, meta, lane, warp, n_warps, [&](const float4 *slot, int kx, int ky) {
                const int np = kx >= 0 ? (kx & 0xffff) : -1;
                const int nq = kx >= 0 ? (kx >> 16) : -1;
                if (__any_sync(0xffffffffu, np != kp)) { flush_runs(sp, kp, lane, acc); kp = np; }
                if (__any_sync(0xffffffffu, nq != kq)) { flush_runs(sq, kq, lane, acc); kq = nq; }
                if (kx >= 0) {
                    const J2 D = j_from(slot[0], slot[32]);
                    J2 M;
                    if constexpr (M16) M = ring_model16(slot, ky);
                    else M = j_from(slot[64], slot[96]);
                    const float4 w = slot[M16 ? 96 : 128];
                    const float4 Gp = g32[np], Gq = g32[nq];
                    const float2 gp0 = make_float2(Gp.x, Gp.y), gp1 = make_float2(Gp.z, Gp.w);
                    const float2 gq0 = make_float2(Gq.x, Gq.y), gq1 = make_float2(Gq.z, Gq.w);
                    // X = M diag(conj g_q), V = diag(g_p) X, r = D - V
                    const float2 X00 = cmulc(M.a, gq0), X01 = cmulc(M.b, gq1);
                    const float2 X10 = cmulc(M.c, gq0), X11 = cmulc(M.d, gq1);
                    const float2 r00 = csub(D.a, cmul(gp0, X00)), r01 = csub(D.b, cmul(gp0, X01));
                    const float2 r10 = csub(D.c, cmul(gp1, X10)), r11 = csub(D.d, cmul(gp1, X11));
                    const float2 wr00 = cscale(r00, w.x), wr01 = cscale(r01, w.y);
                    const float2 wr10 = cscale(r10, w.z), wr11 = cscale(r11, w.w);
                    if (want_chi)
                        chi += fmaf(w.x, cnorm2(r00), fmaf(w.y, cnorm2(r01), fmaf(w.z, cnorm2(r10), w.w * cnorm2(r11))));
                    // p side: parameter k touches row k of V: d V[k][j] / d g_p[k] = X[k][j]
                    sp[0] += fmaf(w.x, cnorm2(X00), w.y * cnorm2(X01));
                    sp[1] += fmaf(w.z, cnorm2(X10), w.w * cnorm2(X11));
                    float2 j0 = cfma_conj(X01, wr01, cfma_conj(X00, wr00, make_float2(sp[2], sp[3])));
                    float2 j1 = cfma_conj(X11, wr11, cfma_conj(X10, wr10, make_float2(sp[4], sp[5])));
                    sp[2] = j0.x; sp[3] = j0.y; sp[4] = j1.x; sp[5] = j1.y;
                    // q side through the conjugate baseline: Y = M^H diag(conj g_p), r' = r^H, w' = P w
                    const float2 Y00 = cmulc(cconj(M.a), gp0), Y01 = cmulc(cconj(M.c), gp1);
                    const float2 Y10 = cmulc(cconj(M.b), gp0), Y11 = cmulc(cconj(M.d), gp1);
                    sq[0] += fmaf(w.x, cnorm2(Y00), w.z * cnorm2(Y01));
                    sq[1] += fmaf(w.y, cnorm2(Y10), w.w * cnorm2(Y11));
                    float2 k0 = cfma_conj(Y01, cconj(wr10), cfma_conj(Y00, cconj(wr00), make_float2(sq[2], sq[3])));
                    float2 k1 = cfma_conj(Y11, cconj(wr11), cfma_conj(Y10, cconj(wr01), make_float2(sq[4], sq[5])));
                    sq[2] = k0.x; sq[3] = k0.y; sq[4] = k1.x; sq[5] = k1.y;
                }
            });
            flush_runs(sp, kp, lane, acc);
            flush_runs(sq, kq, lane, acc);
            if (want_chi) {
                double c = chi;
                for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
                if (lane == 0) atomicAdd(&s_chi, c);
            }
            __syncthreads();
            if (want_chi && !(s_chi <= a.fb_chi2[pi] * (1.0 + 1e-5))) {
                // the starting gains fit worse than the fallback (or are not finite): restart
                // the problem from the fallback gains (every thread sees the same s_chi); the
                // slack covers the different summation orders of the two chi^2 sums
                for (int i = tid; i < na; i += blockDim.x) {
                    const float2 f0 = a.fb_gains[(size_t)(P.gain_off + i) * 2];
                    const float2 f1 = a.fb_gains[(size_t)(P.gain_off + i) * 2 + 1];
                    g32[i] = make_float4(f0.x, f0.y, f1.x, f1.y);
                    g64[2 * i] = make_double2(f0.x, f0.y);
                    g64[2 * i + 1] = make_double2(f1.x, f1.y);
                }
                fell_back = true;
                __syncthreads();
                --k;
                continue;
            }
            // FP64 per-antenna solve and update (diagonal blocks: off-diagonal terms vanish)
            const double alpha = a.damping_mode == QC_DAMP_ALTERNATE ? ((k % 2 == 0) ? 0.5 : 1.0)
                                                                      : (a.damping > 0 ? a.damping : 1.0);
            double num = 0, den = 0;
            for (int ant = tid; ant < na; ant += blockDim.x) {
                const double h0 = acc[ant * 6], h1 = acc[ant * 6 + 1];
                const double hmax = fmax(h0, h1), hmin = fmin(h0, h1);
                const bool singular = !(h0 + h1 > 0) || !(hmin / hmax >= 1e-12);
                double2 d0 = make_double2(0, 0), d1 = d0;
                if (!singular) {
                    d0 = make_double2(alpha * acc[ant * 6 + 2] / h0, alpha * acc[ant * 6 + 3] / h0);
                    d1 = make_double2(alpha * acc[ant * 6 + 4] / h1, alpha * acc[ant * 6 + 5] / h1);
                }
                double2 G0 = g64[2 * ant], G1 = g64[2 * ant + 1];
                G0.x += d0.x; G0.y += d0.y; G1.x += d1.x; G1.y += d1.y;
                g64[2 * ant] = G0;
                g64[2 * ant + 1] = G1;
                g32[ant] = make_float4((float)G0.x, (float)G0.y, (float)G1.x, (float)G1.y);
                if (a.gain_flags) a.gain_flags[P.gain_off + ant] = singular ? 1 : 0;
                num += d0.x * d0.x + d0.y * d0.y + d1.x * d1.x + d1.y * d1.y;
                den += G0.x * G0.x + G0.y * G0.y + G1.x * G1.x + G1.y * G1.y;
            }
            for (int d = 16; d > 0; d >>= 1) {
                num += __shfl_down_sync(0xffffffffu, num, d);
                den += __shfl_down_sync(0xffffffffu, den, d);
            }
            if (lane == 0) { red[0][warp] = num; red[1][warp] = den; }
            __syncthreads();
            if (tid == 0) {
                double tn = 0, td = 0;
                for (int i = 0; i < n_warps; ++i) { tn += red[0][i]; td += red[1][i]; }
                const double delta = td > 0 ? sqrt(tn / td) : 0.0;
                s_done = delta < a.tol ? 1 : 0;
            }
            __syncthreads();
            if (s_done) break;
        }
        const int done_iters = k > a.max_iter ? a.max_iter : k;
        for (int i = tid; i < na; i += blockDim.x) {
            const float4 g = g32[i];
            a.gains[(size_t)(P.gain_off + i) * 2] = make_float2(g.x, g.y);
            a.gains[(size_t)(P.gain_off + i) * 2 + 1] = make_float2(g.z, g.w);
        }
        if (tid == 0) {
            if (a.iters) a.iters[pi] = done_iters;
            const unsigned long long ns = (unsigned long long)n_samp;
            const unsigned long long passes = done_iters + (fell_back ? 1 : 0);   // data passes made
            atomicAdd(a.vis_iters, ns * passes);
            const unsigned long long b = (a.flag ? ns : 0ull) + (unsigned long long)P.n_unflag * (M16 ? 64ull : 80ull);
            atomicAdd(a.bytes, b * passes);
            if (fell_back) atomicAdd(a.n_fallback, 1ull);
        }
        __syncthreads();
    }
}


// chi^2 of every problem at the given gains (one CTA per problem, FP64 block sums)
template <bool M16>
__global__ void __launch_bounds__(256) batch_chi2_kernel(const BatchArgs a, double *chi2)
{
    __shared__ double red[8];
    const int pi = blockIdx.x;
    const BProb P = a.probs[pi];
    const long n = (long)P.n_rows * P.n_chan;
    double tot = 0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) {
        const int row = (int)(i / P.n_chan);
        const int2 pq = __ldg(a.ants + P.row_off + row);
        const size_t s = (size_t)P.vis_off + i;
        if (pq.x == pq.y || (a.flag && __ldg(a.flag + s))) continue;
        const J2 D = j_from(__ldg(a.vis + 2 * s), __ldg(a.vis + 2 * s + 1));
        J2 M;
        if constexpr (M16) {
            const uint4 h = __ldg(a.model16 + s);
            const float sc = __ldg(a.row_scale + P.row_off + row);
            M.a = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.x)), sc);
            M.b = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.y)), sc);
            M.c = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.z)), sc);
            M.d = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.w)), sc);
        } else {
            M = j_from(__ldg(a.model + 2 * s), __ldg(a.model + 2 * s + 1));
        }
        const float4 w = __ldg(a.weight + s);
        const float2 *g = a.gains + (size_t)P.gain_off * 2;
        const float2 gp0 = g[2 * pq.x], gp1 = g[2 * pq.x + 1], gq0 = g[2 * pq.y], gq1 = g[2 * pq.y + 1];
        const float2 r00 = csub(D.a, cmul(gp0, cmulc(M.a, gq0))), r01 = csub(D.b, cmul(gp0, cmulc(M.b, gq1)));
        const float2 r10 = csub(D.c, cmul(gp1, cmulc(M.c, gq0))), r11 = csub(D.d, cmul(gp1, cmulc(M.d, gq1)));
        tot += (double)(w.x * cnorm2(r00)) + (double)(w.y * cnorm2(r01)) + (double)(w.z * cnorm2(r10)) +
               (double)(w.w * cnorm2(r11));
    }
    for (int d = 16; d > 0; d >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < (int)blockDim.x / 32; ++i) t += red[i];
        chi2[pi] = t;
    }
}


// Segmented flush of N register sums per lane (keys as in flush_runs) into acc[key][N].
template <int N>
__device__ __forceinline__ void flush_runs_n(float (&s)[N], int key, int lane, float *acc)
{
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || key != prev;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned after = heads & ~((2u << lane) - 1u);
    const unsigned run_end = after ? (unsigned)(__ffs(after) - 1) : 32u;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float sum = run_sum(s[i], lane, run_end);
        if (head && key >= 0) atomicAdd(acc + key * N + i, sum);
        s[i] = 0.f;
    }
}

constexpr int FEAT_DEPTH = 4;     // ring stages of the features pass

// Per-antenna warm-start features of every problem (one CTA per problem, one data
// pass at unit gains through the solver's streaming skeleton): JHJ diagonal and JHr
// at g = 1 (both baseline orientations), sums of |d_kk| / |m_kk| and their counts,
// and (optionally) chi^2 at the previous-interval gains; then the 10 features per
// antenna.
template <bool M16>
__global__ void __launch_bounds__(256) batch_features_kernel(const BatchArgs a, const float2 *prev, float *feat,
                                                             double *chi2_prev)
{
    constexpr int DEPTH = FEAT_DEPTH, V4 = BatchRing<M16>::V4;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n_warps = blockDim.x >> 5;
    float4 *ring = reinterpret_cast<float4 *>(smem) + (size_t)warp * DEPTH * V4 * 32;
    int2 *meta = reinterpret_cast<int2 *>(reinterpret_cast<float4 *>(smem) + (size_t)n_warps * DEPTH * V4 * 32) +
                 (size_t)warp * DEPTH * 32;
    unsigned char *tail = smem + (size_t)n_warps * batch_ring_bytes_per_warp<M16, DEPTH>();
    float4 *gprev = reinterpret_cast<float4 *>(tail);                  // [max_ant] previous gains (g_XX, g_YY)
    float *acc = reinterpret_cast<float *>(gprev + a.max_ant);        // [max_ant][9]: h0 h1 jr0 ji0 jr1 ji1 s0 s1 cnt
    __shared__ float2 ref[2];
    __shared__ double s_chi;
    const int pi = blockIdx.x;
    const BProb P = a.probs[pi];
    const int na = P.n_ant;
    const bool want_chi = chi2_prev != nullptr && prev != nullptr;
    for (int i = tid; i < na * 9; i += blockDim.x) acc[i] = 0.f;
    for (int i = tid; i < na; i += blockDim.x) {
        const float2 g0 = prev ? prev[(size_t)(P.gain_off + i) * 2] : make_float2(1.f, 0.f);
        const float2 g1 = prev ? prev[(size_t)(P.gain_off + i) * 2 + 1] : make_float2(1.f, 0.f);
        gprev[i] = make_float4(g0.x, g0.y, g1.x, g1.y);
    }
    if (tid == 0) s_chi = 0.0;
    __syncthreads();
    float chi = 0.f;
    float sp[9], sq[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) sp[i] = sq[i] = 0.f;
    int kp = -1, kq = -1;
    stream_pass<M16, DEPTH>(a, P, ring, meta, lane, warp, n_warps, [&](const float4 *slot, int kx, int ky) {
        const int p = kx >= 0 ? (kx & 0xffff) : -1;
        const int q = kx >= 0 ? (kx >> 16) : -1;
        if (__any_sync(0xffffffffu, p != kp)) { flush_runs_n<9>(sp, kp, lane, acc); kp = p; }
        if (__any_sync(0xffffffffu, q != kq)) { flush_runs_n<9>(sq, kq, lane, acc); kq = q; }
        if (kx < 0) return;
        // flagged samples and autocorrelations arrive as zeros: no contribution below
        const J2 D = j_from(slot[0], slot[32]);
        J2 M;
        if constexpr (M16) M = ring_model16(slot, ky);
        else M = j_from(slot[64], slot[96]);
        const float4 w = slot[M16 ? 96 : 128];
        // unit gains: X = M, V = M, r = D - M
        const float2 r00 = csub(D.a, M.a), r01 = csub(D.b, M.b), r10 = csub(D.c, M.c), r11 = csub(D.d, M.d);
        sp[0] += fmaf(w.x, cnorm2(M.a), w.y * cnorm2(M.b));
        sp[1] += fmaf(w.z, cnorm2(M.c), w.w * cnorm2(M.d));
        float2 j0 = cfma_conj(M.b, cscale(r01, w.y), cfma_conj(M.a, cscale(r00, w.x), make_float2(sp[2], sp[3])));
        float2 j1 = cfma_conj(M.d, cscale(r11, w.w), cfma_conj(M.c, cscale(r10, w.z), make_float2(sp[4], sp[5])));
        sp[2] = j0.x; sp[3] = j0.y; sp[4] = j1.x; sp[5] = j1.y;
        const float ma = sqrtf(cnorm2(M.a)), md = sqrtf(cnorm2(M.d));
        const bool okr = ma > 0.f && md > 0.f;
        const float ra = okr ? sqrtf(cnorm2(D.a)) / ma : 0.f, rd = okr ? sqrtf(cnorm2(D.d)) / md : 0.f;
        sp[6] += ra; sp[7] += rd; sp[8] += okr ? 1.f : 0.f;
        // conjugate baseline for antenna q: Y = M^H, r' = r^H, w' = P w
        sq[0] += fmaf(w.x, cnorm2(M.a), w.z * cnorm2(M.c));
        sq[1] += fmaf(w.y, cnorm2(M.b), w.w * cnorm2(M.d));
        float2 k0 = cfma_conj(cconj(M.c), cscale(cconj(r10), w.z), cfma_conj(cconj(M.a), cscale(cconj(r00), w.x), make_float2(sq[2], sq[3])));
        float2 k1 = cfma_conj(cconj(M.d), cscale(cconj(r11), w.w), cfma_conj(cconj(M.b), cscale(cconj(r01), w.y), make_float2(sq[4], sq[5])));
        sq[2] = k0.x; sq[3] = k0.y; sq[4] = k1.x; sq[5] = k1.y;
        sq[6] += ra; sq[7] += rd; sq[8] += okr ? 1.f : 0.f;
        if (want_chi) {
            // chi^2 at the previous-interval gains (Eq. min), for the fallback check
            const float4 Gp = gprev[p], Gq = gprev[q];
            const float2 gp0 = make_float2(Gp.x, Gp.y), gp1 = make_float2(Gp.z, Gp.w);
            const float2 gq0 = make_float2(Gq.x, Gq.y), gq1 = make_float2(Gq.z, Gq.w);
            const float2 e00 = csub(D.a, cmul(gp0, cmulc(M.a, gq0))), e01 = csub(D.b, cmul(gp0, cmulc(M.b, gq1)));
            const float2 e10 = csub(D.c, cmul(gp1, cmulc(M.c, gq0))), e11 = csub(D.d, cmul(gp1, cmulc(M.d, gq1)));
            chi += fmaf(w.x, cnorm2(e00), fmaf(w.y, cnorm2(e01), fmaf(w.z, cnorm2(e10), w.w * cnorm2(e11))));
        }
    });
    flush_runs_n<9>(sp, kp, lane, acc);
    flush_runs_n<9>(sq, kq, lane, acc);
    if (want_chi) {
        double c = chi;
        for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
        if (lane == 0) atomicAdd(&s_chi, c);
    }
    __syncthreads();
    if (want_chi && tid == 0) chi2_prev[pi] = s_chi;
    // references: phase of the sum over antennas, per correlation, of the previous-interval
    // gains (ref) and of the one-step gains 1 + JHr/JHJ at unit gains (ref1)
    __shared__ float2 ref1[2];
    if (tid < 4) {
        const int k = tid & 1;
        float2 sum = make_float2(0.f, 0.f);
        for (int ant = 0; ant < na; ++ant) {
            float2 g;
            if (tid < 2) {
                g = prev ? prev[(size_t)(P.gain_off + ant) * 2 + k] : make_float2(1.f, 0.f);
            } else {
                const float *A = acc + ant * 9;
                const float h = A[k];
                g = h > 0.f ? make_float2(1.f + A[2 + 2 * k] / h, A[3 + 2 * k] / h) : make_float2(0.f, 0.f);
            }
            sum = cadd(sum, g);
        }
        const float mag = sqrtf(cnorm2(sum));
        const float2 r = mag > 0.f ? make_float2(sum.x / mag, -sum.y / mag) : make_float2(1.f, 0.f);
        if (tid < 2) ref[k] = r;
        else ref1[k] = r;
    }
    __syncthreads();
    for (int ant = tid; ant < na; ant += blockDim.x) {
        const float *A = acc + ant * 9;
        float *f = feat + (size_t)(P.gain_off + ant) * 10;
        for (int k = 0; k < 2; ++k) {
            const float h = A[k];
            const float2 z = h > 0.f ? make_float2(A[2 + 2 * k] / h, A[3 + 2 * k] / h) : make_float2(0.f, 0.f);
            f[k] = sqrtf(cnorm2(z));
            const float2 g1 = cmul(make_float2(1.f + z.x, z.y), ref1[k]);
            f[2 + k] = h > 0.f ? atan2f(g1.y, g1.x) : 0.f;
            f[4 + k] = A[8] > 0.f ? A[6 + k] / A[8] : 0.f;
            const float2 g = prev ? prev[(size_t)(P.gain_off + ant) * 2 + k] : make_float2(1.f, 0.f);
            const float2 gr = cmul(g, ref[k]);
            f[6 + 2 * k] = gr.x;
            f[7 + 2 * k] = gr.y;
        }
    }
}


// gains of each problem rotated so that their sum over antennas is real-positive per correlation
__global__ void reference_gains_kernel(const BProb *probs, int n_prob, const float2 *in, float2 *out)
{
    const int pi = blockIdx.x;
    if (pi >= n_prob) return;
    const BProb P = probs[pi];
    __shared__ float2 ref[2];
    if (threadIdx.x < 2) {
        float2 sum = make_float2(0.f, 0.f);
        for (int ant = 0; ant < P.n_ant; ++ant) sum = cadd(sum, in[(size_t)(P.gain_off + ant) * 2 + threadIdx.x]);
        const float mag = sqrtf(cnorm2(sum));
        ref[threadIdx.x] = mag > 0.f ? make_float2(sum.x / mag, -sum.y / mag) : make_float2(1.f, 0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P.n_ant * 2; i += blockDim.x) {
        const size_t g = (size_t)P.gain_off * 2 + i;
        out[g] = cmul(in[g], ref[i & 1]);
    }
}

// gains from network outputs; non-finite outputs make the whole problem fall back
__global__ void warm_gains_kernel(const BProb *probs, int n_prob, const float *y, const float2 *fallback, float2 *out,
                                  int *bad)
{
    const int pi = blockIdx.x;
    if (pi >= n_prob) return;
    const BProb P = probs[pi];
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < P.n_ant * 4; i += blockDim.x)
        if (!isfinite(y[(size_t)P.gain_off * 4 + i])) s_bad = 1;
    __syncthreads();
    for (int ant = threadIdx.x; ant < P.n_ant; ant += blockDim.x) {
        const size_t g = (size_t)(P.gain_off + ant);
        if (s_bad) {
            out[2 * g] = fallback[2 * g];
            out[2 * g + 1] = fallback[2 * g + 1];
        } else {
            out[2 * g] = make_float2(y[4 * g], y[4 * g + 1]);
            out[2 * g + 1] = make_float2(y[4 * g + 2], y[4 * g + 3]);
        }
    }
    if (threadIdx.x == 0) bad[pi] = s_bad;
}

// keep the fallback gains of problems whose chi^2 at the predicted gains is larger
__global__ void warm_select_kernel(const BProb *probs, int n_prob, const double *chi_pred, const double *chi_fb,
                                   const float2 *fallback, float2 *out, int *bad)
{
    const int pi = blockIdx.x;
    if (pi >= n_prob) return;
    const BProb P = probs[pi];
    const bool use_fb = !(chi_pred[pi] <= chi_fb[pi]);
    for (int ant = threadIdx.x; ant < P.n_ant; ant += blockDim.x) {
        const size_t g = (size_t)(P.gain_off + ant);
        if (use_fb) { out[2 * g] = fallback[2 * g]; out[2 * g + 1] = fallback[2 * g + 1]; }
    }
    if (threadIdx.x == 0 && use_fb) bad[pi] = 1;
}

__global__ void row_scale_kernel(const float4 *model, const int2 *ants, const long long *row_vis, const int *row_nc,
                                 const int *row_bl, long n_rows, unsigned *bl_bits)
{
    for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += (long)gridDim.x * blockDim.x) {
        const int2 pq = ants[r];
        if (pq.x == pq.y) continue;
        float m = 0.f;
        for (int c = 0; c < row_nc[r]; ++c) {
            const size_t s = (size_t)row_vis[r] + c;
            const float4 a = model[2 * s], b = model[2 * s + 1];
            m = fmaxf(m, fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))),
                               fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w)))));
        }
        if (!(m <= 3.0e38f)) m = 0.f;
        atomicMax(bl_bits + row_bl[r], __float_as_uint(m));
    }
}

__global__ void row_scale_fill(const int *row_bl, const unsigned *bl_bits, long n_rows, float *row_scale)
{
    for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += (long)gridDim.x * blockDim.x) {
        const float v = __uint_as_float(bl_bits[row_bl[r]]);
        row_scale[r] = v > 0.f ? v : 1.f;
    }
}

__global__ void pack16_rows_kernel(const float4 *model, const float *row_scale, const long long *row_vis,
                                   const int *row_nc, long n_rows, uint4 *out)
{
    for (long r = blockIdx.x; r < n_rows; r += gridDim.x) {
        const float inv = 1.f / row_scale[r];
        for (int c = threadIdx.x; c < row_nc[r]; c += blockDim.x) {
            const size_t s = (size_t)row_vis[r] + c;
            const float4 a = model[2 * s], b = model[2 * s + 1];
            __half2 h0 = __floats2half2_rn(a.x * inv, a.y * inv), h1 = __floats2half2_rn(a.z * inv, a.w * inv);
            __half2 h2 = __floats2half2_rn(b.x * inv, b.y * inv), h3 = __floats2half2_rn(b.z * inv, b.w * inv);
            uint4 o;
            o.x = *reinterpret_cast<unsigned *>(&h0);
            o.y = *reinterpret_cast<unsigned *>(&h1);
            o.z = *reinterpret_cast<unsigned *>(&h2);
            o.w = *reinterpret_cast<unsigned *>(&h3);
            out[s] = o;
        }
    }
}

__global__ void unflag_count_kernel(const uint8_t *flag, const BProb *probs, const int2 *ants, int n_prob,
                                    unsigned long long *out)
{
    const int pi = blockIdx.x;
    if (pi >= n_prob) return;
    const BProb P = probs[pi];
    const long n = (long)P.n_rows * P.n_chan;
    unsigned long long cnt = 0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) {
        const int row = (int)(i / P.n_chan);
        const int2 pq = ants[P.row_off + row];
        if (pq.x != pq.y && !(flag && flag[P.vis_off + i])) ++cnt;
    }
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0) atomicAdd(out + pi, cnt);
}


// ---------------------------------------------------------------------------
// batched solve from per-baseline sums (sufficient-statistics pre-reduction)
// ---------------------------------------------------------------------------
// Not in the paper.  A problem of the batch is one solution interval of one diagonal term,
// so a baseline's samples enter JHJ and JHr only through two weighted sums per correlation c,
// S_c = sum w_c |m_c|^2 and T_c = sum w_c conj(m_c) d_c.  One pass over the problem's samples
// forms them per baseline in shared memory; every iteration then forms the normal equations
// from them in FP64 (correlations XX XY YX YY = 0 1 2 3):
//   antenna p of (p, q):  h0 = S0 |gq0|^2 + S1 |gq1|^2,   h1 = S2 |gq0|^2 + S3 |gq1|^2,
//                         j0 = gq0 T0 + gq1 T1 - gp0 h0,  j1 = gq0 T2 + gq1 T3 - gp1 h1;
//   antenna q through the conjugate baseline: S1 <-> S2, T -> conj(T) with T1 <-> T2, p <-> q.
// The update and the convergence test are those of batch_kernel.

constexpr int MOM_MAX_ANT = 64;   // baselines x 13 floats must fit in shared memory
constexpr int MOM_W = 13;         // S[4], T[4] as (re, im), U = sum_c w_c |d_c|^2

__host__ __device__ constexpr int mom_bl(int p, int q, int n) { return p * (2 * n - p - 1) / 2 + (q - p - 1); }

__host__ __device__ inline size_t mom_smem_bytes(int max_ant)
{
    const size_t m = ((size_t)max_ant * (max_ant - 1) / 2 * MOM_W * sizeof(float) + 15) / 16 * 16;
    return m + (size_t)max_ant * 2 * sizeof(double2) + (size_t)max_ant * 6 * sizeof(double) +
           (size_t)max_ant * 2 * sizeof(float2);
}

template <bool M16>
__global__ void __launch_bounds__(256) batch_moments_kernel(const BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char msm[];
    const size_t mom_bytes = ((size_t)a.max_ant * (a.max_ant - 1) / 2 * MOM_W * sizeof(float) + 15) / 16 * 16;
    float *mom = reinterpret_cast<float *>(msm);                                  // [n_bl][MOM_W]
    double2 *g64 = reinterpret_cast<double2 *>(msm + mom_bytes);                 // [max_ant][2]
    double *acc = reinterpret_cast<double *>(g64 + 2 * a.max_ant);               // [max_ant][6]
    float2 *g32 = reinterpret_cast<float2 *>(acc + 6 * a.max_ant);               // [max_ant][2]
    __shared__ double red[2][8];
    __shared__ int s_done;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n_warps = blockDim.x >> 5;
    const int pi = a.order[blockIdx.x];
    const BProb P = a.probs[pi];
    const int na = P.n_ant, nc = P.n_chan, n_bl = na * (na - 1) / 2;
    for (int i = tid; i < n_bl * MOM_W; i += blockDim.x) mom[i] = 0.f;
    for (int i = tid; i < na; i += blockDim.x) {
        const float2 g0 = a.gains[(size_t)(P.gain_off + i) * 2], g1 = a.gains[(size_t)(P.gain_off + i) * 2 + 1];
        g64[2 * i] = make_double2(g0.x, g0.y);
        g64[2 * i + 1] = make_double2(g1.x, g1.y);
    }
    __syncthreads();
    // one pass over the samples: the baseline sums.  The lanes of a warp take consecutive
    // samples, two groups of 32 per step with both groups' loads issued first; where a group's
    // samples all belong to one baseline (a row of 32 channels or more) a transposed reduction
    // leaves one total per sum and one shared add each, otherwise every lane adds its own (short
    // runs of equal baselines: few conflicts).  Sample indices are 32-bit within a problem.
    const long long n_samp = (long long)P.n_rows * nc;
    struct Samp {
        int key;                 // the row's baseline slot (flagged samples too: keeps runs whole)
        bool use;                // unflagged cross-correlation sample
        float4 w, d0, d1, m0, m1;
        uint4 h;
        float sc;
        bool conj;
    };
    auto load = [&](long long s) {
        Samp x;
        x.key = -1;
        x.use = false;
        x.conj = false;
        if (s < n_samp) {
            const int si = (int)s, row = si / nc;
            const int2 pq = a.ants[P.row_off + row];
            const long long sg = P.vis_off + s;
            if (pq.x != pq.y) {
                x.conj = pq.x > pq.y;
                x.key = x.conj ? mom_bl(pq.y, pq.x, na) : mom_bl(pq.x, pq.y, na);
                x.use = !(a.flag && a.flag[sg]);
            }
            if (x.use) {
                x.d0 = a.vis[2 * sg];
                x.d1 = a.vis[2 * sg + 1];
                if constexpr (M16) {
                    x.h = a.model16[sg];
                    x.sc = a.row_scale[P.row_off + row];
                } else {
                    x.m0 = a.model[2 * sg];
                    x.m1 = a.model[2 * sg + 1];
                }
                x.w = a.weight[sg];
            }
        }
        return x;
    };
    auto add = [&](const Samp &x) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
        if (x.use) {
            J2 D = j_from(x.d0, x.d1);
            J2 M;
            if constexpr (M16) {
                M.a = cscale(h2f(*reinterpret_cast<const __half2 *>(&x.h.x)), x.sc);
                M.b = cscale(h2f(*reinterpret_cast<const __half2 *>(&x.h.y)), x.sc);
                M.c = cscale(h2f(*reinterpret_cast<const __half2 *>(&x.h.z)), x.sc);
                M.d = cscale(h2f(*reinterpret_cast<const __half2 *>(&x.h.w)), x.sc);
            } else {
                M = j_from(x.m0, x.m1);
            }
            float4 w = x.w;
            if (x.conj) {     // the conjugate baseline: D, M -> D^H, M^H, weights permuted
                D = j_herm(D);
                M = j_herm(M);
                w = make_float4(w.x, w.z, w.y, w.w);
            }
            const float2 Mv[4] = { M.a, M.b, M.c, M.d }, Dv[4] = { D.a, D.b, D.c, D.d };
            const float wv[4] = { w.x, w.y, w.z, w.w };
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                v[c] = wv[c] * cnorm2(Mv[c]);
                const float2 t = cscale(cmulc(Dv[c], Mv[c]), wv[c]);      // w conj(m) d
                v[4 + 2 * c] = t.x;
                v[5 + 2 * c] = t.y;
                v[12] = fmaf(wv[c], cnorm2(Dv[c]), v[12]);                 // w |d|^2 (chi^2 from the sums)
            }
        }
        const int key = x.key;
        const int k0 = __shfl_sync(0xffffffffu, key, 0);
        if (__all_sync(0xffffffffu, key == k0)) {
            if (k0 >= 0) {
                // 16 slots (13 sums + 3 zeros) over 32 lanes: four halving exchanges, then a
                // butterfly; lane l holds the total of slot l >> 1
                int idx = 0;
#pragma unroll
                for (int lev = 0; lev < 4; ++lev) {
                    const int d = 16 >> lev, h = 8 >> lev;
                    const bool up = (lane & d) != 0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (i < h) {
                            const float send = up ? v[i] : v[i + h];
                            const float keep = up ? v[i + h] : v[i];
                            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, d);
                        }
                    }
                    if (up) idx += h;
                }
                v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
                if ((lane & 1) == 0 && idx < MOM_W) atomicAdd(&mom[(size_t)k0 * MOM_W + idx], v[0]);
            }
        } else {
            // runs of equal keys (the samples of one row, when rows are shorter than 32): a
            // segmented reduction per sum, one shared add per run; keys that repeat apart (two
            // rows of one baseline in a group) add per lane
            const unsigned m = __match_any_sync(0xffffffffu, key);
            const unsigned lo = m & (0u - m);
            const bool contig = ((m + lo) & m) == 0;          // the set bits of m are one run
            if (__all_sync(0xffffffffu, contig)) {
                const int seg_end = 32 - __clz(m);
                const bool head = lane == __ffs(m) - 1;
#pragma unroll
                for (int i = 0; i < MOM_W; ++i) {
                    float t = v[i];
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const float o = __shfl_down_sync(0xffffffffu, t, d);
                        if (lane + d < seg_end) t += o;
                    }
                    if (head && key >= 0) atomicAdd(&mom[(size_t)key * MOM_W + i], t);
                }
            } else if (key >= 0) {
#pragma unroll
                for (int i = 0; i < MOM_W; ++i) atomicAdd(&mom[(size_t)key * MOM_W + i], v[i]);
            }
        }
    };
    for (long long base = (long long)warp * 64; base < n_samp; base += 2LL * blockDim.x) {
        const Samp x0 = load(base + lane), x1 = load(base + 32 + lane);
        add(x0);
        add(x1);
    }
    __syncthreads();
    // a fallback start: chi^2 at the starting and at the fallback gains from the sums (per
    // baseline U - 2 Re sum_c conj(g_pk) g_qj T_c + sum_c |g_pk|^2 |g_qj|^2 S_c, c = 2k + j, in
    // FP64 from the FP32 sums); a start that fits worse by more than a relative 1e-5, or whose
    // chi^2 is not finite, is replaced by the fallback gains
    if (a.fb_gains) {
        double c0 = 0, c1 = 0;
        for (int idx = tid; idx < na * na; idx += blockDim.x) {
            const int p = idx / na, q = idx - p * na;
            if (p >= q) continue;
            const float *m = mom + (size_t)mom_bl(p, q, na) * MOM_W;
            const float2 *s0 = a.gains + (size_t)P.gain_off * 2, *s1 = a.fb_gains + (size_t)P.gain_off * 2;
            double t0 = m[12], t1 = m[12];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int kk = c >> 1, jj = c & 1;
                const double S = m[c], Tr = m[4 + 2 * c], Ti = m[5 + 2 * c];
                const float2 gp0 = s0[2 * p + kk], gq0 = s0[2 * q + jj], gp1 = s1[2 * p + kk], gq1 = s1[2 * q + jj];
                // conj(g_pk) g_qj
                const double a0r = (double)gp0.x * gq0.x + (double)gp0.y * gq0.y;
                const double a0i = (double)gp0.x * gq0.y - (double)gp0.y * gq0.x;
                const double a1r = (double)gp1.x * gq1.x + (double)gp1.y * gq1.y;
                const double a1i = (double)gp1.x * gq1.y - (double)gp1.y * gq1.x;
                t0 += S * (a0r * a0r + a0i * a0i) - 2.0 * (a0r * Tr - a0i * Ti);
                t1 += S * (a1r * a1r + a1i * a1i) - 2.0 * (a1r * Tr - a1i * Ti);
            }
            c0 += t0;
            c1 += t1;
        }
        for (int d = 16; d > 0; d >>= 1) {
            c0 += __shfl_down_sync(0xffffffffu, c0, d);
            c1 += __shfl_down_sync(0xffffffffu, c1, d);
        }
        if (lane == 0) { red[0][warp] = c0; red[1][warp] = c1; }
        __syncthreads();
        if (tid == 0) {
            double t0 = 0, t1 = 0;
            for (int i = 0; i < n_warps; ++i) { t0 += red[0][i]; t1 += red[1][i]; }
            s_done = !(t0 <= t1 * (1.0 + 1e-5)) ? 1 : 0;
            if (s_done) atomicAdd(a.n_fallback, 1ull);
        }
        __syncthreads();
        if (s_done) {
            for (int i = tid; i < na; i += blockDim.x) {
                const float2 f0 = a.fb_gains[(size_t)(P.gain_off + i) * 2];
                const float2 f1 = a.fb_gains[(size_t)(P.gain_off + i) * 2 + 1];
                g64[2 * i] = make_double2(f0.x, f0.y);
                g64[2 * i + 1] = make_double2(f1.x, f1.y);
            }
        }
        __syncthreads();
    }
    int k;
    for (k = 1; k <= a.max_iter; ++k) {
        // the normal equations of each antenna from the sums of its baselines (no atomics: one
        // thread per antenna, float32 sums as batch_kernel's accumulators)
        for (int i = tid; i < 2 * na; i += blockDim.x) g32[i] = make_float2((float)g64[i].x, (float)g64[i].y);
        __syncthreads();
        for (int ant = tid; ant < na; ant += blockDim.x) {
            const float2 ga0 = g32[2 * ant], ga1 = g32[2 * ant + 1];
            float h0 = 0.f, h1 = 0.f;
            float2 j0 = make_float2(0.f, 0.f), j1 = j0;
            for (int o = 0; o < na; ++o) {
                if (o == ant) continue;
                const float2 go0 = g32[2 * o], go1 = g32[2 * o + 1];
                const float ao0 = cnorm2(go0), ao1 = cnorm2(go1);
                if (ant < o) {      // antenna p of (ant, o)
                    const float *m = mom + (size_t)mom_bl(ant, o, na) * MOM_W;
                    const float e0 = m[0] * ao0 + m[1] * ao1, e1 = m[2] * ao0 + m[3] * ao1;
                    const float2 T0 = make_float2(m[4], m[5]), T1 = make_float2(m[6], m[7]);
                    const float2 T2 = make_float2(m[8], m[9]), T3 = make_float2(m[10], m[11]);
                    h0 += e0;
                    h1 += e1;
                    j0 = cadd(j0, csub(cadd(cmul(go0, T0), cmul(go1, T1)), cscale(ga0, e0)));
                    j1 = cadd(j1, csub(cadd(cmul(go0, T2), cmul(go1, T3)), cscale(ga1, e1)));
                } else {            // antenna q of (o, ant), through the conjugate baseline
                    const float *m = mom + (size_t)mom_bl(o, ant, na) * MOM_W;
                    const float e0 = m[0] * ao0 + m[2] * ao1, e1 = m[1] * ao0 + m[3] * ao1;
                    const float2 T0 = make_float2(m[4], m[5]), T1 = make_float2(m[6], m[7]);
                    const float2 T2 = make_float2(m[8], m[9]), T3 = make_float2(m[10], m[11]);
                    h0 += e0;
                    h1 += e1;
                    j0 = cadd(j0, csub(cadd(cmulc(go0, T0), cmulc(go1, T2)), cscale(ga0, e0)));
                    j1 = cadd(j1, csub(cadd(cmulc(go0, T1), cmulc(go1, T3)), cscale(ga1, e1)));
                }
            }
            acc[ant * 6 + 0] = h0;
            acc[ant * 6 + 1] = h1;
            acc[ant * 6 + 2] = j0.x;
            acc[ant * 6 + 3] = j0.y;
            acc[ant * 6 + 4] = j1.x;
            acc[ant * 6 + 5] = j1.y;
        }
        __syncthreads();
        // FP64 per-antenna solve and update, as batch_kernel
        const double alpha = a.damping_mode == QC_DAMP_ALTERNATE ? ((k % 2 == 0) ? 0.5 : 1.0)
                                                                  : (a.damping > 0 ? a.damping : 1.0);
        double num = 0, den = 0;
        for (int ant = tid; ant < na; ant += blockDim.x) {
            const double h0 = acc[ant * 6], h1 = acc[ant * 6 + 1];
            const double hmax = fmax(h0, h1), hmin = fmin(h0, h1);
            const bool singular = !(h0 + h1 > 0) || !(hmin / hmax >= 1e-12);
            double2 d0 = make_double2(0, 0), d1 = d0;
            if (!singular) {
                d0 = make_double2(alpha * acc[ant * 6 + 2] / h0, alpha * acc[ant * 6 + 3] / h0);
                d1 = make_double2(alpha * acc[ant * 6 + 4] / h1, alpha * acc[ant * 6 + 5] / h1);
            }
            double2 G0 = g64[2 * ant], G1 = g64[2 * ant + 1];
            G0.x += d0.x; G0.y += d0.y; G1.x += d1.x; G1.y += d1.y;
            g64[2 * ant] = G0;
            g64[2 * ant + 1] = G1;
            if (a.gain_flags) a.gain_flags[P.gain_off + ant] = singular ? 1 : 0;
            num += d0.x * d0.x + d0.y * d0.y + d1.x * d1.x + d1.y * d1.y;
            den += G0.x * G0.x + G0.y * G0.y + G1.x * G1.x + G1.y * G1.y;
        }
        for (int d = 16; d > 0; d >>= 1) {
            num += __shfl_down_sync(0xffffffffu, num, d);
            den += __shfl_down_sync(0xffffffffu, den, d);
        }
        if (lane == 0) { red[0][warp] = num; red[1][warp] = den; }
        __syncthreads();
        if (tid == 0) {
            double tn = 0, td = 0;
            for (int i = 0; i < n_warps; ++i) { tn += red[0][i]; td += red[1][i]; }
            const double delta = td > 0 ? sqrt(tn / td) : 0.0;
            s_done = delta < a.tol ? 1 : 0;
        }
        __syncthreads();
        if (s_done) break;
    }
    const int done_iters = k > a.max_iter ? a.max_iter : k;
    for (int i = tid; i < na; i += blockDim.x) {
        const double2 G0 = g64[2 * i], G1 = g64[2 * i + 1];
        a.gains[(size_t)(P.gain_off + i) * 2] = make_float2((float)G0.x, (float)G0.y);
        a.gains[(size_t)(P.gain_off + i) * 2 + 1] = make_float2((float)G1.x, (float)G1.y);
    }
    if (tid == 0) {
        if (a.iters) a.iters[pi] = done_iters;
        const unsigned long long ns = (unsigned long long)n_samp;
        atomicAdd(a.vis_iters, ns * done_iters);
        // one pass over the data
        atomicAdd(a.bytes, (a.flag ? ns : 0ull) + (unsigned long long)P.n_unflag * (M16 ? 64ull : 80ull));
    }
}

} // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct qc_batch {
    int dev = 0, sm_count = 1;
    cudaStream_t own_stream = nullptr;
    int n_prob = 0, max_ant = 0;
    long long n_rows = 0, n_vis = 0, total_ant = 0;
    bool m16 = false, has_flag = false;
    std::vector<void *> owned;
    const float4 *vis = nullptr, *model = nullptr, *weight = nullptr;
    const uint4 *model16 = nullptr;
    const uint8_t *flag = nullptr;
    float *row_scale = nullptr;
    int2 *ants = nullptr;
    BProb *probs = nullptr;
    int *order_lpt = nullptr, *order_idx = nullptr, *queue = nullptr;
    unsigned long long *counters = nullptr;
    void *gstage = nullptr;       // device staging for host gains/flags/iters
    std::vector<BProb> hprobs;
    std::vector<long long> lpt_samples;   // samples of the problems in LPT order (non-increasing)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaStream_t aux_stream = nullptr;    // the small-problem class's launch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // A launch shape: CTA size, residency, schedule, copy depth; with split > 0 the problems
    // with fewer samples than split form a second class launched concurrently with its own
    // CTA size and residency (tile = threads consecutive samples per CTA step).
    struct Shape { int threads, per_sm, schedule, depth; double ms; long long split; int s_threads, s_per_sm; };
    std::string shape_key;
    struct GraphKey { int threads, per_sm, schedule, depth, max_iter, damping_mode; double damping, tol; bool m16;
                      void *gains; void *flags; void *iters; cudaStream_t st; const void *fb_gains, *fb_chi2;
                      long long split; int s_threads, s_per_sm; };
    cudaGraphExec_t exec = nullptr;
    GraphKey gkey;
    std::string err;

    qc_batch() { memset(&gkey, 0, sizeof gkey); }
    ~qc_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        for (void *p : owned) qc_dev_free(p);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (aux_stream) cudaStreamDestroy(aux_stream);
        if (own_stream) cudaStreamDestroy(own_stream);
    }
    void *alloc(size_t bytes, cudaError_t *e)
    {
        void *p = nullptr;
        *e = qc_dev_malloc(&p, bytes);
        if (*e == cudaSuccess) owned.push_back(p);
        return p;
    }
    int fail(int code, const std::string &m) { err = m; return code; }
    int cuda_fail(cudaError_t e, const char *what)
    {
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? QC_ENOMEM : QC_ECUDA;
    }
};

#define BCK(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return b->cuda_fail(e_, #call);      \
    } while (0)

extern "C" int qc_batch_create(const qc_batch_problem *p, qc_batch **out)
{
    g_batch_create_error.clear();
    auto bad = [](const char *m) { g_batch_create_error = m; return QC_EINVAL; };
    if (!out) return bad("out is NULL");
    *out = nullptr;
    if (!p || p->n_prob < 1) return bad("empty batch");
    if (!p->row_offset || !p->vis_offset || !p->n_chan || !p->n_ant || !p->ant1 || !p->ant2)
        return bad("row_offset, vis_offset, n_chan, n_ant, ant1, ant2 are required (host arrays)");
    if (!p->data || !p->model || !p->weight) return bad("data, model and weight are required");
    if (p->memory != QC_MEM_HOST && p->memory != QC_MEM_DEVICE) return bad("memory must be QC_MEM_HOST or DEVICE");
    std::unique_ptr<qc_batch> b(new qc_batch());
    b->n_prob = p->n_prob;
    b->m16 = p->model_fp16 != 0;
    b->has_flag = p->flag != nullptr;
    if (p->row_offset[0] != 0 || p->vis_offset[0] != 0) return bad("offsets must start at 0");
    b->hprobs.resize(p->n_prob);
    long long gain_off = 0;
    for (int i = 0; i < p->n_prob; ++i) {
        const long long r0 = p->row_offset[i], r1 = p->row_offset[i + 1];
        const long long v0 = p->vis_offset[i], v1 = p->vis_offset[i + 1];
        const int nc = p->n_chan[i], na = p->n_ant[i];
        if (r1 < r0 || nc < 1 || na < 2 || na > QC_BATCH_MAX_ANT) return bad("invalid problem sizes");
        if (v1 - v0 != (r1 - r0) * nc) return bad("vis_offset inconsistent with rows x n_chan");
        if (r1 - r0 > (1LL << 30)) return bad("problem too large");
        for (long long r = r0; r < r1; ++r)
            if (p->ant1[r] < 0 || p->ant1[r] >= na || p->ant2[r] < 0 || p->ant2[r] >= na)
                return bad("antenna index out of range");
        BProb &P = b->hprobs[i];
        P.vis_off = v0;
        P.row_off = r0;
        P.n_rows = (int)(r1 - r0);
        P.n_chan = nc;
        P.n_ant = na;
        P.gain_off = (int)gain_off;
        P.n_unflag = 0;
        gain_off += na;
        b->max_ant = std::max(b->max_ant, na);
    }
    b->n_rows = p->row_offset[p->n_prob];
    b->n_vis = p->vis_offset[p->n_prob];
    b->total_ant = gain_off;
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->aux_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) { g_batch_create_error = std::string("CUDA init: ") + cudaGetErrorString(e); return QC_ECUDA; }
    cudaStream_t st = b->own_stream;
#define BALLOC(dst, T, n)                                                                    \
    do {                                                                                     \
        dst = (T *)b->alloc(sizeof(T) * (size_t)(n), &e);                                    \
        if (e != cudaSuccess) { g_batch_create_error = "cudaMalloc failed"; return e == cudaErrorMemoryAllocation ? QC_ENOMEM : QC_ECUDA; } \
    } while (0)
#define BH2D(dst, src, bytes)                                                                \
    do {                                                                                     \
        e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);                             \
        if (e != cudaSuccess) { g_batch_create_error = std::string("H2D: ") + cudaGetErrorString(e); return QC_ECUDA; } \
    } while (0)
    // rows: (p, q) and, for the FP16 model, the baseline id of each row
    std::vector<int2> ants(b->n_rows);
    for (long long r = 0; r < b->n_rows; ++r) ants[r] = make_int2(p->ant1[r], p->ant2[r]);
    BALLOC(b->ants, int2, std::max<long long>(1, b->n_rows));
    if (b->n_rows) BH2D(b->ants, ants.data(), sizeof(int2) * b->n_rows);
    const size_t nv = (size_t)b->n_vis;
    const float4 *model32 = nullptr;
    if (p->memory == QC_MEM_DEVICE) {
        b->vis = (const float4 *)p->data;
        model32 = (const float4 *)p->model;
        b->weight = (const float4 *)p->weight;
        b->flag = p->flag;
    } else {
        float4 *v, *w, *m;
        BALLOC(v, float4, 2 * nv);
        BH2D(v, p->data, sizeof(float4) * 2 * nv);
        BALLOC(m, float4, 2 * nv);
        BH2D(m, p->model, sizeof(float4) * 2 * nv);
        BALLOC(w, float4, nv);
        BH2D(w, p->weight, sizeof(float4) * nv);
        b->vis = v;
        b->weight = w;
        model32 = m;
        if (p->flag) {
            uint8_t *f;
            BALLOC(f, uint8_t, nv);
            BH2D(f, p->flag, nv);
            b->flag = f;
        }
    }
    BALLOC(b->probs, BProb, p->n_prob);
    BH2D(b->probs, b->hprobs.data(), sizeof(BProb) * p->n_prob);
    BALLOC(b->counters, unsigned long long, 3 + p->n_prob);
    // unflagged samples per problem
    e = cudaMemsetAsync(b->counters, 0, sizeof(unsigned long long) * (2 + p->n_prob), st);
    if (e == cudaSuccess) {
        unflag_count_kernel<<<p->n_prob, 256, 0, st>>>(b->flag, b->probs, b->ants, p->n_prob, b->counters + 2);
        e = cudaGetLastError();
    }
    std::vector<unsigned long long> unf(p->n_prob);
    if (e == cudaSuccess) e = cudaMemcpyAsync(unf.data(), b->counters + 2, sizeof(unsigned long long) * p->n_prob,
                                              cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { g_batch_create_error = std::string("flag counts: ") + cudaGetErrorString(e); return QC_ECUDA; }
    for (int i = 0; i < p->n_prob; ++i) b->hprobs[i].n_unflag = (long long)unf[i];
    BH2D(b->probs, b->hprobs.data(), sizeof(BProb) * p->n_prob);
    if (b->m16) {
        std::vector<long long> row_vis(b->n_rows);
        std::vector<int> row_nc(b->n_rows), row_bl(b->n_rows);
        std::map<long long, int> bl_id;
        for (int i = 0; i < p->n_prob; ++i) {
            const BProb &P = b->hprobs[i];
            for (int r = 0; r < P.n_rows; ++r) {
                const long long gr = P.row_off + r;
                row_vis[gr] = P.vis_off + (long long)r * P.n_chan;
                row_nc[gr] = P.n_chan;
                const long long key = ((long long)i * QC_BATCH_MAX_ANT + ants[gr].x) * QC_BATCH_MAX_ANT + ants[gr].y;
                auto it = bl_id.find(key);
                if (it == bl_id.end()) it = bl_id.emplace(key, (int)bl_id.size()).first;
                row_bl[gr] = it->second;
            }
        }
        long long *d_row_vis;
        int *d_row_nc, *d_row_bl;
        unsigned *bits;
        uint4 *m16;
        BALLOC(d_row_vis, long long, std::max<long long>(1, b->n_rows));
        BALLOC(d_row_nc, int, std::max<long long>(1, b->n_rows));
        BALLOC(d_row_bl, int, std::max<long long>(1, b->n_rows));
        BALLOC(bits, unsigned, std::max<size_t>(1, bl_id.size()));
        BALLOC(b->row_scale, float, std::max<long long>(1, b->n_rows));
        BALLOC(m16, uint4, nv);
        if (b->n_rows) {
            BH2D(d_row_vis, row_vis.data(), sizeof(long long) * b->n_rows);
            BH2D(d_row_nc, row_nc.data(), sizeof(int) * b->n_rows);
            BH2D(d_row_bl, row_bl.data(), sizeof(int) * b->n_rows);
        }
        e = cudaMemsetAsync(bits, 0, sizeof(unsigned) * std::max<size_t>(1, bl_id.size()), st);
        if (e == cudaSuccess && b->n_rows) {
            const int grid = (int)std::min<long long>(b->sm_count * 8LL, (b->n_rows + 255) / 256);
            row_scale_kernel<<<grid, 256, 0, st>>>(model32, b->ants, d_row_vis, d_row_nc, d_row_bl, b->n_rows, bits);
            row_scale_fill<<<grid, 256, 0, st>>>(d_row_bl, bits, b->n_rows, b->row_scale);
            pack16_rows_kernel<<<(int)std::min<long long>(b->sm_count * 8LL, b->n_rows), 64, 0, st>>>(
                model32, b->row_scale, d_row_vis, d_row_nc, b->n_rows, m16);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { g_batch_create_error = std::string("fp16 packing: ") + cudaGetErrorString(e); return QC_ECUDA; }
        b->model16 = m16;
        if (p->memory == QC_MEM_HOST) {
            auto it = std::find(b->owned.begin(), b->owned.end(), (void *)model32);
            if (it != b->owned.end()) { qc_dev_free(*it); b->owned.erase(it); }
        }
        model32 = nullptr;
    }
    b->model = model32;
    // schedules: longest problem first (samples), and index order
    std::vector<int> lpt(p->n_prob), idx(p->n_prob);
    std::iota(idx.begin(), idx.end(), 0);
    lpt = idx;
    std::stable_sort(lpt.begin(), lpt.end(), [&](int x, int y) {
        return (long long)b->hprobs[x].n_rows * b->hprobs[x].n_chan > (long long)b->hprobs[y].n_rows * b->hprobs[y].n_chan;
    });
    BALLOC(b->order_lpt, int, p->n_prob);
    BALLOC(b->order_idx, int, p->n_prob);
    BALLOC(b->queue, int, 2);                  // work counters of the two size classes
    b->lpt_samples.resize(p->n_prob);
    for (int i = 0; i < p->n_prob; ++i)
        b->lpt_samples[i] = (long long)b->hprobs[lpt[i]].n_rows * b->hprobs[lpt[i]].n_chan;
    BH2D(b->order_lpt, lpt.data(), sizeof(int) * p->n_prob);
    BH2D(b->order_idx, idx.data(), sizeof(int) * p->n_prob);
    BALLOC(b->gstage, unsigned char, (size_t)b->total_ant * 17 + sizeof(int) * p->n_prob + 64);
    // shape class of the batch for the tuning cache: problem count and log2 size histogram
    int hist[40] = { 0 };
    for (const BProb &P : b->hprobs) {
        const long long n = std::max(1LL, (long long)P.n_rows * P.n_chan);
        hist[std::min(39, 63 - __builtin_clzll((unsigned long long)n))]++;
    }
    b->shape_key = std::to_string(p->n_prob) + (b->m16 ? "h" : "f");
    for (int i = 0; i < 40; ++i) if (hist[i]) b->shape_key += ":" + std::to_string(i) + "x" + std::to_string(hist[i]);
#undef BALLOC
#undef BH2D
    *out = b.release();
    return QC_OK;
}

extern "C" void qc_batch_destroy(qc_batch *b) { delete b; }

extern "C" const char *qc_batch_last_error(const qc_batch *b)
{
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

static BatchArgs batch_args(qc_batch *b)
{
    BatchArgs a;
    memset(&a, 0, sizeof a);
    a.probs = b->probs;
    a.n_prob = b->n_prob;
    a.vis = b->vis;
    a.model = b->model;
    a.model16 = b->model16;
    a.row_scale = b->row_scale;
    a.weight = b->weight;
    a.flag = b->flag;
    a.ants = b->ants;
    a.max_ant = b->max_ant;
    a.vis_iters = b->counters;
    a.bytes = b->counters + 1;
    return a;
}

static size_t batch_smem(const qc_batch *b, int threads, int depth)
{
    const size_t ring = b->m16 ? (depth == 3 ? batch_ring_bytes_per_warp<true, 3>()
                                  : depth == 4 ? batch_ring_bytes_per_warp<true, 4>() : batch_ring_bytes_per_warp<true, 6>())
                               : (depth == 3 ? batch_ring_bytes_per_warp<false, 3>()
                                  : depth == 4 ? batch_ring_bytes_per_warp<false, 4>() : batch_ring_bytes_per_warp<false, 6>());
    return (size_t)(threads / 32) * ring +
           (size_t)b->max_ant * (2 * sizeof(double2) + sizeof(float4) + 6 * sizeof(float));
}

static const void *batch_fn(bool m16, int depth)
{
    if (m16) return depth == 3 ? (const void *)batch_kernel<true, 3>
                  : depth == 4 ? (const void *)batch_kernel<true, 4> : (const void *)batch_kernel<true, 6>;
    return depth == 3 ? (const void *)batch_kernel<false, 3>
         : depth == 4 ? (const void *)batch_kernel<false, 4> : (const void *)batch_kernel<false, 6>;
}

// Tuned launch shapes, per device and shape class (problem count and size histogram),
// shared by every batch of the process.
static std::mutex g_tune_mutex;
static std::map<std::string, qc_batch::Shape> g_tuned;

static std::string tune_key(const qc_batch *b) { return std::to_string(b->dev) + "/" + b->shape_key; }

static bool tuned_shape(const qc_batch *b, qc_batch::Shape &out)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(tune_key(b));
    if (it == g_tuned.end()) return false;
    out = it->second;
    return true;
}

// One class of problems for a launch: a slice of a schedule order and its work counter.
struct LaunchClass { const int *order; int n; int *queue; int threads, per_sm, depth, schedule, grid; };

// Enqueue one solve on stream st: the work counters' reset and the persistent kernel of each
// class; a second class runs on the auxiliary stream, forked from and joined into st.
static int batch_enqueue(qc_batch *b, const BatchArgs &base, const LaunchClass *cls, int n_cls, cudaStream_t st)
{
    BCK(cudaMemsetAsync(b->queue, 0, 2 * sizeof(int), st));
    if (n_cls > 1) {
        BCK(cudaEventRecord(b->ev_fork, st));
        BCK(cudaStreamWaitEvent(b->aux_stream, b->ev_fork, 0));
    }
    for (int c = 0; c < n_cls; ++c) {
        const LaunchClass &L = cls[c];
        if (L.n <= 0) continue;
        BatchArgs a = base;
        a.order = L.order;
        a.n_prob = L.n;
        a.queue = L.queue;
        a.schedule = L.schedule;
        const size_t smem = batch_smem(b, L.threads, L.depth);
        void *args[] = { (void *)&a };
        BCK(cudaLaunchKernel(batch_fn(b->m16, L.depth), dim3(L.grid), dim3(L.threads), args, smem,
                             c == 0 ? st : b->aux_stream));
    }
    if (n_cls > 1) {
        BCK(cudaEventRecord(b->ev_join, b->aux_stream));
        BCK(cudaStreamWaitEvent(st, b->ev_join, 0));
    }
    return QC_OK;
}

// Check one CTA shape and clamp its residency to what fits on an SM (the kernel's dynamic
// shared-memory limit is raised to the per-CTA maximum once, so shapes of both classes fit).
static int check_shape(qc_batch *b, int threads, int depth, int &per_sm)
{
    if (threads < 64 || threads > 512 || threads % 32) return b->fail(QC_EINVAL, "threads must be 64..512, multiple of 32");
    if (depth != 3 && depth != 4 && depth != 6) return b->fail(QC_EINVAL, "depth must be 3, 4 or 6");
    const size_t smem = batch_smem(b, threads, depth);
    int max_smem = 0;
    cudaError_t e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->dev);
    if (e != cudaSuccess) return b->cuda_fail(e, "cudaDeviceGetAttribute");
    const size_t static_smem = 2 * 32 * sizeof(double) + 64;
    if (smem + static_smem > (size_t)max_smem)
        return b->fail(QC_EUNSUPPORTED, "batch kernel shared memory exceeds the per-CTA limit for this shape");
    e = cudaFuncSetAttribute(batch_fn(b->m16, depth), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             max_smem - (int)static_smem);
    if (e != cudaSuccess) return b->cuda_fail(e, "cudaFuncSetAttribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_fn(b->m16, depth), threads, smem);
    if (e != cudaSuccess) return b->cuda_fail(e, "occupancy");
    if (occ < 1) return b->fail(QC_EUNSUPPORTED, "batch kernel does not fit on an SM with this shape");
    if (per_sm <= 0 || per_sm > occ) per_sm = std::min(occ, per_sm <= 0 ? occ : per_sm);
    return QC_OK;
}

static int launch_shape(qc_batch *b, const qc_batch_opts *o, qc_batch::Shape &sh)
{
    sh.threads = o->threads;
    sh.per_sm = o->ctas_per_sm;
    sh.schedule = o->schedule;
    sh.depth = o->depth;
    sh.split = o->split;
    sh.s_threads = o->small_threads;
    sh.s_per_sm = o->small_ctas_per_sm;
    qc_batch::Shape t;
    if (tuned_shape(b, t)) {
        if (sh.threads == 0) sh.threads = t.threads;
        if (sh.per_sm == 0) sh.per_sm = t.per_sm;
        if (sh.schedule == QC_SCHED_AUTO) sh.schedule = t.schedule;
        if (sh.depth == 0) sh.depth = t.depth;
        if (sh.split == 0) sh.split = t.split;
        if (sh.s_threads == 0) sh.s_threads = t.s_threads;
        if (sh.s_per_sm == 0) sh.s_per_sm = t.s_per_sm;
    }
    if (sh.threads == 0) sh.threads = 256;
    if (sh.depth == 0) sh.depth = 4;
    if (sh.schedule == QC_SCHED_AUTO) sh.schedule = QC_SCHED_LPT;
    if (sh.split < 0) sh.split = 0;
    if (sh.s_threads == 0) sh.s_threads = 64;
    int rc = check_shape(b, sh.threads, sh.depth, sh.per_sm);
    if (rc) return rc;
    if (sh.split > 0) {
        if (sh.schedule != QC_SCHED_LPT) return b->fail(QC_EINVAL, "a size split takes the LPT schedule");
        if ((rc = check_shape(b, sh.s_threads, sh.depth, sh.s_per_sm))) return rc;
    }
    return QC_OK;
}

static int batch_solve_impl(qc_batch *b, void *gains, int8_t *gain_flags, int32_t *iters, int32_t mem,
                            const qc_batch_opts *o, qc_batch_stats *stats, bool tuning)
{
    if (!gains) return b->fail(QC_EINVAL, "gains is NULL");
    if (mem != QC_MEM_HOST && mem != QC_MEM_DEVICE) return b->fail(QC_EINVAL, "mem must be QC_MEM_HOST or DEVICE");
    if (o->max_iter < 1) return b->fail(QC_EINVAL, "max_iter must be >= 1");
    if (!(o->tol >= 0)) return b->fail(QC_EINVAL, "tol must be >= 0");
    if ((o->fallback_gains == nullptr) != (o->fallback_chi2 == nullptr))
        return b->fail(QC_EINVAL, "fallback_gains and fallback_chi2 go together");
    if (o->fallback_gains && mem != QC_MEM_DEVICE) return b->fail(QC_EINVAL, "a fallback start needs device gains");
    if (o->damping_mode != QC_DAMP_CONST && o->damping_mode != QC_DAMP_ALTERNATE) return b->fail(QC_EINVAL, "damping_mode");
    qc_batch::Shape sh;
    int rc;
    if ((rc = launch_shape(b, o, sh))) return rc;
    const int threads = sh.threads, per_sm = sh.per_sm, schedule = sh.schedule, depth = sh.depth;
    cudaStream_t st = o->stream ? (cudaStream_t)o->stream : b->own_stream;
    // size classes: the LPT order is by non-increasing samples, so the problems with at least
    // `split` samples are its prefix and the small class its suffix
    int n_big = b->n_prob;
    if (sh.split > 0)
        n_big = (int)(std::lower_bound(b->lpt_samples.begin(), b->lpt_samples.end(), sh.split,
                                       [](long long v, long long x) { return v >= x; }) - b->lpt_samples.begin());
    LaunchClass cls[2];
    cls[0] = { schedule == QC_SCHED_STATIC ? b->order_idx : b->order_lpt, n_big, b->queue, threads, per_sm, depth,
               schedule, std::max(1, std::min(n_big, b->sm_count * per_sm)) };
    cls[1] = { b->order_lpt + n_big, b->n_prob - n_big, b->queue + 1, sh.s_threads, sh.s_per_sm, depth, QC_SCHED_LPT,
               std::max(1, std::min(b->n_prob - n_big, b->sm_count * std::max(1, sh.s_per_sm))) };
    const int n_cls = sh.split > 0 ? 2 : 1;
    const size_t gbytes = (size_t)b->total_ant * 2 * sizeof(float2);
    unsigned char *stage = (unsigned char *)b->gstage;
    float2 *dg = mem == QC_MEM_DEVICE ? (float2 *)gains : (float2 *)stage;
    int8_t *dflags = mem == QC_MEM_DEVICE ? gain_flags : (gain_flags ? (int8_t *)(stage + gbytes) : nullptr);
    int *diters = mem == QC_MEM_DEVICE ? iters
                                       : (iters ? (int *)(stage + gbytes + ((b->total_ant + 15) / 16) * 16) : nullptr);
    BatchArgs a = batch_args(b);
    a.gains = dg;
    a.gain_flags = dflags;
    a.iters = diters;
    a.max_iter = o->max_iter;
    a.damping_mode = o->damping_mode;
    a.damping = o->damping;
    a.tol = o->tol;
    a.fb_gains = (const float2 *)o->fallback_gains;
    a.fb_chi2 = o->fallback_chi2;
    a.n_fallback = b->counters + 2 + b->n_prob;
    const int grid = cls[0].grid;
    BCK(cudaEventRecord(b->ev0, st));
    if (mem == QC_MEM_HOST) BCK(cudaMemcpyAsync(dg, gains, gbytes, cudaMemcpyHostToDevice, st));
    BCK(cudaMemsetAsync(b->counters, 0, 2 * sizeof(unsigned long long), st));
    BCK(cudaMemsetAsync(b->counters + 2 + b->n_prob, 0, sizeof(unsigned long long), st));
    if (o->use_graph && !tuning) {
        qc_batch::GraphKey k;
        memset(&k, 0, sizeof k);
        k.threads = threads; k.per_sm = per_sm; k.schedule = schedule; k.depth = depth; k.max_iter = o->max_iter;
        k.damping_mode = o->damping_mode; k.damping = o->damping; k.tol = o->tol; k.m16 = b->m16;
        k.gains = dg; k.flags = dflags; k.iters = diters; k.st = st;
        k.fb_gains = o->fallback_gains; k.fb_chi2 = o->fallback_chi2;
        k.split = sh.split; k.s_threads = sh.s_threads; k.s_per_sm = sh.s_per_sm;
        const bool same = b->exec && memcmp(&k, &b->gkey, sizeof k) == 0;
        if (!same) {
            if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
            cudaGraph_t g = nullptr;
            BCK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            rc = batch_enqueue(b, a, cls, n_cls, st);
            cudaError_t e = cudaStreamEndCapture(st, &g);
            if (rc || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return rc ? rc : b->cuda_fail(e, "cudaStreamEndCapture");
            }
            e = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return b->cuda_fail(e, "cudaGraphInstantiate");
            b->gkey = k;
        }
        BCK(cudaGraphLaunch(b->exec, st));
    } else {
        if ((rc = batch_enqueue(b, a, cls, n_cls, st))) return rc;
    }
    if (mem == QC_MEM_HOST) {
        BCK(cudaMemcpyAsync(gains, dg, gbytes, cudaMemcpyDeviceToHost, st));
        if (gain_flags) BCK(cudaMemcpyAsync(gain_flags, dflags, (size_t)b->total_ant, cudaMemcpyDeviceToHost, st));
        if (iters) BCK(cudaMemcpyAsync(iters, diters, sizeof(int) * b->n_prob, cudaMemcpyDeviceToHost, st));
    }
    unsigned long long hc[2], hfb = 0;
    BCK(cudaMemcpyAsync(hc, b->counters, sizeof hc, cudaMemcpyDeviceToHost, st));
    BCK(cudaMemcpyAsync(&hfb, b->counters + 2 + b->n_prob, sizeof hfb, cudaMemcpyDeviceToHost, st));
    BCK(cudaEventRecord(b->ev1, st));
    BCK(cudaStreamSynchronize(st));
    float ms = 0;
    BCK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    if (stats) {
        qc_batch_stats S;
        memset(&S, 0, sizeof S);
        S.ms = ms;
        S.vis_iters = (int64_t)hc[0];
        S.bytes = (int64_t)hc[1];
        S.threads = threads;
        S.ctas_per_sm = per_sm;
        S.schedule = schedule;
        S.grid = grid;
        S.depth = depth;
        S.n_fallback = (int32_t)hfb;
        S.split = sh.split;
        S.small_threads = n_cls > 1 ? sh.s_threads : 0;
        S.small_ctas_per_sm = n_cls > 1 ? sh.s_per_sm : 0;
        S.small_grid = n_cls > 1 ? cls[1].grid : 0;
        S.n_small = n_cls > 1 ? cls[1].n : 0;
        double tot_vis = 0;
        for (const BProb &P : b->hprobs) tot_vis += (double)P.n_rows * P.n_chan;
        S.mean_iters = tot_vis > 0 ? (double)hc[0] / tot_vis : 0;
        if (iters) {
            int mx = 0;
            if (mem == QC_MEM_HOST) for (int i = 0; i < b->n_prob; ++i) mx = std::max(mx, iters[i]);
            S.n_iter_max = mx;
        }
        *stats = S;
    }
    return QC_OK;
}

extern "C" int qc_batch_solve(qc_batch *b, void *gains, int8_t *gain_flags, int32_t *iters, int32_t mem,
                              const qc_batch_opts *o, qc_batch_stats *stats)
{
    if (!b) return QC_EINVAL;
    b->err.clear();
    qc_batch_opts def;
    memset(&def, 0, sizeof def);
    def.max_iter = 20;
    def.tol = 1e-6;
    def.damping_mode = QC_DAMP_ALTERNATE;
    def.use_graph = 1;
    return batch_solve_impl(b, gains, gain_flags, iters, mem, o ? o : &def, stats, false);
}

extern "C" int qc_batch_solve_moments(qc_batch *b, void *gains, int8_t *gain_flags, int32_t *iters, int32_t mem,
                                      const qc_batch_opts *o, qc_batch_stats *stats)
{
    if (!b) return QC_EINVAL;
    b->err.clear();
    qc_batch_opts def;
    memset(&def, 0, sizeof def);
    def.max_iter = 20;
    def.tol = 1e-6;
    def.damping_mode = QC_DAMP_ALTERNATE;
    if (!o) o = &def;
    if (!gains) return b->fail(QC_EINVAL, "gains is NULL");
    if (mem != QC_MEM_HOST && mem != QC_MEM_DEVICE) return b->fail(QC_EINVAL, "mem must be QC_MEM_HOST or DEVICE");
    if (o->max_iter < 1) return b->fail(QC_EINVAL, "max_iter must be >= 1");
    if (!(o->tol >= 0)) return b->fail(QC_EINVAL, "tol must be >= 0");
    if (o->damping_mode != QC_DAMP_CONST && o->damping_mode != QC_DAMP_ALTERNATE) return b->fail(QC_EINVAL, "damping_mode");
    if (!o->fallback_gains != !o->fallback_chi2) return b->fail(QC_EINVAL, "fallback_gains and fallback_chi2: both or neither");
    if (b->max_ant > MOM_MAX_ANT) return b->fail(QC_EUNSUPPORTED, "the moments solve takes at most 64 antennas");
    cudaStream_t st = o->stream ? (cudaStream_t)o->stream : b->own_stream;
    const size_t gbytes = (size_t)b->total_ant * 2 * sizeof(float2);
    unsigned char *stage = (unsigned char *)b->gstage;
    float2 *dg = mem == QC_MEM_DEVICE ? (float2 *)gains : (float2 *)stage;
    int8_t *dflags = mem == QC_MEM_DEVICE ? gain_flags : (gain_flags ? (int8_t *)(stage + gbytes) : nullptr);
    int *diters = mem == QC_MEM_DEVICE ? iters
                                       : (iters ? (int *)(stage + gbytes + ((b->total_ant + 15) / 16) * 16) : nullptr);
    BatchArgs a = batch_args(b);
    a.order = b->order_lpt;
    a.gains = dg;
    a.gain_flags = dflags;
    a.iters = diters;
    a.max_iter = o->max_iter;
    a.damping_mode = o->damping_mode;
    a.damping = o->damping;
    a.tol = o->tol;
    a.fb_gains = (const float2 *)o->fallback_gains;
    a.fb_chi2 = o->fallback_chi2;
    a.n_fallback = b->counters + 2 + b->n_prob;
    const size_t smem = mom_smem_bytes(std::max(2, b->max_ant));
    const void *fn = b->m16 ? (const void *)batch_moments_kernel<true> : (const void *)batch_moments_kernel<false>;
    BCK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BCK(cudaEventRecord(b->ev0, st));
    if (mem == QC_MEM_HOST) BCK(cudaMemcpyAsync(dg, gains, gbytes, cudaMemcpyHostToDevice, st));
    BCK(cudaMemsetAsync(b->counters, 0, 2 * sizeof(unsigned long long), st));
    BCK(cudaMemsetAsync(b->counters + 2 + b->n_prob, 0, sizeof(unsigned long long), st));
    if (b->m16) batch_moments_kernel<true><<<b->n_prob, 256, smem, st>>>(a);
    else batch_moments_kernel<false><<<b->n_prob, 256, smem, st>>>(a);
    BCK(cudaGetLastError());
    if (mem == QC_MEM_HOST) {
        BCK(cudaMemcpyAsync(gains, dg, gbytes, cudaMemcpyDeviceToHost, st));
        if (gain_flags) BCK(cudaMemcpyAsync(gain_flags, dflags, (size_t)b->total_ant, cudaMemcpyDeviceToHost, st));
        if (iters) BCK(cudaMemcpyAsync(iters, diters, sizeof(int) * b->n_prob, cudaMemcpyDeviceToHost, st));
    }
    unsigned long long hc[2], hfb = 0;
    BCK(cudaMemcpyAsync(hc, b->counters, sizeof hc, cudaMemcpyDeviceToHost, st));
    BCK(cudaMemcpyAsync(&hfb, b->counters + 2 + b->n_prob, sizeof hfb, cudaMemcpyDeviceToHost, st));
    BCK(cudaEventRecord(b->ev1, st));
    BCK(cudaStreamSynchronize(st));
    float ms = 0;
    BCK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    if (stats) {
        qc_batch_stats S;
        memset(&S, 0, sizeof S);
        S.ms = ms;
        S.vis_iters = (int64_t)hc[0];
        S.bytes = (int64_t)hc[1];
        S.threads = 256;
        S.ctas_per_sm = 0;
        S.schedule = QC_SCHED_LPT;
        S.grid = b->n_prob;
        S.n_fallback = (int32_t)hfb;
        double tot_vis = 0;
        for (const BProb &Pp : b->hprobs) tot_vis += (double)Pp.n_rows * Pp.n_chan;
        S.mean_iters = tot_vis > 0 ? (double)hc[0] / tot_vis : 0;
        if (iters && mem == QC_MEM_HOST) {
            int mx = 0;
            for (int i = 0; i < b->n_prob; ++i) mx = std::max(mx, iters[i]);
            S.n_iter_max = mx;
        }
        *stats = S;
    }
    return QC_OK;
}

extern "C" int qc_batch_autotune(qc_batch *b, const qc_batch_opts *base, qc_batch_stats *best, int32_t *n_tried)
{
    if (!b || !base) return QC_EINVAL;
    b->err.clear();
    // unit gains on the device for every trial
    float2 *g;
    cudaError_t e = qc_dev_malloc((void **)&g, (size_t)b->total_ant * 2 * sizeof(float2));
    if (e != cudaSuccess) return b->cuda_fail(e, "cudaMalloc");
    std::vector<float2> unit((size_t)b->total_ant * 2, make_float2(1.f, 0.f));
    qc_batch::Shape win{ 0, 0, 0, 0, 1e30, 0, 0, 0 };
    int tried = 0, rc = QC_OK;
    qc_batch_stats ws;
    memset(&ws, 0, sizeof ws);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned.erase(tune_key(b));
    }
    auto trial = [&](qc_batch_opts o) -> int {
        o.use_graph = 0;
        e = cudaMemcpy(g, unit.data(), unit.size() * sizeof(float2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return b->cuda_fail(e, "cudaMemcpy");
        qc_batch_stats s;
        const int r = batch_solve_impl(b, g, nullptr, nullptr, QC_MEM_DEVICE, &o, &s, true);
        if (r == QC_EUNSUPPORTED || r == QC_EINVAL) return QC_OK;           // shape not launchable
        if (r) return r;
        ++tried;
        if (s.ctas_per_sm != o.ctas_per_sm) return QC_OK;                   // clamped: a duplicate
        if (o.split > 0 && s.small_ctas_per_sm != o.small_ctas_per_sm) return QC_OK;
        if (s.ms < win.ms) {
            win = { o.threads, o.ctas_per_sm, o.schedule, o.depth, s.ms, o.split > 0 ? o.split : 0,
                    o.split > 0 ? o.small_threads : 0, o.split > 0 ? o.small_ctas_per_sm : 0 };
            ws = s;
        }
        return QC_OK;
    };
    // stage 1: one class -- CTA size (the tile: threads consecutive samples per CTA step),
    // copy depth, residency and schedule
    for (int threads : { 128, 256, 512 })
        for (int depth : { 3, 4, 6 })
            for (int per_sm : { 1, 2, 4 })
                for (int sched : { QC_SCHED_LPT, QC_SCHED_STATIC }) {
                    if (rc) break;
                    qc_batch_opts o = *base;
                    o.threads = threads;
                    o.depth = depth;
                    o.ctas_per_sm = per_sm;
                    o.schedule = sched;
                    o.split = -1;
                    rc = trial(o);
                }
    // stage 2: with the best large-problem shape, a size split -- problems under the threshold
    // (samples) go to concurrent small CTAs, several per SM
    if (!rc && win.threads) {
        const qc_batch::Shape big = win;
        for (long long split : { 1LL << 10, 1LL << 12, 1LL << 14, 1LL << 16 })
            for (int sthreads : { 64, 128 })
                for (int sper : { 4, 8 }) {
                    if (rc) break;
                    qc_batch_opts o = *base;
                    o.threads = big.threads;
                    o.depth = big.depth;
                    o.ctas_per_sm = big.per_sm;
                    o.schedule = QC_SCHED_LPT;
                    o.split = split;
                    o.small_threads = sthreads;
                    o.small_ctas_per_sm = sper;
                    rc = trial(o);
                }
    }
    qc_dev_free(g);
    if (rc) return rc;
    if (!tried || win.threads == 0) return b->fail(QC_EUNSUPPORTED, "no launch shape could be timed");
    if (win.split == 0) win.split = -1;              // tuned: no split
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[tune_key(b)] = win;
    }
    if (best) *best = ws;
    if (n_tried) *n_tried = tried;
    return QC_OK;
}

extern "C" int qc_batch_residual(qc_batch *b, const void *gains, int32_t mem, double *chi2)
{
    if (!b) return QC_EINVAL;
    b->err.clear();
    if (!gains || !chi2) return b->fail(QC_EINVAL, "gains and chi2 are required");
    cudaStream_t st = b->own_stream;
    const size_t gbytes = (size_t)b->total_ant * 2 * sizeof(float2);
    float2 *dg = (float2 *)gains;
    double *dchi = chi2;
    void *tmp = nullptr;
    if (mem == QC_MEM_HOST) {
        BCK(qc_dev_malloc((void **)&tmp, gbytes + sizeof(double) * b->n_prob));
        dg = (float2 *)tmp;
        dchi = (double *)((unsigned char *)tmp + gbytes);
        BCK(cudaMemcpyAsync(dg, gains, gbytes, cudaMemcpyHostToDevice, st));
    }
    BatchArgs a = batch_args(b);
    a.gains = dg;
    if (b->m16) batch_chi2_kernel<true><<<b->n_prob, 256, 0, st>>>(a, dchi);
    else batch_chi2_kernel<false><<<b->n_prob, 256, 0, st>>>(a, dchi);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mem == QC_MEM_HOST)
        e = cudaMemcpyAsync(chi2, dchi, sizeof(double) * b->n_prob, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (tmp) qc_dev_free(tmp);
    if (e != cudaSuccess) return b->cuda_fail(e, "batch residual");
    return QC_OK;
}


extern "C" int qc_batch_features(qc_batch *b, const void *prev_gains, float *features, double *prev_chi2, int32_t mem,
                                 void *stream)
{
    if (!b) return QC_EINVAL;
    b->err.clear();
    if (!features) return b->fail(QC_EINVAL, "features is NULL");
    if (prev_chi2 && !prev_gains) return b->fail(QC_EINVAL, "prev_chi2 needs prev_gains");
    if (mem != QC_MEM_HOST && mem != QC_MEM_DEVICE) return b->fail(QC_EINVAL, "mem must be QC_MEM_HOST or DEVICE");
    cudaStream_t st = stream ? (cudaStream_t)stream : b->own_stream;
    const size_t gbytes = (size_t)b->total_ant * 2 * sizeof(float2), fbytes = (size_t)b->total_ant * 10 * sizeof(float);
    const size_t cbytes = sizeof(double) * b->n_prob;
    void *tmp = nullptr;
    const float2 *dprev = (const float2 *)prev_gains;
    float *dfeat = features;
    double *dchi = prev_chi2;
    if (mem == QC_MEM_HOST) {
        BCK(qc_dev_malloc((void **)&tmp, cbytes + fbytes + gbytes));
        dchi = prev_chi2 ? (double *)tmp : nullptr;
        dfeat = (float *)((unsigned char *)tmp + cbytes);
        if (prev_gains) {
            dprev = (const float2 *)((unsigned char *)tmp + cbytes + fbytes);
            BCK(cudaMemcpyAsync((void *)dprev, prev_gains, gbytes, cudaMemcpyHostToDevice, st));
        }
    }
    BatchArgs a = batch_args(b);
    const size_t smem = 8 * (b->m16 ? batch_ring_bytes_per_warp<true, FEAT_DEPTH>()
                                    : batch_ring_bytes_per_warp<false, FEAT_DEPTH>()) +
                        (size_t)b->max_ant * (sizeof(float4) + 9 * sizeof(float));
    const void *fn = b->m16 ? (const void *)batch_features_kernel<true> : (const void *)batch_features_kernel<false>;
    BCK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (b->m16) batch_features_kernel<true><<<b->n_prob, 256, smem, st>>>(a, dprev, dfeat, dchi);
    else batch_features_kernel<false><<<b->n_prob, 256, smem, st>>>(a, dprev, dfeat, dchi);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mem == QC_MEM_HOST) e = cudaMemcpyAsync(features, dfeat, fbytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && mem == QC_MEM_HOST && prev_chi2)
        e = cudaMemcpyAsync(prev_chi2, dchi, cbytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && mem == QC_MEM_HOST) e = cudaStreamSynchronize(st);
    if (tmp) { cudaStreamSynchronize(st); qc_dev_free(tmp); }
    if (e != cudaSuccess) return b->cuda_fail(e, "batch features");
    return QC_OK;
}

extern "C" int qc_batch_warmstart(qc_batch *b, const float *y, const void *fallback, int32_t check_chi2, void *gains_out,
                                  int32_t *n_fallback, void *stream)
{
    if (!b) return QC_EINVAL;
    b->err.clear();
    if (!y || !fallback || !gains_out) return b->fail(QC_EINVAL, "y, fallback and gains_out are required (device)");
    cudaStream_t st = stream ? (cudaStream_t)stream : b->own_stream;
    void *tmp = nullptr;
    BCK(qc_dev_malloc((void **)&tmp, sizeof(int) * b->n_prob + 2 * sizeof(double) * b->n_prob));
    int *bad = (int *)tmp;
    double *chi_p = (double *)((unsigned char *)tmp + ((sizeof(int) * b->n_prob + 15) / 16) * 16);
    double *chi_f = chi_p + b->n_prob;
    warm_gains_kernel<<<b->n_prob, 128, 0, st>>>(b->probs, b->n_prob, y, (const float2 *)fallback, (float2 *)gains_out, bad);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && check_chi2) {
        BatchArgs a = batch_args(b);
        a.gains = (float2 *)gains_out;
        if (b->m16) batch_chi2_kernel<true><<<b->n_prob, 256, 0, st>>>(a, chi_p);
        else batch_chi2_kernel<false><<<b->n_prob, 256, 0, st>>>(a, chi_p);
        a.gains = (float2 *)fallback;
        if (b->m16) batch_chi2_kernel<true><<<b->n_prob, 256, 0, st>>>(a, chi_f);
        else batch_chi2_kernel<false><<<b->n_prob, 256, 0, st>>>(a, chi_f);
        warm_select_kernel<<<b->n_prob, 128, 0, st>>>(b->probs, b->n_prob, chi_p, chi_f, (const float2 *)fallback,
                                                     (float2 *)gains_out, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n_fallback) {
        std::vector<int> hb(b->n_prob);
        e = cudaMemcpyAsync(hb.data(), bad, sizeof(int) * b->n_prob, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        int nf = 0;
        for (int v : hb) nf += v;
        *n_fallback = nf;
    }
    cudaStreamSynchronize(st);
    qc_dev_free(tmp);
    if (e != cudaSuccess) return b->cuda_fail(e, "batch warm start");
    return QC_OK;
}


extern "C" int qc_batch_reference_gains(qc_batch *b, const void *gains_in, void *gains_out, void *stream)
{
    if (!b) return QC_EINVAL;
    b->err.clear();
    if (!gains_in || !gains_out) return b->fail(QC_EINVAL, "gains_in and gains_out are required (device)");
    cudaStream_t st = stream ? (cudaStream_t)stream : b->own_stream;
    reference_gains_kernel<<<b->n_prob, 128, 0, st>>>(b->probs, b->n_prob, (const float2 *)gains_in, (float2 *)gains_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return b->cuda_fail(e, "reference gains");
    return QC_OK;
}
