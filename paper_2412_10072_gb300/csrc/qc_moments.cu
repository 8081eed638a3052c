// qc_moments.cu -- the solve of one term from per-(interval, antenna pair) sums (not in the paper).
//
// While one term of a chain is solved the others are fixed, so every sample of a baseline
// (p, q) in a solution interval enters J^H W J and J^H W r (Eq. jhj_entry_simplified,
// Eq. jhr_entry_simplified) through sums that do not depend on the solved gains.  The sums are
// kept per unordered pair p < q (a row with ant1 > ant2 enters through its conjugate baseline:
// D -> D^H, M -> M^H, the cross-hand weights swapped, p and q exchanged); kj = 2k + j indexes the
// weight and data of correlation (k, j).
//
// Full form: the solved term G (any kind) has no term to its left.  With X = R_p M R_q^H, R the
// term to its right (X = M when there is none), and u = 2l + m indexing X_lm:
//     S[kj][u][v] = sum w_kj conj(X_u) X_v,  T[kj][u] = sum w_kj conj(X_u) D_kj,
//     U[kj] = sum w_kj |D_kj|^2                                               (100 words)
//     JHJ_p[(k,l),(k,l')] += sum_j sum_m sum_m' G_q,jm conj(G_q,jm') S[kj][(l,m)][(l',m')]
//     b_p[(k,l)]          += sum_j sum_m G_q,jm T[kj][(l,m)]
//     JHJ_q[(k,l),(k,l')] += sum_j sum_m sum_m' G_p,jm conj(G_p,jm') conj(S[jk][(m,l)][(m',l')])
//     b_q[(k,l)]          += sum_j sum_m G_p,jm conj(T[jk][(m,l)])
// Diagonal form: the solved term g (diagonal or phase-only) has a term L to its left.  With
// E_kj,ab = L_p,ka M_ab conj(L_q,jb) and u = 2a + b:
//     S'[u][v] = sum sum_kj w_kj conj(E_kj,u) E_kj,v,  T'[u] = sum sum_kj w_kj conj(E_kj,u) D_kj,
//     U = sum sum_kj w_kj |D_kj|^2                                            (25 words)
//     JHJ_p[a][a'] += sum_b sum_b' g_q,b conj(g_q,b') S'[(a,b)][(a',b')],  b_p[a] += sum_b g_q,b T'[(a,b)]
//     JHJ_q[b][b'] += sum_a sum_a' g_p,a conj(g_p,a') conj(S'[(a,b)][(a',b')]),
//     b_q[b]       += sum_a g_p,a conj(T'[(a,b)])
// In both forms JHr = b - JHJ vec(g).  One pass over the data per term solve forms the sums in
// FP32 (mom_pass_kernel: per-lane register sums, added to the slots by FP32 atomics, a few per
// slot: a warp covers a whole row, or a whole strip of one chunk); every iteration forms each
// antenna's blocks from them and the current gains in FP32 (mom_normal_kernel), JHr = b - JHJ g
// and everything after it in FP64, in the update kernel's accumulator layout (a diagonal or
// phase-only term of the full form takes the (0, 3) rows and columns).  An iteration then reads
// 400 or 112 B per (interval, pair) instead of 81 B per sample.
#include "qc_internal.h"

#include <algorithm>
#include <type_traits>

namespace qc {

constexpr unsigned FULL_MASK = 0xffffffffu;

// (re, im) += conj(x) y, four fused multiply-adds
__device__ __forceinline__ void cacc_conj(float &re, float &im, float2 x, float2 y)
{
    re = fmaf(x.x, y.x, fmaf(x.y, y.y, re));
    im = fmaf(x.x, y.y, fmaf(-x.y, y.x, im));
}

// One sample's terms added to a lane's register sums, full form (one lane per sample; words as
// the slot: S[kj] at 16 kj, T[kj] at MOM_T + 8 kj, U[kj] at MOM_U + kj; all indices compile-time
// constants after unrolling; X = R_p M R_q^H).
__device__ __forceinline__ void mom_add(float (&acc)[MOM_N], const J2 &D, const J2 &X, float4 w)
{
    const float2 x[4] = { X.a, X.b, X.c, X.d };
    const float2 d[4] = { D.a, D.b, D.c, D.d };
    const float wv[4] = { w.x, w.y, w.z, w.w };
    float diag[4];
    float2 off[6];
#pragma unroll
    for (int u = 0; u < 4; ++u) diag[u] = cnorm2(x[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = u + 1; v < 4; ++v) off[mom_pair(u, v)] = cmulc(x[v], x[u]);   // conj(x_u) x_v
#pragma unroll
    for (int kj = 0; kj < 4; ++kj) {
        const int s = 16 * kj;
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[s + u] = fmaf(wv[kj], diag[u], acc[s + u]);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            acc[s + 4 + 2 * i] = fmaf(wv[kj], off[i].x, acc[s + 4 + 2 * i]);
            acc[s + 5 + 2 * i] = fmaf(wv[kj], off[i].y, acc[s + 5 + 2 * i]);
        }
        const float2 wd = cscale(d[kj], wv[kj]);
        const int t = MOM_T + 8 * kj;
#pragma unroll
        for (int u = 0; u < 4; ++u) cacc_conj(acc[t + 2 * u], acc[t + 2 * u + 1], x[u], wd);   // conj(x_u) w d
        acc[MOM_U + kj] = fmaf(wv[kj], cnorm2(d[kj]), acc[MOM_U + kj]);
    }
}

// The diagonal form, one lane per sample: register words [0, 16) S' packed as the full form's
// S blocks, [16, 24) T', 24 U.
constexpr int MOM_EW = 25;

template <int LK>
__device__ __forceinline__ void mom_add_e(float (&acc)[MOM_EW], const J2 &D, const J2 &M, const J2 &Lp,
                                          const J2 &Lq, float4 w)
{
    const float2 m[4] = { M.a, M.b, M.c, M.d };       // M_ab at 2a + b
    const float2 lp[4] = { Lp.a, Lp.b, Lp.c, Lp.d };  // L_p,ka at 2k + a
    const float2 lq[4] = { Lq.a, Lq.b, Lq.c, Lq.d };
    const float2 d[4] = { D.a, D.b, D.c, D.d };
    const float wv[4] = { w.x, w.y, w.z, w.w };
#pragma unroll
    for (int kj = 0; kj < 4; ++kj) {
        const int k = kj >> 1, j = kj & 1;
        if constexpr (LK == KIND_DIAG) {
            // E_kj,ab is non-zero only at (a, b) = (k, j): S' stays diagonal
            const float2 e = cmulc(cmul(lp[3 * k], m[kj]), lq[3 * j]);
            acc[kj] = fmaf(wv[kj], cnorm2(e), acc[kj]);
            cacc_conj(acc[16 + 2 * kj], acc[17 + 2 * kj], e, cscale(d[kj], wv[kj]));   // conj(e) w d
        } else {
            // sqrt(w) E_kj: S' += conj(e_u) e_v, T' += conj(e_u) sqrt(w) d
            const float sw = sqrtf(wv[kj]);
            float2 e[4];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const float2 l = cscale(lp[2 * k + a], sw);
#pragma unroll
                for (int b = 0; b < 2; ++b) e[2 * a + b] = cmul(l, cmulc(m[2 * a + b], lq[2 * j + b]));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(e[u].x, e[u].x, fmaf(e[u].y, e[u].y, acc[u]));
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = u + 1; v < 4; ++v)
                    cacc_conj(acc[4 + 2 * mom_pair(u, v)], acc[5 + 2 * mom_pair(u, v)], e[u], e[v]);
            const float2 ds = cscale(d[kj], sw);
#pragma unroll
            for (int u = 0; u < 4; ++u) cacc_conj(acc[16 + 2 * u], acc[17 + 2 * u], e[u], ds);
        }
        acc[24] = fmaf(wv[kj], cnorm2(d[kj]), acc[24]);
    }
}

// Add the warp's register sums (NW words, the slot's order) to the sums of each lane's key
// (-1: nothing) and zero them:
//  - one key for the warp: a reduce-scatter (words padded to P = a power of two; after the
//    halvings at lane offsets 16 .. 1 lane L holds words F L .. F L + F - 1, F = P / 32), then
//    one atomic per word;
//  - 32 distinct keys: each lane adds its own words;
//  - otherwise: a segmented reduction per word over the run of equal keys (channel intervals
//    are contiguous, so a run is a range of lanes), added by the run's first lane.
template <int NW>
__device__ __forceinline__ void mom_flush(float (&acc)[NW], int key, int lane, float *mom, int stride)
{
    constexpr int P = NW <= 32 ? 32 : (NW <= 64 ? 64 : 128);
    constexpr int F = P / 32;
    const int k0 = __shfl_sync(FULL_MASK, key, 0);
    if (__all_sync(FULL_MASK, key == k0)) {
        if (k0 >= 0) {
            // in place: after the halving at offset o the live words are acc[0 .. h)
#pragma unroll
            for (int h = P / 2, o = 16; o >= 1; h >>= 1, o >>= 1) {
                const bool up = (lane & o) != 0;
#pragma unroll
                for (int i = 0; i < h; ++i) {
                    const float lo = i < NW ? acc[i] : 0.f;
                    const float hi = i + h < NW ? acc[i + h] : 0.f;
                    const float send = up ? lo : hi;
                    const float keep = up ? hi : lo;
                    if (i < NW) acc[i] = keep + __shfl_xor_sync(FULL_MASK, send, o);
                }
            }
            float *dst = mom + (size_t)k0 * stride + F * lane;
#pragma unroll
            for (int j = 0; j < F; ++j)
                if (F * lane + j < NW) atomicAdd(dst + j, acc[j]);
        }
    } else {
        const unsigned m = __match_any_sync(FULL_MASK, key);
        if (__all_sync(FULL_MASK, m == (1u << lane))) {
            if (key >= 0) {
                float *dst = mom + (size_t)key * stride;
#pragma unroll
                for (int v = 0; v < NW; ++v) atomicAdd(dst + v, acc[v]);
            }
        } else {
            const int seg_end = 32 - __clz(m);
            const bool head = lane == __ffs(m) - 1;
            float *dst = mom + (size_t)(key >= 0 ? key : 0) * stride;
#pragma unroll
            for (int v = 0; v < NW; ++v) {
                float x = acc[v];
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const float o = __shfl_down_sync(FULL_MASK, x, d);
                    if (lane + d < seg_end) x += o;
                }
                if (head && key >= 0) atomicAdd(dst + v, x);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < NW; ++v) acc[v] = 0.f;
}

// The rows of the baseline strips in strip order, as the pass reads them: {row (-1: no usable
// sample), time, pair | conj << 31, p | q << 16} with (p, q) the baseline as the sums orient it.
static __global__ void mom_rows_kernel(long n, const int *strip_rows, const int4 *rows, const uint8_t *row_live,
                                       const int *up_of_bl, int4 *out)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int row = strip_rows[k];
    const int4 r = rows[row];
    const bool conj = r.x > r.y;
    const int p = conj ? r.y : r.x, q = conj ? r.x : r.y;
    out[k] = make_int4(row_live[row] ? row : -1, r.z, (int)((unsigned)up_of_bl[r.w] | (conj ? 0x80000000u : 0u)),
                       p | (q << 16));
}

template <int K>
__device__ __forceinline__ J2 fac_jones(const float4 *o)
{
    if constexpr (K == KIND_FULL) return j_from(o[0], o[1]);
    else if constexpr (K == KIND_DIAG) return j_diag(o[0]);
    else return j_identity();
}

// Shape of a warp's ring of the pass (one lane per sample, 32-channel chunks): per stage, in
// float4 units, the chunk's data quads d0 [0, 32), d1 [32, 64), model quads m0 [64, 96),
// m1 [96, 128), folded weights w [128, 160), then the fixed term's table entries for p and for
// q (NO float4 each, per channel, or only the first one when the chunk lies in one of the term's
// frequency intervals), the lanes' keys (32 ints) and one int4 of meta data.
template <int FORM, int OK> struct MomRing {
    static constexpr int NO = OK == KIND_FULL ? 2 : (OK == KIND_DIAG ? 1 : 0);
    static constexpr int OFF_OP = 160, OFF_OQ = OFF_OP + 32 * NO, OFF_KEY = OFF_OQ + 32 * NO;
    static constexpr int OFF_META = OFF_KEY + 8;
    static constexpr int STAGE = OFF_META + 1;               // float4 per stage
    // three CTAs of 4 warps per SM (the full form's 100 register sums fit 168 registers); ring
    // depth as the shared memory of three CTAs allows
    static constexpr int PER_SM = 3;
    static constexpr int DEPTH = NO == 2 ? 3 : (NO == 1 ? 4 : 6);
    static constexpr size_t SMEM = (size_t)4 * DEPTH * STAGE * sizeof(float4);
};

constexpr int MOM_END = 2;       // meta: the warp's steps have run out (bit 0: conjugate baseline)

// The issuing side of a warp: its steps in order, unit by unit (grid stride; a unit is a block
// of rb rows of one baseline strip x a group of chunks), each copied into a ring stage by
// cp.async (zero-filled past the last channel and for rows without usable data, whose weights
// then read 0).
template <int FORM, int OK> struct MomCursor {
    using R = MomRing<FORM, OK>;
    long unit, n_units, stride;
    int n_groups;
    int k0, k1, ch0, ch1, k, ch;
    bool cm;

    __device__ __forceinline__ void bounds(const MomArgs &a)
    {
        // the first unit from here on with rows (or none: unit >= n_units)
        for (; unit < n_units; unit += stride) {
            const int g = (int)(unit % n_groups);
            const long sr = unit / n_groups;
            const int s = (int)(sr / a.n_rb), b = (int)(sr % a.n_rb);
            ch0 = g * a.group;
            ch1 = min(a.n_chunks, ch0 + a.group);
            const int kb = __ldg(a.strip_off + s);
            k0 = kb + b * a.rb;
            k1 = min(__ldg(a.strip_off + s + 1), k0 + a.rb);
            if (k0 < k1) break;
        }
        k = k0;
        ch = ch0;
    }

    __device__ __forceinline__ void start(const MomArgs &a, long first, long step)
    {
        n_groups = (a.n_chunks + a.group - 1) / a.group;
        n_units = (long)a.n_strips * a.n_rb * n_groups;
        stride = step;
        unit = first;
        cm = a.chunk_major != 0;
        bounds(a);
    }

    __device__ __forceinline__ void advance(const MomArgs &a)
    {
        bool done;
        if (cm) { if (++k == k1) { k = k0; ++ch; } done = ch >= ch1; }
        else { if (++ch == ch1) { ch = ch0; ++k; } done = k >= k1; }
        if (done) {
            unit += stride;
            bounds(a);
        }
    }

    __device__ __forceinline__ void issue(const MomArgs &a, int lane, float4 *stage)
    {
        int meta = MOM_END;
        if (unit < n_units) {
            const int4 mr = __ldg(a.mrows + k);
            const int c0 = ch * 32, c = c0 + lane;
            const bool in = c < a.n_chan;
            const bool rd = mr.x >= 0 && in;
            meta = mr.z < 0 ? 1 : 0;
            const size_t i = rd ? (size_t)mr.x * a.n_chan + c : 0;
            const uint32_t nb = rd ? 16u : 0u;
            cp_async16(stage + lane, a.vis + 2 * i, nb);
            cp_async16(stage + 32 + lane, a.vis + 2 * i + 1, nb);
            cp_async16(stage + 64 + lane, a.model + 2 * i, nb);
            cp_async16(stage + 96 + lane, a.model + 2 * i + 1, nb);
            cp_async16(stage + 128 + lane, a.wf + i, nb);
            if constexpr (R::NO > 0) {
                const int ti = __ldg(a.to.t_map + mr.y);
                const int f_first = __ldg(a.to.f_map + c0);
                const int f_last = __ldg(a.to.f_map + min(a.n_chan, c0 + 32) - 1);
                const bool uni = f_first == f_last;       // f_map is non-decreasing
                if (uni) meta |= 4;
                const int pa = mr.w & 0xffff, qa = mr.w >> 16;
                if (uni) {
                    if (lane < 2 * R::NO) {
                        const int side = lane / R::NO, part = lane % R::NO;
                        const size_t idx = ((size_t)ti * a.n_ant + (side ? qa : pa)) * a.to.n_fint + f_first;
                        cp_async16(stage + (side ? R::OFF_OQ : R::OFF_OP) + part, a.to.tab + R::NO * idx + part,
                                   mr.x >= 0 ? 16u : 0u);
                    }
                } else {
                    const int fi = in ? __ldg(a.to.f_map + c) : 0;
                    const size_t ip = ((size_t)ti * a.n_ant + pa) * a.to.n_fint + fi;
                    const size_t iq = ((size_t)ti * a.n_ant + qa) * a.to.n_fint + fi;
#pragma unroll
                    for (int part = 0; part < R::NO; ++part) {
                        cp_async16(stage + R::OFF_OP + R::NO * lane + part, a.to.tab + R::NO * ip + part, nb);
                        cp_async16(stage + R::OFF_OQ + R::NO * lane + part, a.to.tab + R::NO * iq + part, nb);
                    }
                }
            }
            reinterpret_cast<int *>(stage + R::OFF_KEY)[lane] =
                in ? (__ldg(a.tn.t_map + mr.y) * a.tn.n_fint + __ldg(a.tn.f_map + c)) * a.n_up + (mr.z & 0x7fffffff)
                   : -1;
        }
        if (lane == 0) reinterpret_cast<int *>(stage + R::OFF_META)[0] = meta;
        cp_async_commit();
        if (unit < n_units) advance(a);
    }
};

// One pass: warps walk units of a baseline strip (the rows of one ordered baseline in time
// order): blocks of rb rows x groups of 32-channel chunks, a row's chunks inside each row or,
// with chunk_major, the rows inside each chunk (an interval several times long then keeps its
// keys).  Each warp streams its steps through a ring of DEPTH cp.async stages in shared memory,
// DEPTH - 1 steps ahead of the arithmetic, which adds each lane's sample to its register sums;
// the sums are flushed when any lane's (interval, pair) key changes.  The fixed term is L
// (diagonal form) or R (full form) of kind OK.
template <int FORM, int OK>
static __global__ void __launch_bounds__(128, MomRing<FORM, OK>::PER_SM) mom_pass_kernel(const MomArgs a)
{
    using R = MomRing<FORM, OK>;
    constexpr int NW = FORM == FORM_FULL ? MOM_N : MOM_EW;
    if (__ldg(a.n_active) == 0) return;
    extern __shared__ float4 mom_ring[];
    const int lane = threadIdx.x & 31;
    float4 *ring = mom_ring + (size_t)(threadIdx.x >> 5) * R::DEPTH * R::STAGE;
    const int stride = FORM == FORM_FULL ? MOM_N : MOM_E;
    float acc[NW];
#pragma unroll
    for (int v = 0; v < NW; ++v) acc[v] = 0.f;
    MomCursor<FORM, OK> cur;
    cur.start(a, ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5, ((long)gridDim.x * blockDim.x) >> 5);
    int is = 0;
#pragma unroll
    for (int d = 0; d < R::DEPTH - 1; ++d) {
        cur.issue(a, lane, ring + (size_t)is * R::STAGE);
        if (++is == R::DEPTH) is = 0;
    }
    auto add = [&](const float4 *st, int meta) {
        float4 w = st[128 + lane];
        if (w.x != 0.f || w.y != 0.f || w.z != 0.f || w.w != 0.f) {
            J2 D = j_from(st[lane], st[32 + lane]), M = j_from(st[64 + lane], st[96 + lane]);
            if (meta & 1) {                    // the conjugate baseline: D -> D^H, M -> M^H, w permuted
                D = j_herm(D);
                M = j_herm(M);
                w = make_float4(w.x, w.z, w.y, w.w);
            }
            const int oc = (meta & 4) ? 0 : lane * R::NO;
            if constexpr (FORM == FORM_FULL) {
                if constexpr (OK == KIND_DIAG) {
                    const float4 rp = st[R::OFF_OP + oc], rq = st[R::OFF_OQ + oc];
                    M = j_muld(j_dmul(make_float2(rp.x, rp.y), make_float2(rp.z, rp.w), M),
                               make_float2(rq.x, -rq.y), make_float2(rq.z, -rq.w));
                } else if constexpr (OK == KIND_FULL) {
                    M = j_mul_h(j_mul(fac_jones<OK>(st + R::OFF_OP + oc), M), fac_jones<OK>(st + R::OFF_OQ + oc));
                }
                mom_add(acc, D, M, w);
            } else {
                mom_add_e<OK>(acc, D, M, fac_jones<OK>(st + R::OFF_OP + oc), fac_jones<OK>(st + R::OFF_OQ + oc), w);
            }
        }
    };
    // runs of steps with unchanged keys: the inner loop only adds; a key change leaves it to
    // flush the sums, then adds the step that changed the key
    int key_cur = -1, stage = 0;
    bool done = false;
    for (;;) {
        const float4 *st;
        int meta = 0, key = -1;
        for (;;) {
            __syncwarp();                      // every lane is done with the stage about to be refilled
            cur.issue(a, lane, ring + (size_t)is * R::STAGE);
            if (++is == R::DEPTH) is = 0;
            cp_async_wait<R::DEPTH - 1>();
            __syncwarp();
            st = ring + (size_t)stage * R::STAGE;
            meta = reinterpret_cast<const int *>(st + R::OFF_META)[0];
            if (meta & MOM_END) { done = true; break; }
            key = reinterpret_cast<const int *>(st + R::OFF_KEY)[lane];
            if (__any_sync(FULL_MASK, key != key_cur)) break;
            add(st, meta);
            if (++stage == R::DEPTH) stage = 0;
        }
        mom_flush<NW>(acc, key_cur, lane, a.mom, stride);
        if (done) break;
        key_cur = key;
        add(st, meta);
        if (++stage == R::DEPTH) stage = 0;
    }
    cp_async_wait<0>();
}

// gains of an antenna in a bin as complex FP64 entries (row-major; phase-only: diag(e^{i phi}))
__device__ __forceinline__ void gains_of(const MomNormArgs &A, int bin, int ant, double2 G[4])
{
    const size_t pidx = (size_t)bin * A.n_ant + ant;
    if (A.type == QC_TERM_PHASE) {
        double sn, cs;
        sincos(A.params[2 * pidx], &sn, &cs);
        G[0] = make_double2(cs, sn);
        sincos(A.params[2 * pidx + 1], &sn, &cs);
        G[3] = make_double2(cs, sn);
        G[1] = G[2] = make_double2(0.0, 0.0);
    } else {
        const double2 *P = reinterpret_cast<const double2 *>(A.params) + 4 * pidx;
#pragma unroll
        for (int e = 0; e < 4; ++e) G[e] = P[e];
    }
}

__device__ __forceinline__ float2 f2(double2 a) { return make_float2((float)a.x, (float)a.y); }

// a slot's words held in registers (loaded as 16-byte or 8-byte vectors); word i of the slot
template <int NV> struct SlotRegs {
    float4 v[NV];
    __device__ __forceinline__ float at(int i) const
    {
        const float4 &x = v[i >> 2];
        const int c = i & 3;
        return c == 0 ? x.x : c == 1 ? x.y : c == 2 ? x.z : x.w;
    }
    // element (u, v) of the Hermitian S block at word `base` (u, v compile-time after unrolling)
    __device__ __forceinline__ float2 S(int base, int u, int v) const
    {
        if (u == v) return make_float2(at(base + u), 0.f);
        const int i = base + 4 + 2 * (u < v ? mom_pair(u, v) : mom_pair(v, u));
        return u < v ? make_float2(at(i), at(i + 1)) : make_float2(at(i), -at(i + 1));
    }
    __device__ __forceinline__ float2 C(int i) const { return make_float2(at(i), at(i + 1)); }
};

// the other antenna's gains from the solved term's FP32 table (the update kernel writes it with
// every update): row-major entries, a diagonal or phase-only term as diag(g_0, g_1)
__device__ __forceinline__ void gains_f32(const MomNormArgs &A, int bin, int ant, float2 G[4])
{
    const int tint = bin / A.n_fint, fint = bin - tint * A.n_fint;
    const size_t idx = ((size_t)tint * A.n_ant + ant) * A.n_fint + fint;
    if (A.type == QC_TERM_FULL) {
        const float4 lo = __ldg(A.tab + 2 * idx), hi = __ldg(A.tab + 2 * idx + 1);
        G[0] = make_float2(lo.x, lo.y); G[1] = make_float2(lo.z, lo.w);
        G[2] = make_float2(hi.x, hi.y); G[3] = make_float2(hi.z, hi.w);
    } else {
        const float4 d = __ldg(A.tab + idx);
        G[0] = make_float2(d.x, d.y); G[3] = make_float2(d.z, d.w);
        G[1] = G[2] = make_float2(0.f, 0.f);
    }
}

// One warp per (interval, antenna a): lanes take the other antennas o, form the contributions
// of the pair (a, o) to a's block-diagonal J^H W J (the 2x2 blocks k = 0, 1 on rows
// (k, l), l = 0, 1) and to b, in FP32; a warp reduction sums them; lane 0 forms
// JHr = b - JHJ vec(G_a) in FP64 and writes the update kernel's accumulator layout.
static __global__ void __launch_bounds__(128) mom_normal_kernel(const MomNormArgs A)
{
    if (__ldg(A.n_active) == 0) return;
    const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (long)A.n_bins * A.n_ant) return;
    const int lane = threadIdx.x & 31;
    const int bin = (int)(w / A.n_ant), a = (int)(w % A.n_ant);
    if (!A.active[bin]) return;
    // h[k][0] = H[(k,0),(k,0)], h[k][1] = H[(k,0),(k,1)], h[k][2] = H[(k,1),(k,1)]; b[(k,l)]
    float2 h[2][3], b[4];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) h[k][i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = make_float2(0.f, 0.f);
    for (int o = lane; o < A.n_ant; o += 32) {
        if (o == a) continue;
        const int up = __ldg(A.upair + (size_t)a * A.n_ant + o);
        if (up < 0) continue;
        SlotRegs<MOM_N / 4> sl;
        const float4 *Mo = reinterpret_cast<const float4 *>(A.mom + ((size_t)bin * A.n_up + up) * MOM_N);
#pragma unroll
        for (int i = 0; i < MOM_N / 4; ++i) sl.v[i] = __ldg(Mo + i);
        float2 G[4];
        gains_f32(A, bin, o, G);
        const bool p_side = a < o;           // the sums are oriented with the smaller index first
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            // gg[m][m2] = G_jm conj(G_jm2)
            float2 gg[2][2];
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int m2 = 0; m2 < 2; ++m2) gg[m][m2] = cmulc(G[2 * j + m], G[2 * j + m2]);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int kp = 2 * k + j, kq = 2 * j + k;      // the slot block for the p and the q side
#pragma unroll
                for (int l = 0; l < 2; ++l)
#pragma unroll
                    for (int l2 = l; l2 < 2; ++l2) {
                        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int m = 0; m < 2; ++m)
#pragma unroll
                            for (int m2 = 0; m2 < 2; ++m2) {
                                // p side: S[kj][(l,m)][(l2,m2)]; q side: conj(S[jk][(m,l)][(m2,l2)])
                                const float2 sv = p_side ? sl.S(16 * kp, 2 * l + m, 2 * l2 + m2)
                                                         : cconj(sl.S(16 * kq, 2 * m + l, 2 * m2 + l2));
                                const float2 t = cmul(gg[m][m2], sv);
                                acc.x += t.x;
                                acc.y += t.y;
                            }
                        float2 &hh = h[k][l + l2];
                        hh.x += acc.x;
                        hh.y += acc.y;
                    }
#pragma unroll
                for (int l = 0; l < 2; ++l)
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const float2 tv = p_side ? sl.C(MOM_T + 8 * kp + 2 * (2 * l + m))
                                                 : cconj(sl.C(MOM_T + 8 * kq + 2 * (2 * m + l)));
                        const float2 t = cmul(G[2 * j + m], tv);
                        b[2 * k + l].x += t.x;
                        b[2 * k + l].y += t.y;
                    }
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                h[k][i].x += __shfl_xor_sync(FULL_MASK, h[k][i].x, d);
                h[k][i].y += __shfl_xor_sync(FULL_MASK, h[k][i].y, d);
            }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            b[i].x += __shfl_xor_sync(FULL_MASK, b[i].x, d);
            b[i].y += __shfl_xor_sync(FULL_MASK, b[i].y, d);
        }
    }
    if (lane != 0) return;
    // the full 4x4 (zero between the k blocks) in FP64, JHr = b - H g
    double2 H[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) H[i][j] = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        H[2 * k][2 * k] = make_double2(h[k][0].x, 0.0);
        H[2 * k][2 * k + 1] = make_double2(h[k][1].x, h[k][1].y);
        H[2 * k + 1][2 * k] = make_double2(h[k][1].x, -(double)h[k][1].y);
        H[2 * k + 1][2 * k + 1] = make_double2(h[k][2].x, 0.0);
    }
    double2 G[4];
    gains_of(A, bin, a, G);
    double2 r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double2 s = make_double2(b[i].x, b[i].y);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s.x -= H[i][j].x * G[j].x - H[i][j].y * G[j].y;
            s.y -= H[i][j].x * G[j].y + H[i][j].y * G[j].x;
        }
        r[i] = s;
    }
    double *out = A.acc + ((size_t)bin * A.n_ant + a) * (A.type == QC_TERM_FULL ? KG_FULL : KG_DIAG);
    if (A.type == QC_TERM_FULL) {
#pragma unroll
        for (int u = 0; u < 4; ++u) out[u] = H[u][u].x;
        int o = 4;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = u + 1; v < 4; ++v) { out[o] = H[u][v].x; out[o + 1] = H[u][v].y; o += 2; }
#pragma unroll
        for (int u = 0; u < 4; ++u) { out[16 + 2 * u] = r[u].x; out[17 + 2 * u] = r[u].y; }
    } else {
        out[0] = H[0][0].x;
        out[1] = H[3][3].x;
        out[2] = H[0][3].x;
        out[3] = H[0][3].y;
        out[4] = r[0].x; out[5] = r[0].y;
        out[6] = r[3].x; out[7] = r[3].y;
    }
}

// Diagonal form: one warp per (interval, antenna a); lanes take the other antennas o and form
// the pair's contributions to a's 2x2 block and right-hand side in FP32 (p side when a < o, q
// side otherwise); a warp reduction sums them; lane 0 forms JHr = b - JHJ g in FP64 and writes
// the update kernel's diagonal accumulator layout.
static __global__ void __launch_bounds__(128) mom_normal_e_kernel(const MomNormArgs A)
{
    if (__ldg(A.n_active) == 0) return;
    const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (long)A.n_bins * A.n_ant) return;
    const int lane = threadIdx.x & 31;
    const int bin = (int)(w / A.n_ant), a = (int)(w % A.n_ant);
    if (!A.active[bin]) return;
    float h00 = 0.f, h11 = 0.f;
    float2 h01 = make_float2(0.f, 0.f), b0 = h01, b1 = h01;
    for (int o = lane; o < A.n_ant; o += 32) {
        if (o == a) continue;
        const int up = __ldg(A.upair + (size_t)a * A.n_ant + o);
        if (up < 0) continue;
        SlotRegs<MOM_E / 4> sl;
        const float4 *Mo = reinterpret_cast<const float4 *>(A.mom + ((size_t)bin * A.n_up + up) * MOM_E);
#pragma unroll
        for (int i = 0; i < MOM_E / 4; ++i) sl.v[i] = __ldg(Mo + i);
        float2 Go[4];
        gains_f32(A, bin, o, Go);
        const float2 g[2] = { Go[0], Go[3] };
        const bool p_side = a < o;
        // the slot's S' entry for this antenna's parameters (x, x') and the other's (y, y'):
        // p side S'[(x,y)][(x',y')] with the other's gains g_y conj(g_y'); q side
        // conj(S'[(y,x)][(y',x')]) with the same weights
        float2 hh[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) hh[i] = make_float2(0.f, 0.f);
        float2 bb[2] = { make_float2(0.f, 0.f), make_float2(0.f, 0.f) };
#pragma unroll
        for (int x = 0; x < 2; ++x) {
#pragma unroll
            for (int x2 = x; x2 < 2; ++x2)
#pragma unroll
                for (int y = 0; y < 2; ++y)
#pragma unroll
                    for (int y2 = 0; y2 < 2; ++y2) {
                        const float2 gg = cmulc(g[y], g[y2]);
                        const float2 sv = p_side ? sl.S(0, 2 * x + y, 2 * x2 + y2)
                                                 : cconj(sl.S(0, 2 * y + x, 2 * y2 + x2));
                        const float2 t = cmul(gg, sv);
                        hh[x + x2].x += t.x;
                        hh[x + x2].y += t.y;
                    }
#pragma unroll
            for (int y = 0; y < 2; ++y) {
                const float2 tf = p_side ? sl.C(MOM_ET + 2 * (2 * x + y)) : cconj(sl.C(MOM_ET + 2 * (2 * y + x)));
                const float2 t = cmul(g[y], tf);
                bb[x].x += t.x;
                bb[x].y += t.y;
            }
        }
        h00 += hh[0].x;
        h01.x += hh[1].x;
        h01.y += hh[1].y;
        h11 += hh[2].x;
        b0.x += bb[0].x; b0.y += bb[0].y;
        b1.x += bb[1].x; b1.y += bb[1].y;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        h00 += __shfl_xor_sync(FULL_MASK, h00, d);
        h11 += __shfl_xor_sync(FULL_MASK, h11, d);
        h01.x += __shfl_xor_sync(FULL_MASK, h01.x, d);
        h01.y += __shfl_xor_sync(FULL_MASK, h01.y, d);
        b0.x += __shfl_xor_sync(FULL_MASK, b0.x, d);
        b0.y += __shfl_xor_sync(FULL_MASK, b0.y, d);
        b1.x += __shfl_xor_sync(FULL_MASK, b1.x, d);
        b1.y += __shfl_xor_sync(FULL_MASK, b1.y, d);
    }
    if (lane != 0) return;
    double2 G[4];
    gains_of(A, bin, a, G);
    // JHr = b - H g, H = [[h00, h01], [conj(h01), h11]] on (g_0, g_1) = (G[0], G[3])
    const double r0x = (double)b0.x - (h00 * G[0].x + (h01.x * G[3].x - h01.y * G[3].y));
    const double r0y = (double)b0.y - (h00 * G[0].y + (h01.x * G[3].y + h01.y * G[3].x));
    const double r1x = (double)b1.x - ((h01.x * G[0].x + h01.y * G[0].y) + h11 * G[3].x);
    const double r1y = (double)b1.y - ((h01.x * G[0].y - h01.y * G[0].x) + h11 * G[3].y);
    double *out = A.acc + ((size_t)bin * A.n_ant + a) * KG_DIAG;
    out[0] = h00;
    out[1] = h11;
    out[2] = h01.x;
    out[3] = h01.y;
    out[4] = r0x; out[5] = r0y;
    out[6] = r1x; out[7] = r1y;
}

// algorithmic bytes: the pass reads every sample of the bins once (their streaming bytes);
// an iteration reads each bin's sums twice (once per side) and writes its accumulators
static __global__ void mom_bytes_kernel(int n_bins, const long long *bin_nbytes, long long per_iter,
                                        long long *iter_nbytes, unsigned long long *acc_bytes)
{
    unsigned long long s = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_bins; b += gridDim.x * blockDim.x) {
        s += (unsigned long long)bin_nbytes[b];
        iter_nbytes[b] = per_iter;
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(acc_bytes, s);
}

} // namespace qc

// the pass kernel of a form and fixed-term kind (ok: KIND_* of R in the full form, of L in the
// diagonal form; the diagonal form needs one)
template <int FORM, int OK>
static cudaError_t launch_pass(const qc::MomArgs &a, int sm_count, cudaStream_t st)
{
    using R = qc::MomRing<FORM, OK>;
    static bool configured = false;              // the raised shared-memory limit, once per process
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute(qc::mom_pass_kernel<FORM, OK>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int block = 128;
    const int n_groups = (a.n_chunks + a.group - 1) / a.group;
    const long units = (long)a.n_strips * a.n_rb * n_groups;
    const int grid = (int)std::max(1L, std::min((long)sm_count * R::PER_SM, (units * 32 + block - 1) / block));
    qc::mom_pass_kernel<FORM, OK><<<grid, block, R::SMEM, st>>>(a);
    return cudaGetLastError();
}

// the pass kernel of a form and fixed-term kind (ok: KIND_* of R in the full form, of L in the
// diagonal form; the diagonal form needs one)
cudaError_t mom_launch_pass(const qc::MomArgs &a, int form, int ok, int sm_count, cudaStream_t st)
{
    using namespace qc;
    if (form == FORM_FULL) {
        if (ok == KIND_NONE) return launch_pass<FORM_FULL, KIND_NONE>(a, sm_count, st);
        if (ok == KIND_DIAG) return launch_pass<FORM_FULL, KIND_DIAG>(a, sm_count, st);
        return launch_pass<FORM_FULL, KIND_FULL>(a, sm_count, st);
    }
    if (ok == KIND_DIAG) return launch_pass<FORM_E, KIND_DIAG>(a, sm_count, st);
    if (ok == KIND_FULL) return launch_pass<FORM_E, KIND_FULL>(a, sm_count, st);
    return cudaErrorInvalidValue;
}

cudaError_t mom_launch_bytes(int n_bins, const long long *bin_nbytes, long long per_iter, long long *iter_nbytes,
                             unsigned long long *acc_bytes, cudaStream_t st)
{
    qc::mom_bytes_kernel<<<(n_bins + 255) / 256, 256, 0, st>>>(n_bins, bin_nbytes, per_iter, iter_nbytes, acc_bytes);
    return cudaGetLastError();
}

cudaError_t mom_launch_normal(const qc::MomNormArgs &a, cudaStream_t st)
{
    const long warps = (long)a.n_bins * a.n_ant;
    if (a.form == qc::FORM_FULL) qc::mom_normal_kernel<<<(int)((warps + 3) / 4), 128, 0, st>>>(a);
    else qc::mom_normal_e_kernel<<<(int)((warps + 3) / 4), 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t mom_launch_rows(long n, const int *strip_rows, const int4 *rows, const uint8_t *row_live,
                            const int *up_of_bl, int4 *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    qc::mom_rows_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(n, strip_rows, rows, row_live, up_of_bl, out);
    return cudaGetLastError();
}

size_t mom_words(int form) { return form == qc::FORM_FULL ? qc::MOM_N : qc::MOM_E; }
