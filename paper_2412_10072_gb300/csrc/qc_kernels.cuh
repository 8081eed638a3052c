// qc_kernels.cuh -- device side of the per-interval approximate Gauss-Newton solve.
//
// One iteration of Algorithm 1 (arxiv 2412.10072, Section 4.3) for term n of
// a Jones chain is two kernels:
//   acc_kernel     one pass over the data: forms the corrected-model residual
//                  r = D - L_p G_p (R_p M C_q^H) of every sample on the fly and
//                  accumulates the per-(interval, antenna) blocks of J^H W J and
//                  J^H W r for both antennas of the baseline (the q side through
//                  the conjugate baseline), Eq. jhj_entry_simplified and
//                  Eq. jhr_entry_simplified.  Nothing visibility-sized is
//                  written (Section 4.3: no visibility-sized intermediaries;
//                  JHJ and JHr evaluated in tandem).
//   update_kernel  per (interval, antenna) FP64 block solve and update
//                  g <- g + alpha JHJ^{-1} JHr (Eq. update, Algorithm 1), the
//                  FP64 relative-change norm of each interval and its
//                  convergence flag.
//
// Work decomposition of acc_kernel: one warp owns a tile of 32 consecutive
// channels (lane = channel, so every 128-bit load of a warp is contiguous)
// and walks either along the channels of one row ("row tiles", order 0) or
// along the rows of one baseline in time order ("strip tiles", order 1).
// Each lane keeps its partial block sums in registers while its sample's
// interval bin stays the same; when any lane's bin changes the warp does a
// segmented shuffle reduction over lanes with equal bins and the segment
// heads add the sums into FP64 accumulators in global memory.  The host
// picks the order that makes these flushes rare for the term's interval
// shape (row tiles for intervals wide in frequency, strip tiles for
// intervals long in time).
#pragma once
#include <stdint.h>

#include "qc_async.cuh"
#include "qc_jones.cuh"

namespace qc {

constexpr int MAXT = 4;
constexpr int KIND_NONE = 0, KIND_DIAG = 1, KIND_FULL = 2;
constexpr int TS_DIAG = 0, TS_FULL = 1;       // accumulator family of the solved term
constexpr int KG_DIAG = 8, KG_FULL = 24;      // FP64 accumulator words per (bin, antenna)

// Global accumulator layout per (bin, antenna):
//   FULL (4 parameters u = 0..3, row-major g entries):
//     [0..3]   JHJ[u][u] (real)
//     [4..15]  JHJ[u][v] u<v as (re, im) for (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
//     [16..23] JHr[u] as (re, im)
//   DIAG (2 parameters g_XX, g_YY; phase-only terms use it too):
//     [0,1] JHJ[0][0], JHJ[1][1];  [2,3] JHJ[0][1];  [4..7] JHr[0], JHr[1]

struct DevTerm {
    int type;              // QC_TERM_* of the public API (0 diag, 1 full, 2 phase)
    int n_tint, n_fint;
    const int *t_map;      // [n_time]
    const int *f_map;      // [n_chan]
    const float4 *tab;     // [n_tint][n_ant][n_fint] x (type == full ? 2 : 1) float4
};

struct Chain {
    int n_terms;
    int n;                 // index of the solved term (-1: none)
    int n_ant;
    DevTerm t[MAXT];
};

struct Data {
    int n_row, n_chan;
    const float4 *vis;     // [n_row][n_chan] x 2 float4 (complex64 x 4)
    const float4 *model;   // same, or nullptr when model16 is used
    const uint4 *model16;  // [n_row][n_chan] x (4 half2), or nullptr
    const float *bl_scale; // [n_bl] per-baseline model scale (model16 only)
    const float4 *weight;  // [n_row][n_chan]
    const uint8_t *flag;   // [n_row][n_chan] or nullptr
    const int4 *rows;      // [n_row] {ant1, ant2, time, baseline id}
    const int *strip_rows; // rows grouped by (ant1, ant2), time order
    const int *strip_off;  // [n_strips + 1]
    int n_strips;
};

struct AccArgs {
    Data D;
    Chain C;
    DevTerm tn;              // copy of C.t[C.n] (avoids dynamic indexing of kernel parameters)
    DevTerm to;              // the other term of a two-term chain (unused otherwise)
    const uint8_t *row_live; // [n_row] 1: cross-correlation row with an unflagged sample
    const int4 *row_info;    // [n_row] {p, q, tn, to}, tn = -1 for rows without usable data
    const uint8_t *chunk_active;  // [n_tint of term n][n_chunks]: a 32-channel chunk has an active bin
    double *acc;             // [n_bins][n_ant][KG]
    const uint8_t *active;   // [n_bins]
    const int *n_active;     // nonzero: some interval of the solved term is still iterating
    int order;               // 0 row tiles, 1 strip tiles
    int n_chunks;            // ceil(n_chan / 32)
};

__device__ __forceinline__ J2 fetch_jones(const DevTerm &T, int n_ant, int tint, int fint, int ant)
{
    const size_t idx = ((size_t)tint * n_ant + ant) * T.n_fint + fint;
    if (T.type == 1) return j_from(__ldg(T.tab + 2 * idx), __ldg(T.tab + 2 * idx + 1));
    return j_diag(__ldg(T.tab + idx));
}

// Jones matrix of a term whose kind is known at compile time (diag/phase tables hold
// the two diagonal entries in one float4, full tables the four entries in two).
template <int K> __device__ __forceinline__ J2 fetch_k(const DevTerm &T, int n_ant, int tint, int fint, int ant)
{
    const unsigned idx = ((unsigned)tint * n_ant + ant) * (unsigned)T.n_fint + fint;
    if constexpr (K == KIND_FULL) return j_from(__ldg(T.tab + 2 * (size_t)idx), __ldg(T.tab + 2 * (size_t)idx + 1));
    else return j_diag(__ldg(T.tab + idx));
}

// Multiply helpers specialised on the kind of one operand.
template <int K> __device__ __forceinline__ J2 lmulk(const J2 &A, const J2 &B)
{
    if constexpr (K == KIND_NONE) return B;
    else if constexpr (K == KIND_DIAG) return j_dmul(A.a, A.d, B);
    else return j_mul(A, B);
}
template <int K> __device__ __forceinline__ J2 rmulk(const J2 &A, const J2 &B)
{
    if constexpr (K == KIND_NONE) return A;
    else if constexpr (K == KIND_DIAG) return j_muld(A, B.a, B.d);
    else return j_mul(A, B);
}

// A B^H with B of kind K
template <int K> __device__ __forceinline__ J2 rmulk_h(const J2 &A, const J2 &B)
{
    if constexpr (K == KIND_NONE) return A;
    else if constexpr (K == KIND_DIAG) return j_muld(A, cconj(B.a), cconj(B.d));
    else return j_mul_h(A, B);
}

// ---------------------------------------------------------------------------
// register accumulators of one side (antenna) of a sample
// ---------------------------------------------------------------------------

template <int TS, bool HAS_L> struct AccLayout;
// DIAG without L: JHJ diagonal (2 reals) + JHr (2 complex); off-diagonal is exactly 0.
template <> struct AccLayout<TS_DIAG, false> {
    static constexpr int KR = 6, KG = KG_DIAG;
    __device__ static constexpr int g(int i) { return i < 2 ? i : i + 2; }
};
template <> struct AccLayout<TS_DIAG, true> {
    static constexpr int KR = 8, KG = KG_DIAG;
    __device__ static constexpr int g(int i) { return i; }
};
// FULL without L: E = I (x) X^T couples only parameters in the same row of G,
// so only JHJ[0][1] and JHJ[2][3] are off-diagonal non-zeros.
template <> struct AccLayout<TS_FULL, false> {
    static constexpr int KR = 16, KG = KG_FULL;
    __device__ static constexpr int g(int i) { return i < 6 ? i : (i < 8 ? i + 8 : i + 8); }
};
template <> struct AccLayout<TS_FULL, true> {
    static constexpr int KR = 24, KG = KG_FULL;
    __device__ static constexpr int g(int i) { return i; }
};

template <int KR, bool KAHAN> struct Acc {
    float s[KR];
    float c[KAHAN ? KR : 1];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < KR; ++i) s[i] = 0.f;
        if constexpr (KAHAN) {
#pragma unroll
            for (int i = 0; i < KR; ++i) c[i] = 0.f;
        }
    }
    __device__ __forceinline__ void add(int i, float x)
    {
        if constexpr (KAHAN) two_sum_add(s[i], c[i], x);
        else s[i] += x;
    }
    // s[i] += a b
    __device__ __forceinline__ void fma(int i, float a, float b)
    {
        if constexpr (KAHAN) two_sum_add(s[i], c[i], a * b);
        else s[i] = fmaf(a, b, s[i]);
    }
    // (s[i], s[i+1]) += conj(x) y
    __device__ __forceinline__ void cfma(int i, float2 x, float2 y)
    {
        if constexpr (KAHAN) {
            two_sum_add(s[i], c[i], fmaf(x.x, y.x, x.y * y.y));
            two_sum_add(s[i + 1], c[i + 1], fmaf(x.x, y.y, -x.y * y.x));
        } else {
            s[i] = fmaf(x.x, y.x, fmaf(x.y, y.y, s[i]));
            s[i + 1] = fmaf(x.x, y.y, fmaf(-x.y, y.x, s[i + 1]));
        }
    }
};

// Contribution of one sample to antenna a's blocks: E = L_a (x) X^T (Eq. vectrick,
// Eq. g_derivative_dd) restricted to the term's free parameters, weights w
// per correlation and weighted residual wr = w * r, element by element (both in
// the orientation of this side).
template <int TS, bool HAS_L, bool KAHAN>
__device__ __forceinline__ void accumulate_side(Acc<AccLayout<TS, HAS_L>::KR, KAHAN> &A, const J2 &L,
                                                const J2 &X, float4 w, const J2 &wr)
{
    const float wv[4] = { w.x, w.y, w.z, w.w };
    const float2 wrv[4] = { wr.a, wr.b, wr.c, wr.d };
    const float2 Xv[4] = { X.a, X.b, X.c, X.d };            // X[l][j] = Xv[2l+j]
    if constexpr (!HAS_L) {
        if constexpr (TS == TS_DIAG) {
            // parameter k in {XX, YY} touches row k of V: E[(k,j), k] = X[k][j]
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float2 x = Xv[2 * k + j];
                    const float ww = wv[2 * k + j];
                    A.fma(k, ww, cnorm2(x));
                    A.cfma(2 + 2 * k, x, wrv[2 * k + j]);
                }
        } else {
            // parameter u = (k, l): E[(k,j), (k,l)] = X[l][j]
            const float2 x00 = Xv[0], x01 = Xv[1], x10 = Xv[2], x11 = Xv[3];
            const float n00 = cnorm2(x00), n01 = cnorm2(x01), n10 = cnorm2(x10), n11 = cnorm2(x11);
            const float2 o0 = cmulc(x10, x00);   // conj(X[0][0]) X[1][0]
            const float2 o1 = cmulc(x11, x01);   // conj(X[0][1]) X[1][1]
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float w0 = wv[2 * k], w1 = wv[2 * k + 1];
                A.fma(2 * k + 0, w0, n00);
                A.fma(2 * k + 0, w1, n01);
                A.fma(2 * k + 1, w0, n10);
                A.fma(2 * k + 1, w1, n11);
                A.fma(4 + 2 * k, w0, o0.x);
                A.fma(4 + 2 * k, w1, o1.x);
                A.fma(5 + 2 * k, w0, o0.y);
                A.fma(5 + 2 * k, w1, o1.y);
                const float2 wr0 = wrv[2 * k], wr1 = wrv[2 * k + 1];
                A.cfma(8 + 4 * k, x00, wr0);
                A.cfma(8 + 4 * k, x01, wr1);
                A.cfma(10 + 4 * k, x10, wr0);
                A.cfma(10 + 4 * k, x11, wr1);
            }
        }
    } else {
        const float2 Lv[4] = { L.a, L.b, L.c, L.d };
        if constexpr (TS == TS_DIAG) {
            // free columns (0,0) and (1,1): E[(i,j), k] = L[i][k] X[k][j]
            float2 E0[4], E1[4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    E0[2 * i + j] = cmul(Lv[2 * i + 0], Xv[0 + j]);
                    E1[2 * i + j] = cmul(Lv[2 * i + 1], Xv[2 + j]);
                }
            float h00 = 0.f, h11 = 0.f;
            float2 h01 = make_float2(0.f, 0.f), j0 = h01, j1 = h01;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                h00 = fmaf(wv[m], cnorm2(E0[m]), h00);
                h11 = fmaf(wv[m], cnorm2(E1[m]), h11);
                h01 = cfma_conj(E0[m], cscale(E1[m], wv[m]), h01);
                j0 = cfma_conj(E0[m], wrv[m], j0);
                j1 = cfma_conj(E1[m], wrv[m], j1);
            }
            A.add(0, h00); A.add(1, h11); A.add(2, h01.x); A.add(3, h01.y);
            A.add(4, j0.x); A.add(5, j0.y); A.add(6, j1.x); A.add(7, j1.y);
        } else {
            // E[(i,j), (k,l)] = L[i][k] X[l][j]
            float2 E[4][4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int k = 0; k < 2; ++k)
#pragma unroll
                        for (int l = 0; l < 2; ++l) E[2 * i + j][2 * k + l] = cmul(Lv[2 * i + k], Xv[2 * l + j]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                float h = 0.f;
                float2 jr = make_float2(0.f, 0.f);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    h = fmaf(wv[m], cnorm2(E[m][u]), h);
                    jr = cfma_conj(E[m][u], wrv[m], jr);
                }
                A.add(u, h);
                A.add(16 + 2 * u, jr.x);
                A.add(17 + 2 * u, jr.y);
            }
            int o = 4;
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = u + 1; v < 4; ++v) {
                    float2 h = make_float2(0.f, 0.f);
#pragma unroll
                    for (int m = 0; m < 4; ++m) h = cfma_conj(E[m][u], cscale(E[m][v], wv[m]), h);
                    A.add(o, h.x);
                    A.add(o + 1, h.y);
                    o += 2;
                }
        }
    }
}

// ---------------------------------------------------------------------------
// flush: segmented warp reduction over lanes with equal bins + FP64 atomics
// ---------------------------------------------------------------------------

template <int KR, int KG, bool KAHAN, typename Layout>
__device__ __forceinline__ void flush_side(Acc<KR, KAHAN> &A, int key, int ant, int lane, unsigned seg_end,
                                           bool head, bool live, double *__restrict__ acc, int n_ant)
{
#pragma unroll
    for (int i = 0; i < KR; ++i) {
        float v = A.s[i];
        if constexpr (KAHAN) v += A.c[i];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float o = __shfl_down_sync(0xffffffffu, v, d);
            if (lane + d < (int)seg_end) v += o;
        }
        if (head && live) atomicAdd(acc + ((size_t)key * n_ant + ant) * KG + Layout::g(i), (double)v);
    }
    A.zero();
}

// ---------------------------------------------------------------------------
// one sample: chain factors, residual and both antennas' contributions
// ---------------------------------------------------------------------------

// Chain factors of antenna a around the solved term n (Eq. jonesfactor) from
// per-term interval indices (tint: per row, fint: per channel).
template <int LK, int RK>
__device__ __forceinline__ void chain_at(const Chain &C, const int *tint, const int *fint, int a, J2 &L, J2 &G, J2 &R)
{
    bool hl = false, hr = false;
    L = j_identity();
    R = j_identity();
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {
        if (j >= C.n_terms) break;
        const J2 J = fetch_jones(C.t[j], C.n_ant, tint[j], fint[j], a);
        if (j < C.n) {
            if constexpr (LK != KIND_NONE) { L = hl ? j_mul(L, J) : J; hl = true; }
        } else if (j == C.n) {
            G = J;
        } else {
            if constexpr (RK != KIND_NONE) { R = hr ? j_mul(R, J) : J; hr = true; }
        }
    }
}

// Interval indices of one sample: for the solved term n and the other term of a
// two-term chain, or for every term of a longer chain.
struct SampleIdx {
    int tn, fn;            // solved term
    int to, fo;            // other term (two-term chains)
    int t[MAXT], f[MAXT];  // every term (longer chains)
};

// Chain factors of antenna a around the solved term (Eq. jonesfactor).  SIMPLE:
// the chain has at most one other term, on the left (LK) or on the right (RK).
template <int GK, int LK, int RK, bool SIMPLE>
__device__ __forceinline__ void factors(const AccArgs &a, const SampleIdx &ix, int ant, J2 &L, J2 &G, J2 &R)
{
    if constexpr (SIMPLE) {
        G = fetch_k<GK>(a.tn, a.C.n_ant, ix.tn, ix.fn, ant);
        if constexpr (LK != KIND_NONE) L = fetch_k<LK>(a.to, a.C.n_ant, ix.to, ix.fo, ant);
        if constexpr (RK != KIND_NONE) R = fetch_k<RK>(a.to, a.C.n_ant, ix.to, ix.fo, ant);
    } else {
        chain_at<LK, RK>(a.C, ix.t, ix.f, ant, L, G, R);
    }
}

// Contribution of one unflagged sample of baseline (p, q) to the p and q blocks.
// With Z = R_p M R_q^H:  X = Z G_q^H L_q^H = R_p M C_q^H,  V = L_p G_p X  (Eq. chain_trick),
// and for the conjugate baseline Y = R_q M^H C_p^H = (L_p G_p Z)^H.
// BF: the J^H W r slots receive J^H W d instead.  V is linear in the solved gains of
// either side (V = E g_p, V^H = E' g_q), so J^H W r = J^H W d - JHJ g per block, and the
// update forms the difference in FP64 (UpdArgs::b_form); the sample then needs neither
// V nor the residual.
template <int TS, int LK, int RK, bool KAHAN, bool BF = false>
__device__ __forceinline__ void sample_math(const J2 &Lp, const J2 &Gp, const J2 &Rp, const J2 &Lq, const J2 &Gq,
                                            const J2 &Rq, const J2 &Dm, const J2 &M, float4 w,
                                            Acc<AccLayout<TS, LK != KIND_NONE>::KR, KAHAN> &Ap,
                                            Acc<AccLayout<TS, LK != KIND_NONE>::KR, KAHAN> &Aq)
{
    constexpr bool HAS_L = LK != KIND_NONE;
    constexpr int GK = TS == TS_FULL ? KIND_FULL : KIND_DIAG;
    J2 X, Y, V;
    if constexpr (RK == KIND_NONE) {
        const J2 Cp = HAS_L ? rmulk<GK>(Lp, Gp) : Gp;
        const J2 Cq = HAS_L ? rmulk<GK>(Lq, Gq) : Gq;
        constexpr int CK = HAS_L ? KIND_FULL : GK;
        const J2 A = lmulk<CK>(Cp, M);                 // C_p M
        X = rmulk_h<CK>(M, Cq);                        // M C_q^H
        if constexpr (!BF) V = rmulk_h<CK>(A, Cq);     // C_p M C_q^H
        Y = j_herm(A);                                 // M^H C_p^H
    } else {
        J2 Z;
        if constexpr (RK == KIND_DIAG) Z = j_muld(j_dmul(Rp.a, Rp.d, M), cconj(Rq.a), cconj(Rq.d));
        else Z = j_mul_h(j_mul(Rp, M), Rq);
        X = rmulk_h<LK>(rmulk_h<GK>(Z, Gq), Lq);
        const J2 W = lmulk<LK>(Lp, lmulk<GK>(Gp, Z));
        Y = j_herm(W);
        if constexpr (!BF) V = lmulk<LK>(Lp, lmulk<GK>(Gp, X));
    }
    // weighted residual w * (D - V) (BF: the weighted data w * D); the conjugate
    // baseline's is its conjugate transpose
    J2 wr;
    if constexpr (BF) {
        wr.a = cscale(Dm.a, w.x); wr.b = cscale(Dm.b, w.y);
        wr.c = cscale(Dm.c, w.z); wr.d = cscale(Dm.d, w.w);
    } else {
        wr.a = cscale(csub(Dm.a, V.a), w.x); wr.b = cscale(csub(Dm.b, V.b), w.y);
        wr.c = cscale(csub(Dm.c, V.c), w.z); wr.d = cscale(csub(Dm.d, V.d), w.w);
    }
    accumulate_side<TS, HAS_L, KAHAN>(Ap, Lp, X, w, wr);
    accumulate_side<TS, HAS_L, KAHAN>(Aq, Lq, Y, make_float4(w.x, w.z, w.y, w.w), j_herm(wr));
}

template <int TS, int LK, int RK, bool SIMPLE, bool KAHAN>
__device__ __forceinline__ void sample_contrib(const AccArgs &a, const SampleIdx &ix, int p, int q, const J2 &Dm,
                                               const J2 &M, float4 w,
                                               Acc<AccLayout<TS, LK != KIND_NONE>::KR, KAHAN> &Ap,
                                               Acc<AccLayout<TS, LK != KIND_NONE>::KR, KAHAN> &Aq)
{
    constexpr int GK = TS == TS_FULL ? KIND_FULL : KIND_DIAG;
    J2 Lp, Gp, Rp, Lq, Gq, Rq;
    factors<GK, LK, RK, SIMPLE>(a, ix, p, Lp, Gp, Rp);
    factors<GK, LK, RK, SIMPLE>(a, ix, q, Lq, Gq, Rq);
    sample_math<TS, LK, RK, KAHAN>(Lp, Gp, Rp, Lq, Gq, Rq, Dm, M, w, Ap, Aq);
}

// Interval indices of a sample at data time `time` and channel c.
template <bool SIMPLE>
__device__ __forceinline__ void sample_index(const AccArgs &a, int time, int c, bool in_range, SampleIdx &ix)
{
    ix.tn = __ldg(a.tn.t_map + time);
    ix.fn = in_range ? __ldg(a.tn.f_map + c) : 0;
    if constexpr (SIMPLE) {
        if (a.C.n_terms > 1) {
            ix.to = __ldg(a.to.t_map + time);
            ix.fo = in_range ? __ldg(a.to.f_map + c) : 0;
        } else {
            ix.to = 0;
            ix.fo = 0;
        }
    } else {
#pragma unroll
        for (int j = 0; j < MAXT; ++j) {
            ix.t[j] = j < a.C.n_terms ? __ldg(a.C.t[j].t_map + time) : 0;
            ix.f[j] = (j < a.C.n_terms && in_range) ? __ldg(a.C.t[j].f_map + c) : 0;
        }
    }
}

__device__ __forceinline__ J2 load_model16(uint4 h, float sc)
{
    J2 M;
    M.a = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.x)), sc);
    M.b = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.y)), sc);
    M.c = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.z)), sc);
    M.d = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.w)), sc);
    return M;
}

// ---------------------------------------------------------------------------
// the accumulate kernel
// ---------------------------------------------------------------------------


// Position in a warp's stream of row segments: unit u (a row for row tiles, a
// baseline strip x 32-channel chunk for strip tiles), segment i of len.
struct SegCursor {
    long u;
    int i, len, beg, c0;
    int row;          // row of the current segment (-1: nothing to read)
    int tn;           // row tiles: time-interval index of the unit's row (-1: nothing to read)
};

// Locate the current segment; with SKIP set, rows without unflagged data and (row
// tiles) 32-channel chunks whose intervals have all converged read nothing.
template <bool SKIP>
__device__ __forceinline__ void seg_locate(const AccArgs &a, SegCursor &k)
{
    if (a.order == 0) {
        k.row = (int)k.u;
        if (SKIP && (k.tn < 0 || !__ldg(a.chunk_active + (size_t)k.tn * a.n_chunks + k.i))) k.row = -1;
    } else {
        k.row = __ldg(a.D.strip_rows + k.beg + k.i);
        if (SKIP && !__ldg(a.row_live + k.row)) k.row = -1;
    }
}

__device__ __forceinline__ void seg_unit(const AccArgs &a, SegCursor &k, long n_units)
{
    k.i = 0;
    k.len = 0;
    if (k.u >= n_units) return;
    if (a.order == 0) {
        k.len = a.n_chunks; k.beg = 0; k.c0 = 0;
        k.tn = __ldg(a.row_info + k.u).z;
    }
    else {
        const int s = (int)(k.u / a.n_chunks);
        k.c0 = (int)(k.u % a.n_chunks) * 32;
        k.beg = __ldg(a.D.strip_off + s);
        k.len = __ldg(a.D.strip_off + s + 1) - k.beg;
    }
}

__device__ __forceinline__ void seg_next(const AccArgs &a, SegCursor &k, long n_units, long stride)
{
    if (++k.i < k.len) return;
    do {
        k.u += stride;
        seg_unit(a, k, n_units);
    } while (k.u < n_units && k.len == 0);
}

// Accumulate kernel with per-lane asynchronous prefetch.
//
// Every warp streams through its own work units (a unit is one row for row
// tiles, or one baseline strip x 32 channels for strip tiles); lane l handles
// channel c0 + l of every row segment and keeps its register partial sums while
// its sample's interval bin stays the same (see flush_side).  The d, m and w of
// the lane's sample are fetched DEPTH - 1 segments ahead with 16-byte cp.async
// copies into the warp's ring in shared memory, so the HBM latency of a segment
// is overlapped with the arithmetic of the previous ones; rows without an
// unflagged cross-correlation sample are not read at all.  The Jones factors
// come from the small gain tables through the read-only cache.
template <int TS, int LK, int RK, bool SIMPLE, bool M16, int DEPTH>
__global__ void __launch_bounds__(256) acc_kernel(const AccArgs a)
{
    if (__ldg(a.n_active) == 0) return;
    constexpr bool HAS_L = LK != KIND_NONE;
    constexpr bool KAHAN = M16;
    using Lay = AccLayout<TS, HAS_L>;
    constexpr int KR = Lay::KR, KG = Lay::KG;
    constexpr int V4 = M16 ? 4 : 5;                 // 16-byte words per sample: d (2), m (2 or 1), w (1)
    extern __shared__ float4 s_ring[];
    const Data &D = a.D;
    const DevTerm &Tn = a.tn;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float4 *ring = s_ring + (size_t)wib * DEPTH * 32 * V4;
    const long n_units = a.order == 0 ? (long)D.n_row : (long)D.n_strips * a.n_chunks;
    const long stride = ((long)gridDim.x * blockDim.x) >> 5;

    SegCursor ck, pf;
    ck.u = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    seg_unit(a, ck, n_units);
    if (ck.u < n_units && ck.len == 0) seg_next(a, ck, n_units, stride);
    pf = ck;
    int pf_stage = 0;

    auto issue = [&](SegCursor &k) {
        seg_locate<true>(a, k);
        const int c = a.order == 0 ? k.i * 32 + lane : k.c0 + lane;
        const bool rd = k.row >= 0 && c < D.n_chan;
        const size_t s = rd ? (size_t)k.row * D.n_chan + c : 0;
        const uint32_t nb = rd ? 16u : 0u;
        float4 *slot = ring + ((size_t)pf_stage * 32 + lane) * V4;
        cp_async16(slot + 0, D.vis + 2 * s, nb);
        cp_async16(slot + 1, D.vis + 2 * s + 1, nb);
        if constexpr (M16) {
            cp_async16(slot + 2, D.model16 + s, nb);
            cp_async16(slot + 3, D.weight + s, nb);
        } else {
            cp_async16(slot + 2, D.model + 2 * s, nb);
            cp_async16(slot + 3, D.model + 2 * s + 1, nb);
            cp_async16(slot + 4, D.weight + s, nb);
        }
        if (++pf_stage == DEPTH) pf_stage = 0;
    };

    // prime the ring with DEPTH - 1 segments (one commit group each)
#pragma unroll
    for (int d = 0; d < DEPTH - 1; ++d) {
        if (pf.u < n_units) {
            issue(pf);
            seg_next(a, pf, n_units, stride);
        }
        cp_async_commit();
    }

    Acc<KR, KAHAN> Ap, Aq;
    Ap.zero();
    Aq.zero();
    int stage = 0, cur_key = -1, p = 0, q = 0;
    while (ck.u < n_units) {
        if (pf.u < n_units) {
            issue(pf);
            seg_next(a, pf, n_units, stride);
        }
        cp_async_commit();
        cp_async_wait<DEPTH - 1>();                 // this lane's copies of the current segment landed
        seg_locate<false>(a, ck);
        const int row = ck.row;
        const int c = a.order == 0 ? ck.i * 32 + lane : ck.c0 + lane;
        const int4 meta = __ldg(D.rows + row);
        p = meta.x;
        q = meta.y;
        const bool in_range = c < D.n_chan && p != q;
        SampleIdx ix;
        sample_index<SIMPLE>(a, meta.z, c, in_range, ix);
        const int key = in_range ? ix.tn * Tn.n_fint + ix.fn : -1;
        if (__any_sync(0xffffffffu, cur_key >= 0 && key != cur_key)) {
            const unsigned m = __match_any_sync(0xffffffffu, cur_key);
            const unsigned seg_end = 32 - __clz(m);
            const bool head = lane == __ffs(m) - 1;
            const bool live = cur_key >= 0 && __ldg(a.active + cur_key);
            flush_side<KR, KG, KAHAN, Lay>(Ap, cur_key, p, lane, seg_end, head, live, a.acc, a.C.n_ant);
            flush_side<KR, KG, KAHAN, Lay>(Aq, cur_key, q, lane, seg_end, head, live, a.acc, a.C.n_ant);
        }
        cur_key = key;
        bool ok = in_range && __ldg(a.active + key);
        if (ok && D.flag) ok = __ldg(D.flag + (size_t)row * D.n_chan + c) == 0;
        if (ok) ok = __ldg(a.row_live + row) != 0;
        if (ok) {
            const float4 *slot = ring + ((size_t)stage * 32 + lane) * V4;
            const J2 Dm = j_from(slot[0], slot[1]);
            J2 M;
            float4 w;
            if constexpr (M16) {
                M = load_model16(*reinterpret_cast<const uint4 *>(slot + 2), __ldg(D.bl_scale + meta.w));
                w = slot[3];
            } else {
                M = j_from(slot[2], slot[3]);
                w = slot[4];
            }
            sample_contrib<TS, LK, RK, SIMPLE, KAHAN>(a, ix, p, q, Dm, M, w, Ap, Aq);
        }
        if (++stage == DEPTH) stage = 0;
        const long u_prev = ck.u;
        seg_next(a, ck, n_units, stride);
        if (ck.u != u_prev) {
            if (__any_sync(0xffffffffu, cur_key >= 0)) {
                const unsigned m = __match_any_sync(0xffffffffu, cur_key);
                const unsigned seg_end = 32 - __clz(m);
                const bool head = lane == __ffs(m) - 1;
                const bool live = cur_key >= 0 && __ldg(a.active + cur_key);
                flush_side<KR, KG, KAHAN, Lay>(Ap, cur_key, p, lane, seg_end, head, live, a.acc, a.C.n_ant);
                flush_side<KR, KG, KAHAN, Lay>(Aq, cur_key, q, lane, seg_end, head, live, a.acc, a.C.n_ant);
            }
            cur_key = -1;
        }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// FP64 block solve and update
// ---------------------------------------------------------------------------

// LU with partial pivoting; returns 1 when the block is treated as singular
// (zero trace, zero pivot, or reciprocal 1-norm condition number < 1e-12).
template <int N>
__device__ int block_solve(double2 (&A)[N][N], const double2 (&b)[N], double2 (&x)[N])
{
    auto cabs = [](double2 z) { return sqrt(z.x * z.x + z.y * z.y); };
    auto cm = [](double2 u, double2 v) { return make_double2(u.x * v.x - u.y * v.y, u.x * v.y + u.y * v.x); };
    double trace = 0, anorm = 0;
    for (int i = 0; i < N; ++i) trace += A[i][i].x;
    if (!(trace > 0)) return 1;
    if constexpr (N == 2) {
        // closed form: A^-1 = [[d, -b], [-c, a]] / (a d - b c); the same singularity tests (a zero
        // determinant is a zero pivot; reciprocal 1-norm condition number from the inverse)
        const double2 a = A[0][0], bb = A[0][1], c = A[1][0], d = A[1][1];
        const double2 ad = cm(a, d), bc = cm(bb, c);
        const double2 det = make_double2(ad.x - bc.x, ad.y - bc.y);
        const double den = det.x * det.x + det.y * det.y;
        if (!(den > 0)) return 1;
        const double2 r = make_double2(det.x / den, -det.y / den);       // 1 / det
        const double2 i00 = cm(d, r), i11 = cm(a, r);
        const double2 i01 = cm(make_double2(-bb.x, -bb.y), r), i10 = cm(make_double2(-c.x, -c.y), r);
        anorm = fmax(cabs(a) + cabs(c), cabs(bb) + cabs(d));
        const double inorm = fmax(cabs(i00) + cabs(i10), cabs(i01) + cabs(i11));
        if (!(1.0 / (anorm * inorm) >= 1e-12)) return 1;
        const double2 t0 = cm(i00, b[0]), t1 = cm(i01, b[1]), t2 = cm(i10, b[0]), t3 = cm(i11, b[1]);
        x[0] = make_double2(t0.x + t1.x, t0.y + t1.y);
        x[1] = make_double2(t2.x + t3.x, t2.y + t3.y);
        return 0;
    }
    for (int j = 0; j < N; ++j) {
        double s = 0;
        for (int i = 0; i < N; ++i) s += cabs(A[i][j]);
        anorm = fmax(anorm, s);
    }
    // partial pivoting on |.|^2 (the same order as |.|); divisions by a pivot as products with
    // its reciprocal, one reciprocal per pivot (FP64 division is slow on this part)
    auto cn2 = [](double2 z) { return z.x * z.x + z.y * z.y; };
    auto crecip = [](double2 v) {
        const double den = v.x * v.x + v.y * v.y;
        const double r = 1.0 / den;
        return make_double2(v.x * r, -v.y * r);
    };
    int piv[N];
    double2 rpiv[N];
    for (int i = 0; i < N; ++i) piv[i] = i;
    for (int k = 0; k < N; ++k) {
        int m = k;
        for (int i = k + 1; i < N; ++i) if (cn2(A[i][k]) > cn2(A[m][k])) m = i;
        if (cn2(A[m][k]) == 0) return 1;
        if (m != k) {
            for (int j = 0; j < N; ++j) { double2 t = A[k][j]; A[k][j] = A[m][j]; A[m][j] = t; }
            int t = piv[k]; piv[k] = piv[m]; piv[m] = t;
        }
        rpiv[k] = crecip(A[k][k]);
        for (int i = k + 1; i < N; ++i) {
            A[i][k] = cm(A[i][k], rpiv[k]);
            for (int j = k + 1; j < N; ++j) {
                const double2 t = cm(A[i][k], A[k][j]);
                A[i][j].x -= t.x; A[i][j].y -= t.y;
            }
        }
    }
    double2 inv[N][N];
    for (int col = 0; col < N; ++col) {
        double2 y[N];
        for (int i = 0; i < N; ++i) {
            double2 s = make_double2(piv[i] == col ? 1.0 : 0.0, 0.0);
            for (int j = 0; j < i; ++j) { const double2 t = cm(A[i][j], y[j]); s.x -= t.x; s.y -= t.y; }
            y[i] = s;
        }
        for (int i = N - 1; i >= 0; --i) {
            double2 s = y[i];
            for (int j = i + 1; j < N; ++j) { const double2 t = cm(A[i][j], y[j]); s.x -= t.x; s.y -= t.y; }
            y[i] = cm(s, rpiv[i]);
        }
        for (int i = 0; i < N; ++i) inv[i][col] = y[i];
    }
    double inorm = 0;
    for (int j = 0; j < N; ++j) {
        double s = 0;
        for (int i = 0; i < N; ++i) s += cabs(inv[i][j]);
        inorm = fmax(inorm, s);
    }
    if (!(1.0 / (anorm * inorm) >= 1e-12)) return 1;
    for (int i = 0; i < N; ++i) {
        double2 s = make_double2(0, 0);
        for (int j = 0; j < N; ++j) { const double2 t = cm(inv[i][j], b[j]); s.x += t.x; s.y += t.y; }
        x[i] = s;
    }
    return 0;
}

struct UpdArgs {
    int type;                // QC_TERM_*
    int n_bins, n_fint, n_ant;
    double *acc;             // [n_bins][n_ant][KG]  (read, then zeroed)
    double *params;          // FP64 master: complex [n_bins][n_ant][4] or phase [n_bins][n_ant][2]
    float4 *tab;             // FP32 kernel table [n_tint][n_ant][n_fint] x (1|2)
    int8_t *gain_flags;      // [n_bins][n_ant]
    int *iters;              // [n_bins]
    uint8_t *active;         // [n_bins]
    const int *n_active_prev;// counter of intervals active entering this iteration
    int *n_active_next;      // incremented for every interval still active after it
    const long long *bin_nvis, *bin_nbytes;   // per-bin samples and algorithmic bytes
    unsigned long long *vis_iters, *acc_bytes;
    int k;                   // iteration (1-based)
    double alpha, tol;
    // gain flagging on divergence (div != 0; max_iter >= 4): per (bin, antenna) the larger of the
    // first two and of the last two relative updates, and the parameters before the solve
    int div, max_iter;
    double *div_stats;       // [n_bins][n_ant][2], zero before the first iteration
    const double *params0;   // as params
    // nonzero: the J^H W r slots of acc hold J^H W d (the streaming kernel), and the update
    // takes J^H W r = J^H W d - JHJ g at the gains of this iteration, in FP64
    int b_form;
};

// b -= M g (complex N x N block times the complex gain vector)
template <int N>
__device__ __forceinline__ void sub_block_times(double2 (&b)[N], const double2 (&M)[N][N], const double2 (&g)[N])
{
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            b[i].x -= M[i][j].x * g[j].x - M[i][j].y * g[j].y;
            b[i].y -= M[i][j].x * g[j].y + M[i][j].y * g[j].x;
        }
}

__device__ __forceinline__ void store_jones_tab(const UpdArgs &u, int bin, int ant, const double2 g[4])
{
    const int tint = bin / u.n_fint, fint = bin % u.n_fint;
    const size_t idx = ((size_t)tint * u.n_ant + ant) * u.n_fint + fint;
    if (u.type == 1) {
        u.tab[2 * idx] = make_float4((float)g[0].x, (float)g[0].y, (float)g[1].x, (float)g[1].y);
        u.tab[2 * idx + 1] = make_float4((float)g[2].x, (float)g[2].y, (float)g[3].x, (float)g[3].y);
    } else {
        u.tab[idx] = make_float4((float)g[0].x, (float)g[0].y, (float)g[3].x, (float)g[3].y);
    }
}

static __global__ void __launch_bounds__(128) update_kernel(const UpdArgs u)
{
    if (*u.n_active_prev == 0) return;
    const int bin = blockIdx.x;
    if (!u.active[bin]) return;
    const int KG = u.type == 1 ? KG_FULL : KG_DIAG;
    double num = 0, den = 0;
    for (int ant = threadIdx.x; ant < u.n_ant; ant += blockDim.x) {
        double *A = u.acc + ((size_t)bin * u.n_ant + ant) * KG;
        const size_t pidx = (size_t)bin * u.n_ant + ant;
        double2 gold[4], gnew[4];
        int singular;
        if (u.type == 1) {
            double2 M[4][4], b[4], x[4];
            for (int i = 0; i < 4; ++i) M[i][i] = make_double2(A[i], 0.0);
            int o = 4;
            for (int i = 0; i < 4; ++i)
                for (int j = i + 1; j < 4; ++j) {
                    M[i][j] = make_double2(A[o], A[o + 1]);
                    M[j][i] = make_double2(A[o], -A[o + 1]);
                    o += 2;
                }
            for (int i = 0; i < 4; ++i) b[i] = make_double2(A[16 + 2 * i], A[17 + 2 * i]);
            double2 *P = reinterpret_cast<double2 *>(u.params) + 4 * pidx;
            for (int e = 0; e < 4; ++e) gold[e] = P[e];
            if (u.b_form) sub_block_times<4>(b, M, gold);
            singular = block_solve<4>(M, b, x);
            for (int e = 0; e < 4; ++e)
                gnew[e] = singular ? gold[e] : make_double2(gold[e].x + u.alpha * x[e].x, gold[e].y + u.alpha * x[e].y);
            for (int e = 0; e < 4; ++e) P[e] = gnew[e];
        } else {
            double2 M[2][2], b[2], x[2];
            M[0][0] = make_double2(A[0], 0.0);
            M[1][1] = make_double2(A[1], 0.0);
            M[0][1] = make_double2(A[2], A[3]);
            M[1][0] = make_double2(A[2], -A[3]);
            b[0] = make_double2(A[4], A[5]);
            b[1] = make_double2(A[6], A[7]);
            if (u.type == 2) {
                // Scenario 1 chain rule with dg/dphi = i g (constant over the interval):
                // JHJ_phi = 2 Re(conj(g_u) g_v JHJ[u][v]), JHr_phi = 2 Im(conj(g_u) JHr[u]).
                double *phi = u.params + 2 * pidx;
                double2 g[2];
                for (int k = 0; k < 2; ++k) { double sn, cs; sincos(phi[k], &sn, &cs); g[k] = make_double2(cs, sn); }
                if (u.b_form) sub_block_times<2>(b, M, g);
                auto cmc = [](double2 p, double2 q) {     // conj(p) * q
                    return make_double2(p.x * q.x + p.y * q.y, p.x * q.y - p.y * q.x);
                };
                double2 R[2][2], rb[2];
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) {
                        const double2 gg = cmc(g[i], g[j]);
                        R[i][j] = make_double2(2.0 * (gg.x * M[i][j].x - gg.y * M[i][j].y), 0.0);
                    }
                for (int i = 0; i < 2; ++i) {
                    const double2 t = cmc(g[i], b[i]);
                    rb[i] = make_double2(2.0 * t.y, 0.0);
                }
                gold[0] = g[0]; gold[1] = make_double2(0, 0); gold[2] = gold[1]; gold[3] = g[1];
                singular = block_solve<2>(R, rb, x);
                if (!singular) { phi[0] += u.alpha * x[0].x; phi[1] += u.alpha * x[1].x; }
                for (int k = 0; k < 2; ++k) { double sn, cs; sincos(phi[k], &sn, &cs); g[k] = make_double2(cs, sn); }
                gnew[0] = g[0]; gnew[1] = make_double2(0, 0); gnew[2] = gnew[1]; gnew[3] = g[1];
            } else {
                double2 *P = reinterpret_cast<double2 *>(u.params) + 4 * pidx;
                for (int e = 0; e < 4; ++e) gold[e] = P[e];
                if (u.b_form) {
                    const double2 g[2] = { gold[0], gold[3] };
                    sub_block_times<2>(b, M, g);
                }
                singular = block_solve<2>(M, b, x);
                gnew[0] = gold[0]; gnew[1] = make_double2(0, 0); gnew[2] = gnew[1]; gnew[3] = gold[3];
                if (!singular) {
                    gnew[0] = make_double2(gold[0].x + u.alpha * x[0].x, gold[0].y + u.alpha * x[0].y);
                    gnew[3] = make_double2(gold[3].x + u.alpha * x[1].x, gold[3].y + u.alpha * x[1].y);
                }
                for (int e = 0; e < 4; ++e) P[e] = gnew[e];
            }
        }
        if (u.gain_flags) u.gain_flags[pidx] = (int8_t)singular;
        store_jones_tab(u, bin, ant, gnew);
        double na = 0, da = 0;
        for (int e = 0; e < 4; ++e) {
            const double dx = gnew[e].x - gold[e].x, dy = gnew[e].y - gold[e].y;
            na += dx * dx + dy * dy;
            da += gnew[e].x * gnew[e].x + gnew[e].y * gnew[e].y;
        }
        num += na;
        den += da;
        if (u.div) {
            const double d = da > 0 ? sqrt(na / da) : 0.0;
            double *ds = u.div_stats + 2 * pidx;
            if (u.k <= 2) ds[0] = fmax(ds[0], d);
            if (u.k >= u.max_iter - 1) ds[1] = fmax(ds[1], d);
        }
        for (int i = 0; i < KG; ++i) A[i] = 0.0;
    }
    // interval norms: block reduction in FP64
    __shared__ double s_num[4], s_den[4];
    __shared__ int s_unconverged;
    for (int d = 16; d > 0; d >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, d);
        den += __shfl_down_sync(0xffffffffu, den, d);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_num[w] = num; s_den[w] = den; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tn = 0, td = 0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) { tn += s_num[i]; td += s_den[i]; }
        const double delta = td > 0 ? sqrt(tn / td) : 0.0;
        if (u.iters) u.iters[bin] = u.k;
        atomicAdd(u.vis_iters, (unsigned long long)u.bin_nvis[bin]);
        atomicAdd(u.acc_bytes, (unsigned long long)u.bin_nbytes[bin]);
        if (delta < u.tol) u.active[bin] = 0;
        else atomicAdd(u.n_active_next, 1);
        s_unconverged = delta >= u.tol;
    }
    if (u.div && u.k == u.max_iter) {
        // the interval ends here: unconverged, it flags and restores the antennas whose last
        // two updates have not shrunk by more than a tenth from their first two
        __syncthreads();
        if (s_unconverged) {
            for (int ant = threadIdx.x; ant < u.n_ant; ant += blockDim.x) {
                const size_t pidx = (size_t)bin * u.n_ant + ant;
                const double *ds = u.div_stats + 2 * pidx;
                if (!(ds[0] > 0 && ds[1] >= 0.9 * ds[0])) continue;
                double2 g0[4];
                if (u.type == 2) {
                    const double *phi0 = u.params0 + 2 * pidx;
                    double *phi = u.params + 2 * pidx;
                    for (int e = 0; e < 2; ++e) phi[e] = phi0[e];
                    double sn, cs;
                    sincos(phi0[0], &sn, &cs);
                    g0[0] = make_double2(cs, sn);
                    sincos(phi0[1], &sn, &cs);
                    g0[3] = make_double2(cs, sn);
                    g0[1] = g0[2] = make_double2(0, 0);
                } else {
                    const double2 *P0 = reinterpret_cast<const double2 *>(u.params0) + 4 * pidx;
                    double2 *P = reinterpret_cast<double2 *>(u.params) + 4 * pidx;
                    for (int e = 0; e < 4; ++e) { g0[e] = P0[e]; P[e] = P0[e]; }
                }
                store_jones_tab(u, bin, ant, g0);
                if (u.gain_flags) u.gain_flags[pidx] = 2;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// residual and chi^2 (Eq. min): full chain, row tiles, FP64 block sums
// ---------------------------------------------------------------------------

struct ResArgs {
    Data D;
    Chain C;              // n = -1: product of all terms
    float4 *resid;        // [n_row][n_chan] x 2, or nullptr
    double *chi2;         // one double
};

template <bool M16>
__global__ void __launch_bounds__(256) residual_kernel(const ResArgs a)
{
    const Data &D = a.D;
    const Chain &C = a.C;
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long n_warps = ((long)gridDim.x * blockDim.x) >> 5;
    const int n_chunks = (D.n_chan + 31) / 32;
    double tot = 0.0;
    for (long u = warp; u < (long)D.n_row * n_chunks; u += n_warps) {
        const int row = (int)(u / n_chunks);
        const int c = (int)(u % n_chunks) * 32 + lane;
        if (c >= D.n_chan) continue;
        const int4 meta = __ldg(D.rows + row);
        const size_t s = (size_t)row * D.n_chan + c;
        bool ok = meta.x != meta.y;
        if (ok && D.flag) ok = __ldg(D.flag + s) == 0;
        if (!ok) {
            if (a.resid) { a.resid[2 * s] = make_float4(0, 0, 0, 0); a.resid[2 * s + 1] = make_float4(0, 0, 0, 0); }
            continue;
        }
        J2 Cp = j_identity(), Cq = j_identity();
        for (int j = 0; j < C.n_terms; ++j) {
            const DevTerm &T = C.t[j];
            const int tint = __ldg(T.t_map + meta.z), fint = __ldg(T.f_map + c);
            Cp = j_mul(Cp, fetch_jones(T, C.n_ant, tint, fint, meta.x));
            Cq = j_mul(Cq, fetch_jones(T, C.n_ant, tint, fint, meta.y));
        }
        J2 M;
        if constexpr (M16) {
            const uint4 h = __ldg(D.model16 + s);
            const float sc = __ldg(D.bl_scale + meta.w);
            M.a = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.x)), sc);
            M.b = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.y)), sc);
            M.c = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.z)), sc);
            M.d = cscale(h2f(*reinterpret_cast<const __half2 *>(&h.w)), sc);
        } else {
            M = j_from(__ldg(D.model + 2 * s), __ldg(D.model + 2 * s + 1));
        }
        const J2 V = j_mul_h(j_mul(Cp, M), Cq);
        const J2 Dm = j_from(__ldg(D.vis + 2 * s), __ldg(D.vis + 2 * s + 1));
        J2 r;
        r.a = csub(Dm.a, V.a); r.b = csub(Dm.b, V.b); r.c = csub(Dm.c, V.c); r.d = csub(Dm.d, V.d);
        const float4 w = __ldg(D.weight + s);
        tot += (double)(w.x * cnorm2(r.a)) + (double)(w.y * cnorm2(r.b)) + (double)(w.z * cnorm2(r.c)) +
               (double)(w.w * cnorm2(r.d));
        if (a.resid) {
            a.resid[2 * s] = make_float4(r.a.x, r.a.y, r.b.x, r.b.y);
            a.resid[2 * s + 1] = make_float4(r.c.x, r.c.y, r.d.x, r.d.y);
        }
    }
    for (int d = 16; d > 0; d >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, d);
    __shared__ double part[8];
    if (lane == 0) part[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < (int)blockDim.x / 32; ++i) t += part[i];
        atomicAdd(a.chi2, t);
    }
}

// ---------------------------------------------------------------------------
// per-bin sample counts of a term (for the throughput and byte accounting)
// ---------------------------------------------------------------------------

struct CountArgs {
    Data D;
    const int *t_map, *f_map;
    int n_fint;
    long long *nvis;        // [n_bins] cross-correlation samples
    long long *nunflag;     // [n_bins] unflagged cross-correlation samples
};

static __global__ void __launch_bounds__(256) count_kernel(const CountArgs a)
{
    const Data &D = a.D;
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long n_warps = ((long)gridDim.x * blockDim.x) >> 5;
    const int n_chunks = (D.n_chan + 31) / 32;
    for (long row = warp; row < D.n_row; row += n_warps) {
        const int4 meta = __ldg(D.rows + row);
        if (meta.x == meta.y) continue;
        const int tint = __ldg(a.t_map + meta.z);
        for (int ch = 0; ch < n_chunks; ++ch) {
            const int c = ch * 32 + lane;
            const bool in = c < D.n_chan;
            const int key = in ? tint * a.n_fint + __ldg(a.f_map + c) : -1;
            const bool unf = in && (!D.flag || __ldg(D.flag + (size_t)row * D.n_chan + c) == 0);
            const unsigned m = __match_any_sync(0xffffffffu, key);
            const unsigned mu = m & __ballot_sync(0xffffffffu, unf);
            if (in && lane == __ffs(m) - 1) {
                atomicAdd((unsigned long long *)(a.nvis + key), (unsigned long long)__popc(m));
                if (mu) atomicAdd((unsigned long long *)(a.nunflag + key), (unsigned long long)__popc(mu));
            }
        }
    }
}

} // namespace qc

namespace qc {

// ---------------------------------------------------------------------------
// pipelined accumulate kernel: bulk-copy producer warp + consumer warps
// ---------------------------------------------------------------------------
//
// The CTA owns groups of NW work units (a unit is one row for row tiles, or
// one baseline strip x 32 channels for strip tiles); consumer warp w always
// takes slot w of the group, so its register partial sums follow one row or
// one strip.  For every step the producer warp copies, per slot, the row
// segment [c0, c0 + 32) of d, m and w (contiguous in [row][chan][corr]) into
// one stage of an NS-deep shared-memory ring with cp.async.bulk, completing
// the transaction count of that stage's "full" mbarrier; consumers wait on
// it, compute from shared memory and release the stage through its "empty"
// mbarrier.  Row segments that are fully flagged, autocorrelations, or whose
// intervals have all converged are not copied at all.  Every wait is bounded
// in wall time; a timeout sets *err and the CTA leaves after waiting (again
// bounded) for its copies in flight.

struct PipeArgs {
    AccArgs a;
    const int4 *row_info;         // [n_row] {p, q, tn, to}; tn = -1 for rows without usable data
    const int4 *chunk_info;       // [n_chunks] {fn0, fn count, fo0, fo count} of the 32-channel chunks
    const uint8_t *chunk_active;  // [n_tint of term n][n_chunks]: a 32-channel chunk has an active bin
    int *err;                     // set to 1 when a bounded wait gives up
    unsigned long long wait_ns;   // wall-time limit of every wait on a stage barrier
    int stall_issue;              // tests: the n-th issue of every warp is never made (-1: none)
    // shared-memory layout (bytes), fixed per launch by the host
    int ns;                       // ring stages per warp
    int slot_bytes;               // one stage of one warp: d, m, w and Jones slices
    int off_m, off_w, off_jn, off_jo;   // offsets inside a slot
    int jn_cap, jo_cap;           // Jones entries per antenna for the solved / other term
    int warp_bytes;               // ring + descriptors + barriers of one warp
    int desc_off, bar_off;        // offsets inside a warp's area
    int fmap_off;                 // f_maps of both terms (stage_fmap)
    int stage_fmap;
};


// Descriptor of one row segment of a warp's step (written when its copies are issued).
struct __align__(16) SlotDesc {
    int row, cc, nch, live;       // row segment [cc, cc + nch) of `row`; live = data copied
    int p, q, tn, pad0;           // antennas, time-interval index of the solved term
    int fn0, fo0;                 // first frequency-interval index of the staged Jones slices
    float scale;                  // per-baseline model scale (FP16 model)
    int pad1;
};

template <int K> __device__ __forceinline__ J2 smem_jones(const unsigned char *base, int i)
{
    if constexpr (K == KIND_FULL) {
        const float4 *v = reinterpret_cast<const float4 *>(base) + 2 * i;
        return j_from(v[0], v[1]);
    } else {
        return j_diag(reinterpret_cast<const float4 *>(base)[i]);
    }
}

// Position in a warp's stream of steps: unit u (a row for row tiles, a strip x
// 32-channel chunk for strip tiles), step i of len; a step covers H row segments.
struct Cursor {
    long u;
    int i, len, beg, c0, n_seg;
};

template <int H>
__device__ __forceinline__ void cursor_unit(const AccArgs &a, Cursor &k, long n_units)
{
    k.i = 0;
    k.len = 0;
    if (k.u >= n_units) return;
    if (a.order == 0) { k.n_seg = a.n_chunks; k.beg = 0; k.c0 = 0; }
    else {
        const int s = (int)(k.u / a.n_chunks);
        k.c0 = (int)(k.u % a.n_chunks) * 32;
        k.beg = __ldg(a.D.strip_off + s);
        k.n_seg = __ldg(a.D.strip_off + s + 1) - k.beg;
    }
    k.len = (k.n_seg + H - 1) / H;
}

template <int H>
__device__ __forceinline__ void cursor_next(const AccArgs &a, Cursor &k, long n_units, long stride)
{
    if (++k.i < k.len) return;
    do {
        k.u += stride;
        cursor_unit<H>(a, k, n_units);
    } while (k.u < n_units && k.len == 0);
}

// Pipelined accumulate kernel for chains of one or two terms.
//
// Every warp streams through its own work units (a unit is one row for row
// tiles, or one baseline strip x 32 channels for strip tiles) and keeps its
// register partial sums for the unit's antennas.  A step covers H row segments
// of 32 channels (consecutive channel chunks of a row, or consecutive rows of a
// strip).  Each warp owns an NS-deep ring of shared-memory stages with one
// mbarrier per stage: NS - 1 steps ahead of the step it computes, its lanes
// issue cp.async.bulk copies (one per lane) of the segments of d, m and w
// (contiguous in [row][chan][corr]) and of the slices of both terms' Jones
// tables that each segment touches for antennas p and q (contiguous in the
// [tint][ant][fint] table layout), completing the stage's transaction count.
// The sample arithmetic then reads shared memory only.  Segments that are fully
// flagged, autocorrelations, or whose intervals have all converged are not
// copied.  Warps never wait on each other; every wait on a stage barrier is
// bounded in wall time (a timeout sets *err, and the warp leaves after waiting,
// again bounded, for its own copies in flight).
template <int TS, int LK, int RK, bool M16, int NW, int H>
__global__ void __launch_bounds__(NW * 32, 1) acc_pipe_kernel(const PipeArgs P)
{
    constexpr bool HAS_L = LK != KIND_NONE;
    constexpr bool KAHAN = M16;
    using Lay = AccLayout<TS, HAS_L>;
    constexpr int KR = Lay::KR, KG = Lay::KG;
    constexpr int MB = M16 ? 16 : 32;
    constexpr int GK = TS == TS_FULL ? KIND_FULL : KIND_DIAG;
    constexpr int OK_ = LK != KIND_NONE ? LK : RK;          // kind of the other term (NONE: single term)
    constexpr int ESN = GK == KIND_FULL ? 32 : 16;
    constexpr int ESO = OK_ == KIND_FULL ? 32 : 16;
    constexpr int NCOPY = OK_ != KIND_NONE ? 7 : 5;         // bulk copies per row segment
    static_assert(H * 8 <= 32, "one lane per copy");
    extern __shared__ __align__(128) unsigned char smem[];
    const AccArgs &a = P.a;
    const Data &D = a.D;
    const DevTerm &Tn = a.tn;
    const DevTerm &To = a.to;
    const int n_ant = a.C.n_ant;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + (size_t)warp * P.warp_bytes;
    SlotDesc *desc = reinterpret_cast<SlotDesc *>(wbase + P.desc_off);
    uint64_t *full = reinterpret_cast<uint64_t *>(wbase + P.bar_off);
    const int *sfn = reinterpret_cast<const int *>(smem + P.fmap_off);
    const int *sfo = sfn + D.n_chan;

    if (__ldg(a.n_active) == 0) return;
    if (P.stage_fmap) {
        int *wfn = reinterpret_cast<int *>(smem + P.fmap_off);
        for (int c = threadIdx.x; c < D.n_chan; c += blockDim.x) {
            wfn[c] = __ldg(Tn.f_map + c);
            if constexpr (OK_ != KIND_NONE) wfn[D.n_chan + c] = __ldg(To.f_map + c);
        }
    }
    if (lane == 0) {
        for (int s = 0; s < P.ns; ++s) mbar_init(full + s, 1);
        fence_barrier_init();
    }
    __syncthreads();

    // the copy this lane issues for each step: segment `hseg`, kind `kind`
    const int hseg = lane >> 3, kind = lane & 7;
    const bool copier = hseg < H && kind < NCOPY;
    const unsigned char *cbase;
    uint32_t cdst, ces;
    {
        const unsigned char *tb_n = reinterpret_cast<const unsigned char *>(Tn.tab);
        const unsigned char *tb_o = reinterpret_cast<const unsigned char *>(To.tab);
        const uint32_t seg_off = hseg * P.slot_bytes;
        switch (kind) {
        case 0: cbase = reinterpret_cast<const unsigned char *>(D.vis); cdst = seg_off; ces = 32; break;
        case 1: cbase = M16 ? reinterpret_cast<const unsigned char *>(D.model16) : reinterpret_cast<const unsigned char *>(D.model);
                cdst = seg_off + P.off_m; ces = MB; break;
        case 2: cbase = reinterpret_cast<const unsigned char *>(D.weight); cdst = seg_off + P.off_w; ces = 16; break;
        case 3: cbase = tb_n; cdst = seg_off + P.off_jn; ces = ESN; break;
        case 4: cbase = tb_n; cdst = seg_off + P.off_jn + P.jn_cap * ESN; ces = ESN; break;
        case 5: cbase = tb_o; cdst = seg_off + P.off_jo; ces = ESO; break;
        default: cbase = tb_o; cdst = seg_off + P.off_jo + P.jo_cap * ESO; ces = ESO; break;
        }
    }

    const long n_units = a.order == 0 ? (long)D.n_row : (long)D.n_strips * a.n_chunks;
    const long stride = (long)gridDim.x * NW;
    Cursor ck, pf;                 // compute cursor, prefetch cursor
    ck.u = (long)blockIdx.x * NW + warp;
    cursor_unit<H>(a, ck, n_units);
    if (ck.u < n_units && ck.len == 0) cursor_next<H>(a, ck, n_units, stride);
    pf = ck;
    uint32_t n_issued = 0;
    int is_stage = 0;              // stage of the next issue

    // issue the copies of the step under cursor k into the next stage
    auto issue = [&](const Cursor &k) {
        const int stage = is_stage;
        // every lane describes segment h = lane >> 3 (lanes of a segment agree)
        SlotDesc d;
        d.row = -1; d.cc = 0; d.nch = 0; d.live = 0;
        d.p = 0; d.q = 0; d.tn = 0; d.pad0 = 0; d.fn0 = 0; d.fo0 = 0; d.scale = 1.f; d.pad1 = 0;
        int cn = 0, co = 0, to = 0;
        const int seg = k.i * H + hseg;
        if (hseg < H && seg < k.n_seg) {
            d.row = a.order == 0 ? (int)k.u : __ldg(D.strip_rows + k.beg + seg);
            d.cc = a.order == 0 ? seg * 32 : k.c0;
            d.nch = min(32, D.n_chan - d.cc);
            const int4 ri = __ldg(P.row_info + d.row);
            if (ri.z >= 0 && __ldg(P.chunk_active + (size_t)ri.z * a.n_chunks + d.cc / 32)) {
                const int4 ci = __ldg(P.chunk_info + d.cc / 32);
                d.live = 1;
                d.p = ri.x; d.q = ri.y; d.tn = ri.z; to = ri.w;
                d.fn0 = ci.x; cn = ci.y;
                d.fo0 = ci.z; co = ci.w;
                if constexpr (M16) d.scale = __ldg(D.bl_scale + __ldg(D.rows + d.row).w);
            }
        }
        uint32_t seg_bytes = 0;
        if (d.live) {
            seg_bytes = (uint32_t)d.nch * (32u + MB + 16u) + 2u * cn * ESN;
            if constexpr (OK_ != KIND_NONE) seg_bytes += 2u * co * ESO;
        }
        // total over the step's segments: lane 8h holds segment h
        uint32_t total = 0;
#pragma unroll
        for (int h = 0; h < H; ++h) total += __shfl_sync(0xffffffffu, seg_bytes, 8 * h);
        if (kind == 0 && hseg < H) desc[stage * H + hseg] = d;
        __syncwarp();
        // a test can leave one stage's barrier without its arrival: the wait on it must give up
        const bool stalled = (int)n_issued == P.stall_issue;
        if (lane == 0 && !stalled) mbar_arrive_expect_tx(full + stage, total);
        __syncwarp();
        if (copier && d.live && !stalled) {
            size_t idx;
            uint32_t n;
            if (kind < 3) { idx = (size_t)d.row * D.n_chan + d.cc; n = d.nch; }
            else if (kind < 5) { idx = ((size_t)d.tn * n_ant + (kind == 3 ? d.p : d.q)) * Tn.n_fint + d.fn0; n = cn; }
            else { idx = ((size_t)to * n_ant + (kind == 5 ? d.p : d.q)) * To.n_fint + d.fo0; n = co; }
            bulk_copy_g2s(wbase + (size_t)stage * H * P.slot_bytes + cdst, cbase + idx * ces, n * ces, full + stage);
        }
        ++n_issued;
        if (++is_stage == P.ns) is_stage = 0;
    };

    // prime the ring
    for (int s = 0; s < P.ns - 1 && pf.u < n_units; ++s) {
        issue(pf);
        cursor_next<H>(a, pf, n_units, stride);
    }

    Acc<KR, KAHAN> Ap, Aq;
    Ap.zero();
    Aq.zero();
    uint32_t n_done = 0;
    int stage = 0;                 // stage of the step being computed
    uint32_t phase = 0;            // parity of that stage's current use
    int cur_key = -1, p = 0, q = 0;
    bool failed = false;
    while (ck.u < n_units) {
        if (pf.u < n_units) {
            issue(pf);
            cursor_next<H>(a, pf, n_units, stride);
        }
        if (!mbar_wait_bounded(full + stage, phase, P.wait_ns)) { failed = true; break; }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const SlotDesc d = desc[stage * H + h];
            if (!d.live) continue;
            p = d.p;
            q = d.q;
            const int c = d.cc + lane;
            const bool in_range = lane < d.nch;
            int fn = 0, fo = 0;
            if (in_range) {
                fn = P.stage_fmap ? sfn[c] : __ldg(Tn.f_map + c);
                if constexpr (OK_ != KIND_NONE) fo = P.stage_fmap ? sfo[c] : __ldg(To.f_map + c);
            }
            const int key = in_range ? d.tn * Tn.n_fint + fn : -1;
            if (__any_sync(0xffffffffu, cur_key >= 0 && key != cur_key)) {
                const unsigned m = __match_any_sync(0xffffffffu, cur_key);
                const unsigned seg_end = 32 - __clz(m);
                const bool head = lane == __ffs(m) - 1;
                const bool live = cur_key >= 0 && __ldg(a.active + cur_key);
                flush_side<KR, KG, KAHAN, Lay>(Ap, cur_key, p, lane, seg_end, head, live, a.acc, n_ant);
                flush_side<KR, KG, KAHAN, Lay>(Aq, cur_key, q, lane, seg_end, head, live, a.acc, n_ant);
            }
            cur_key = key;
            bool ok = in_range && __ldg(a.active + key);
            if (ok && D.flag) ok = __ldg(D.flag + (size_t)d.row * D.n_chan + c) == 0;
            if (ok) {
                const unsigned char *sb = wbase + ((size_t)stage * H + h) * P.slot_bytes;
                const float4 *sd = reinterpret_cast<const float4 *>(sb) + 2 * lane;
                const J2 Dm = j_from(sd[0], sd[1]);
                J2 M;
                if constexpr (M16) M = load_model16(reinterpret_cast<const uint4 *>(sb + P.off_m)[lane], d.scale);
                else {
                    const float4 *sm = reinterpret_cast<const float4 *>(sb + P.off_m) + 2 * lane;
                    M = j_from(sm[0], sm[1]);
                }
                const float4 w = reinterpret_cast<const float4 *>(sb + P.off_w)[lane];
                const J2 Gp = smem_jones<GK>(sb + P.off_jn, fn - d.fn0);
                const J2 Gq = smem_jones<GK>(sb + P.off_jn + P.jn_cap * ESN, fn - d.fn0);
                J2 Op, Oq;
                if constexpr (OK_ != KIND_NONE) {
                    Op = smem_jones<OK_>(sb + P.off_jo, fo - d.fo0);
                    Oq = smem_jones<OK_>(sb + P.off_jo + P.jo_cap * ESO, fo - d.fo0);
                } else {
                    Op = j_identity();
                    Oq = Op;
                }
                sample_math<TS, LK, RK, KAHAN>(Op, Gp, Op, Oq, Gq, Oq, Dm, M, w, Ap, Aq);
            }
        }
        __syncwarp();
        ++n_done;
        if (++stage == P.ns) { stage = 0; phase ^= 1u; }
        const long u_prev = ck.u;
        cursor_next<H>(a, ck, n_units, stride);
        if (ck.u != u_prev) {
            if (__any_sync(0xffffffffu, cur_key >= 0)) {
                // end of the unit
                const unsigned m = __match_any_sync(0xffffffffu, cur_key);
                const unsigned seg_end = 32 - __clz(m);
                const bool head = lane == __ffs(m) - 1;
                const bool live = cur_key >= 0 && __ldg(a.active + cur_key);
                flush_side<KR, KG, KAHAN, Lay>(Ap, cur_key, p, lane, seg_end, head, live, a.acc, n_ant);
                flush_side<KR, KG, KAHAN, Lay>(Aq, cur_key, q, lane, seg_end, head, live, a.acc, n_ant);
            }
            cur_key = -1;
        }
    }
    if (failed) {
        if (lane == 0) atomicExch(P.err, 1);
        // let this warp's copies in flight land before it leaves (bounded)
        for (uint32_t k = n_done; k < n_issued; ++k) {
            mbar_wait_bounded(full + stage, phase, P.wait_ns);
            if (++stage == P.ns) { stage = 0; phase ^= 1u; }
        }
    }
}

// Static per-row information of a term solve: {p, q, tn, to} with tn = -1 for
// rows without an unflagged cross-correlation sample.
static __global__ void row_info_kernel(const Data D, const uint8_t *row_live, const DevTerm tn, const DevTerm to,
                                       int has_o, int4 *out)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.n_row) return;
    const int4 meta = D.rows[i];
    const int t = meta.z;
    int4 r;
    r.x = meta.x;
    r.y = meta.y;
    r.z = row_live[i] ? tn.t_map[t] : -1;
    r.w = has_o ? to.t_map[t] : 0;
    out[i] = r;
}

// chunk_active[tint][chunk] = some interval bin of the solved term touched by this
// (time interval, 32-channel chunk) is still active
static __global__ void chunk_active_kernel(const DevTerm tn, int n_chan, int n_chunks, const uint8_t *active,
                                           const int *n_active, uint8_t *out)
{
    if (*n_active == 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tn.n_tint * n_chunks) return;
    const int tint = i / n_chunks, ch = i % n_chunks;
    const int f0 = tn.f_map[ch * 32], f1 = tn.f_map[min(n_chan, ch * 32 + 32) - 1];
    uint8_t any = 0;
    for (int f = f0; f <= f1 && !any; ++f) any = active[tint * tn.n_fint + f];
    out[i] = any;
}

// row_live[row] = cross-correlation row with at least one unflagged channel
static __global__ void row_live_kernel(const Data D, uint8_t *row_live)
{
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long n_warps = ((long)gridDim.x * blockDim.x) >> 5;
    for (long row = warp; row < D.n_row; row += n_warps) {
        const int4 meta = __ldg(D.rows + row);
        bool any = false;
        if (meta.x != meta.y) {
            for (int c = lane; c < D.n_chan && !any; c += 32)
                any = !D.flag || __ldg(D.flag + (size_t)row * D.n_chan + c) == 0;
        }
        any = __any_sync(0xffffffffu, any);
        if (lane == 0) row_live[row] = any ? 1 : 0;
    }
}

} // namespace qc
