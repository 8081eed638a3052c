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

__device__ __forceinline__ J2 fetch_jones(const DevTerm &T, int n_ant, int tint, int fint, int ant)
{
    const size_t idx = ((size_t)tint * n_ant + ant) * T.n_fint + fint;
    if (T.type == 1) return j_from(__ldg(T.tab + 2 * idx), __ldg(T.tab + 2 * idx + 1));
    return j_diag(__ldg(T.tab + idx));
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
};

// Contribution of one sample to antenna a's blocks: E = L_a (x) X^T (Eq. vectrick,
// Eq. g_derivative_dd) restricted to the term's free parameters, weights w
// per correlation, residual r (both in the orientation of this side).
template <int TS, bool HAS_L, bool KAHAN>
__device__ __forceinline__ void accumulate_side(Acc<AccLayout<TS, HAS_L>::KR, KAHAN> &A, const J2 &L,
                                                const J2 &X, float4 w, const J2 &r)
{
    const float wv[4] = { w.x, w.y, w.z, w.w };
    const float2 rv[4] = { r.a, r.b, r.c, r.d };
    const float2 Xv[4] = { X.a, X.b, X.c, X.d };            // X[l][j] = Xv[2l+j]
    if constexpr (!HAS_L) {
        if constexpr (TS == TS_DIAG) {
            // parameter k in {XX, YY} touches row k of V: E[(k,j), k] = X[k][j]
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                float h = 0.f;
                float2 jr = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float2 x = Xv[2 * k + j];
                    const float ww = wv[2 * k + j];
                    h = fmaf(ww, cnorm2(x), h);
                    jr = cfma_conj(x, cscale(rv[2 * k + j], ww), jr);
                }
                A.add(k, h);
                A.add(2 + 2 * k, jr.x);
                A.add(3 + 2 * k, jr.y);
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
                A.add(2 * k + 0, fmaf(w0, n00, w1 * n01));
                A.add(2 * k + 1, fmaf(w0, n10, w1 * n11));
                const float2 off = make_float2(fmaf(w0, o0.x, w1 * o1.x), fmaf(w0, o0.y, w1 * o1.y));
                A.add(4 + 2 * k, off.x);
                A.add(5 + 2 * k, off.y);
                const float2 wr0 = cscale(rv[2 * k], w0), wr1 = cscale(rv[2 * k + 1], w1);
                const float2 j0 = cfma_conj(x01, wr1, cfma_conj(x00, wr0, make_float2(0.f, 0.f)));
                const float2 j1 = cfma_conj(x11, wr1, cfma_conj(x10, wr0, make_float2(0.f, 0.f)));
                A.add(8 + 4 * k + 0, j0.x);
                A.add(8 + 4 * k + 1, j0.y);
                A.add(8 + 4 * k + 2, j1.x);
                A.add(8 + 4 * k + 3, j1.y);
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
                const float2 wr = cscale(rv[m], wv[m]);
                j0 = cfma_conj(E0[m], wr, j0);
                j1 = cfma_conj(E1[m], wr, j1);
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
                    jr = cfma_conj(E[m][u], cscale(rv[m], wv[m]), jr);
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
// the accumulate kernel
// ---------------------------------------------------------------------------

struct AccArgs {
    Data D;
    Chain C;
    DevTerm tn;              // copy of C.t[C.n] (avoids dynamic indexing of kernel parameters)
    double *acc;             // [n_bins][n_ant][KG]
    const uint8_t *active;   // [n_bins]
    const int *n_active;     // nonzero: some interval of the solved term is still iterating
    int order;               // 0 row tiles, 1 strip tiles
    int n_chunks;            // ceil(n_chan / 32)
};

// Chain factors of antenna a at one sample around the solved term n
// (Eq. jonesfactor): L = prod_{j<n} G_j, G = G_n, R = prod_{j>n} G_j.
template <int LK, int RK>
__device__ __forceinline__ void chain_factors(const Chain &C, const int *tint, int c, int a, J2 &L, J2 &G, J2 &R)
{
    bool hl = false, hr = false;
    L = j_identity();
    R = j_identity();
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {
        if (j >= C.n_terms) break;
        const DevTerm &T = C.t[j];
        const int fint = __ldg(T.f_map + c);
        const J2 J = fetch_jones(T, C.n_ant, tint[j], fint, a);
        if (j < C.n) {
            if constexpr (LK != KIND_NONE) { L = hl ? j_mul(L, J) : J; hl = true; }
        } else if (j == C.n) {
            G = J;
        } else {
            if constexpr (RK != KIND_NONE) { R = hr ? j_mul(R, J) : J; hr = true; }
        }
    }
}

template <int TS, int LK, int RK, bool M16>
__global__ void __launch_bounds__(256) acc_kernel(const AccArgs a)
{
    if (__ldg(a.n_active) == 0) return;
    constexpr bool HAS_L = LK != KIND_NONE;
    constexpr bool KAHAN = M16;
    using Lay = AccLayout<TS, HAS_L>;
    constexpr int KR = Lay::KR, KG = Lay::KG;
    constexpr int GK = TS == TS_FULL ? KIND_FULL : KIND_DIAG;
    const Data &D = a.D;
    const Chain &C = a.C;
    const DevTerm &Tn = a.tn;
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long n_warps = ((long)gridDim.x * blockDim.x) >> 5;
    const long n_units = a.order == 0 ? (long)D.n_row : (long)D.n_strips * a.n_chunks;

    Acc<KR, KAHAN> Ap, Aq;
    Ap.zero();
    Aq.zero();

    for (long u = warp; u < n_units; u += n_warps) {
        int cur_key = -1;
        int p = 0, q = 0;
        long i_beg, i_end;
        int c_fixed = 0;
        if (a.order == 0) { i_beg = 0; i_end = a.n_chunks; }
        else {
            const int s = (int)(u / a.n_chunks);
            c_fixed = (int)(u % a.n_chunks) * 32 + lane;
            i_beg = __ldg(D.strip_off + s);
            i_end = __ldg(D.strip_off + s + 1);
        }
        for (long i = i_beg; i < i_end; ++i) {
            const int row = a.order == 0 ? (int)u : __ldg(D.strip_rows + i);
            const int c = a.order == 0 ? (int)i * 32 + lane : c_fixed;
            const int4 meta = __ldg(D.rows + row);
            p = meta.x;
            q = meta.y;
            if (p == q) break;                       // autocorrelation: whole unit skipped
            const bool in_range = c < D.n_chan;
            int tint[MAXT];
#pragma unroll
            for (int j = 0; j < MAXT; ++j) tint[j] = j < C.n_terms ? __ldg(C.t[j].t_map + meta.z) : 0;
            const int key = in_range ? __ldg(Tn.t_map + meta.z) * Tn.n_fint + __ldg(Tn.f_map + c) : -1;
            // flush when any lane's bin changes
            const bool change = cur_key >= 0 && key != cur_key;
            if (__any_sync(0xffffffffu, change)) {
                const unsigned m = __match_any_sync(0xffffffffu, cur_key);
                const unsigned seg_end = 32 - __clz(m);
                const bool head = lane == __ffs(m) - 1;
                const bool live = cur_key >= 0 && __ldg(a.active + cur_key);
                flush_side<KR, KG, KAHAN, Lay>(Ap, cur_key, p, lane, seg_end, head, live, a.acc, C.n_ant);
                flush_side<KR, KG, KAHAN, Lay>(Aq, cur_key, q, lane, seg_end, head, live, a.acc, C.n_ant);
            }
            cur_key = key;
            const size_t s = (size_t)row * D.n_chan + c;
            bool ok = in_range && __ldg(a.active + key);
            if (ok && D.flag) ok = __ldg(D.flag + s) == 0;
            if (!__any_sync(0xffffffffu, ok)) continue;
            if (!ok) continue;
            // ---- loads (128-bit, contiguous across the warp) ----
            const J2 Dm = j_from(__ldg(D.vis + 2 * s), __ldg(D.vis + 2 * s + 1));
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
            const float4 w = __ldg(D.weight + s);
            // ---- chain factors for both antennas ----
            J2 Lp, Gp, Rp, Lq, Gq, Rq;
            chain_factors<LK, RK>(C, tint, c, p, Lp, Gp, Rp);
            chain_factors<LK, RK>(C, tint, c, q, Lq, Gq, Rq);
            // C_a = L_a G_a R_a
            const J2 Cp = lmulk<LK>(Lp, rmulk<RK>(Gp, Rp));
            const J2 Cq = lmulk<LK>(Lq, rmulk<RK>(Gq, Rq));
            // p side: X = R_p M C_q^H, V = L_p G_p X, r = D - V
            const J2 X = j_mul_h(lmulk<RK>(Rp, M), Cq);
            const J2 V = lmulk<LK>(Lp, lmulk<GK>(Gp, X));
            J2 r;
            r.a = csub(Dm.a, V.a); r.b = csub(Dm.b, V.b); r.c = csub(Dm.c, V.c); r.d = csub(Dm.d, V.d);
            accumulate_side<TS, HAS_L, KAHAN>(Ap, Lp, X, w, r);
            // q side through the conjugate baseline: Y = R_q M^H C_p^H, r' = r^H, w' = P w
            const J2 Y = j_mul_h(lmulk<RK>(Rq, j_herm(M)), Cp);
            const J2 rh = j_herm(r);
            accumulate_side<TS, HAS_L, KAHAN>(Aq, Lq, Y, make_float4(w.x, w.z, w.y, w.w), rh);
        }
        // end of the unit: flush what is left
        {
            const unsigned m = __match_any_sync(0xffffffffu, cur_key);
            const unsigned seg_end = 32 - __clz(m);
            const bool head = lane == __ffs(m) - 1;
            const bool live = cur_key >= 0 && __ldg(a.active + cur_key);
            if (__any_sync(0xffffffffu, cur_key >= 0)) {
                flush_side<KR, KG, KAHAN, Lay>(Ap, cur_key, p, lane, seg_end, head, live, a.acc, C.n_ant);
                flush_side<KR, KG, KAHAN, Lay>(Aq, cur_key, q, lane, seg_end, head, live, a.acc, C.n_ant);
            }
        }
    }
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
    auto cdiv = [](double2 u, double2 v) {
        const double den = v.x * v.x + v.y * v.y;
        return make_double2((u.x * v.x + u.y * v.y) / den, (u.y * v.x - u.x * v.y) / den);
    };
    double trace = 0, anorm = 0;
    for (int i = 0; i < N; ++i) trace += A[i][i].x;
    if (!(trace > 0)) return 1;
    for (int j = 0; j < N; ++j) {
        double s = 0;
        for (int i = 0; i < N; ++i) s += cabs(A[i][j]);
        anorm = fmax(anorm, s);
    }
    int piv[N];
    for (int i = 0; i < N; ++i) piv[i] = i;
    for (int k = 0; k < N; ++k) {
        int m = k;
        for (int i = k + 1; i < N; ++i) if (cabs(A[i][k]) > cabs(A[m][k])) m = i;
        if (cabs(A[m][k]) == 0) return 1;
        if (m != k) {
            for (int j = 0; j < N; ++j) { double2 t = A[k][j]; A[k][j] = A[m][j]; A[m][j] = t; }
            int t = piv[k]; piv[k] = piv[m]; piv[m] = t;
        }
        for (int i = k + 1; i < N; ++i) {
            A[i][k] = cdiv(A[i][k], A[k][k]);
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
            y[i] = cdiv(s, A[i][i]);
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
};

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
        for (int e = 0; e < 4; ++e) {
            const double dx = gnew[e].x - gold[e].x, dy = gnew[e].y - gold[e].y;
            num += dx * dx + dy * dy;
            den += gnew[e].x * gnew[e].x + gnew[e].y * gnew[e].y;
        }
        for (int i = 0; i < KG; ++i) A[i] = 0.0;
    }
    // interval norms: block reduction in FP64
    __shared__ double s_num[4], s_den[4];
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
