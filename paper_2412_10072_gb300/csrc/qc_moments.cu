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
// In both forms JHr = b - JHJ vec(g).  One pass over the data per term solve forms the sums
// (mom_pass_kernel: FP32 per lane, FP64 sums); every iteration forms each antenna's blocks from
// them and the current gains in FP32 (mom_normal_kernel), JHr = b - JHJ g and everything after
// it in FP64, in the update kernel's accumulator layout (a diagonal or phase-only term of the
// full form takes the (0, 3) rows and columns).  An iteration then reads 800 or 208 B per
// (interval, pair) instead of 81 B per sample.
#include "qc_internal.h"

#include <algorithm>
#include <type_traits>

namespace qc {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Two lanes share a sample: lane 2c + k takes channel c of a 16-channel chunk and the
// correlations (k, j), j = 0, 1, i.e. the words of kj = 2k and 2k + 1, kept in registers as
//   [0, 32)  S[2k + (i / 16)][i % 16],   [32, 48)  T[2k + (i - 32) / 8][(i - 32) % 8],
//   48, 49   U[2k], U[2k + 1].
constexpr int MOM_H = 50;

__device__ __forceinline__ int mom_word(int i, int k)
{
    return i < 32 ? 16 * (2 * k + i / 16) + i % 16
                  : (i < 48 ? MOM_T + 8 * (2 * k + (i - 32) / 8) + (i - 32) % 8 : MOM_U + 2 * k + (i - 48));
}

// One sample's terms for correlation row k added to a lane's register sums, full form (all
// indices compile-time constants after unrolling; k selects the data row and the weights; M is
// the sample's X = R_p M R_q^H).
__device__ __forceinline__ void mom_add(float (&acc)[MOM_H], const J2 &D, const J2 &M, float4 w, int k)
{
    const float2 m[4] = { M.a, M.b, M.c, M.d };
    const float2 d[2] = { k ? D.c : D.a, k ? D.d : D.b };
    const float wv[2] = { k ? w.z : w.x, k ? w.w : w.y };
    float diag[4];
    float2 off[6];
#pragma unroll
    for (int u = 0; u < 4; ++u) diag[u] = cnorm2(m[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = u + 1; v < 4; ++v) off[mom_pair(u, v)] = cmulc(m[v], m[u]);   // conj(m_u) m_v
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int s = 16 * j;
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[s + u] = fmaf(wv[j], diag[u], acc[s + u]);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            acc[s + 4 + 2 * i] = fmaf(wv[j], off[i].x, acc[s + 4 + 2 * i]);
            acc[s + 5 + 2 * i] = fmaf(wv[j], off[i].y, acc[s + 5 + 2 * i]);
        }
        const float2 wd = cscale(d[j], wv[j]);
        const int t = 32 + 8 * j;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float2 c = cmulc(wd, m[u]);             // conj(m_u) w d
            acc[t + 2 * u] += c.x;
            acc[t + 2 * u + 1] += c.y;
        }
        acc[48 + j] = fmaf(wv[j], cnorm2(d[j]), acc[48 + j]);
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
            const float2 c = cmulc(cscale(d[kj], wv[kj]), e);           // conj(e) w d
            acc[16 + 2 * kj] += c.x;
            acc[17 + 2 * kj] += c.y;
        } else {
            // sqrt(w) E_kj: S' += conj(e_u) e_v, T' += conj(e_u) sqrt(w) d
            const float sw = sqrtf(wv[kj]);
            float2 e[4];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
                    e[2 * a + b] = cscale(cmul(lp[2 * k + a], cmulc(m[2 * a + b], lq[2 * j + b])), sw);
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(e[u].x, e[u].x, fmaf(e[u].y, e[u].y, acc[u]));
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = u + 1; v < 4; ++v) {
                    const float2 c = cmulc(e[v], e[u]);                 // conj(e_u) e_v
                    acc[4 + 2 * mom_pair(u, v)] += c.x;
                    acc[5 + 2 * mom_pair(u, v)] += c.y;
                }
            const float2 ds = cscale(d[kj], sw);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 c = cmulc(ds, e[u]);
                acc[16 + 2 * u] += c.x;
                acc[17 + 2 * u] += c.y;
            }
        }
        acc[24] = fmaf(wv[kj], cnorm2(d[kj]), acc[24]);
    }
}

// register word -> word of the slot: full form (two lanes per sample, part k = lane & 1), and
// the diagonal form (one lane per sample, the same order)
struct FullWord {
    __device__ __forceinline__ int operator()(int i, int k) const { return mom_word(i, k); }
};
struct DiagWord {
    __device__ __forceinline__ int operator()(int i, int) const { return i; }
};

// Add the warp's register sums to the FP64 sums of each key (-1: nothing) and zero them.  LPS
// lanes share a sample (lanes of one part hold the same words), so every reduction runs over
// lane offsets LPS .. 16:
//  - one key for the warp: a reduce-scatter (NW words padded to P = a power of two; after the
//    halvings at offsets 16 .. LPS lane L holds words F (L / LPS) .. + F - 1, F = P LPS / 32),
//    then one atomic per word;
//  - a distinct key per sample: each lane adds its own words;
//  - otherwise: a segmented reduction per word over the run of equal keys (channel intervals
//    are contiguous, so a run is a range of lanes), added by the run's first sample.
template <int NW, int LPS, typename WordOf>
__device__ __forceinline__ void mom_flush(float (&acc)[NW], int key, int lane, double *mom, int stride, WordOf word)
{
    constexpr int P = NW <= 32 ? 32 : (NW <= 64 ? 64 : 128);
    constexpr int F = P * LPS / 32;
    const int k = lane & (LPS - 1);
    const int k0 = __shfl_sync(FULL_MASK, key, 0);
    if (__all_sync(FULL_MASK, key == k0)) {
        if (k0 >= 0) {
            // in place: after the halving at offset o the live words are acc[0 .. h)
#pragma unroll
            for (int h = P / 2, o = 16; o >= LPS; h >>= 1, o >>= 1) {
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
            double *dst = mom + (size_t)k0 * stride;
            const int base = F * (lane / LPS);
#pragma unroll
            for (int j = 0; j < F; ++j)
                if (base + j < NW) atomicAdd(dst + word(base + j, k), (double)acc[j]);
        }
    } else {
        const unsigned m = __match_any_sync(FULL_MASK, key);
        const unsigned own = ((1u << LPS) - 1u) << (lane & ~(LPS - 1));
        if (__all_sync(FULL_MASK, m == own)) {
            if (key >= 0) {
                double *dst = mom + (size_t)key * stride;
#pragma unroll
                for (int v = 0; v < NW; ++v) atomicAdd(dst + word(v, k), (double)acc[v]);
            }
        } else {
            const int seg_end = 32 - __clz(m);
            const bool head = (lane / LPS) == ((__ffs(m) - 1) / LPS);
            double *dst = mom + (size_t)(key >= 0 ? key : 0) * stride;
#pragma unroll
            for (int v = 0; v < NW; ++v) {
                float x = acc[v];
#pragma unroll
                for (int d = LPS; d < 32; d <<= 1) {
                    const float o = __shfl_down_sync(FULL_MASK, x, d);
                    if (lane + d < seg_end) x += o;
                }
                if (head && key >= 0) atomicAdd(dst + word(v, k), (double)x);
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

// a streamed 16-byte load: read-only for the kernel's lifetime, not kept in L1
__device__ __forceinline__ float4 ld_stream(const float4 *p)
{
    float4 r;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}

// one sample as loaded: its key, folded weights, the raw data and model quads, and the fixed
// term's table entries for p ([0, 2)) and q ([2, 4))
struct MomSample {
    int key;
    float4 w, d0, d1, m0, m1;
    float4 o[4];
};

template <int K>
__device__ __forceinline__ void fac_load(const DevTerm &T, int n_ant, int ti, int fi, int ant, float4 *o)
{
    const size_t idx = ((size_t)ti * n_ant + ant) * T.n_fint + fi;
    if constexpr (K == KIND_FULL) {
        o[0] = __ldg(T.tab + 2 * idx);
        o[1] = __ldg(T.tab + 2 * idx + 1);
    } else if constexpr (K == KIND_DIAG) {
        o[0] = __ldg(T.tab + idx);
    }
}

template <int K>
__device__ __forceinline__ J2 fac_jones(const float4 *o)
{
    if constexpr (K == KIND_FULL) return j_from(o[0], o[1]);
    else if constexpr (K == KIND_DIAG) return j_diag(o[0]);
    else return j_identity();
}

template <int CW, int OK>
__device__ __forceinline__ MomSample mom_load(const MomArgs &a, const int4 &mr, int ch, int lane_ch)
{
    MomSample x;
    const int c = ch * CW + lane_ch;
    const bool in = c < a.n_chan;
    x.key = in ? (__ldg(a.tn.t_map + mr.y) * a.tn.n_fint + __ldg(a.tn.f_map + c)) * a.n_up + (mr.z & 0x7fffffff)
               : -1;
    if (in && mr.x >= 0) {
        const size_t i = (size_t)mr.x * a.n_chan + c;
        x.w = ld_stream(a.wf + i);
        x.d0 = ld_stream(a.vis + 2 * i);
        x.d1 = ld_stream(a.vis + 2 * i + 1);
        x.m0 = ld_stream(a.model + 2 * i);
        x.m1 = ld_stream(a.model + 2 * i + 1);
        if constexpr (OK != KIND_NONE) {
            const int ti = __ldg(a.to.t_map + mr.y), fi = __ldg(a.to.f_map + c);
            fac_load<OK>(a.to, a.n_ant, ti, fi, mr.w & 0xffff, x.o);
            fac_load<OK>(a.to, a.n_ant, ti, fi, mr.w >> 16, x.o + 2);
        }
    } else {
        x.w = make_float4(0.f, 0.f, 0.f, 0.f);
        x.d0 = x.d1 = x.m0 = x.m1 = x.w;
        if constexpr (OK != KIND_NONE) x.o[0] = x.o[1] = x.o[2] = x.o[3] = x.w;
    }
    return x;
}

// One pass: warps walk units of a baseline strip (the rows of one ordered baseline in time
// order) x a group of chunks (16 channels in the full form, two lanes per sample; 32 in the
// diagonal form), a row's chunks inside each row or, with chunk_major, the rows inside each
// chunk (an interval several times long then keeps its keys), with the next sample's loads in
// flight while the current one is added to the lane's register sums.  The sums are flushed when
// any lane's (interval, pair) key changes.  The fixed term is L (diagonal form) or R (full form)
// of kind OK.
template <int FORM, int OK>
constexpr int mom_pass_ctas() { return (FORM == FORM_FULL && OK != KIND_NONE) ? 2 : 3; }

template <int FORM, int OK>
static __global__ void __launch_bounds__(128, mom_pass_ctas<FORM, OK>()) mom_pass_kernel(const MomArgs a)
{
    constexpr int LPS = FORM == FORM_FULL ? 2 : 1;
    constexpr int NW = FORM == FORM_FULL ? MOM_H : MOM_EW;
    constexpr int CW = 32 / LPS;
    if (__ldg(a.n_active) == 0) return;
    const int lane = threadIdx.x & 31, lane_ch = lane / LPS;
    const int stride = FORM == FORM_FULL ? MOM_N : MOM_E;
    using Word = typename std::conditional<FORM == FORM_FULL, FullWord, DiagWord>::type;
    float acc[NW];
#pragma unroll
    for (int v = 0; v < NW; ++v) acc[v] = 0.f;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long n_warps = ((long)gridDim.x * blockDim.x) >> 5;
    const int n_groups = (a.n_chunks + a.group - 1) / a.group;
    const long n_units = (long)a.n_strips * n_groups;
    const bool cm = a.chunk_major != 0;
    int cur = -1;
    for (long unit = warp; unit < n_units; unit += n_warps) {
        const int s = (int)(unit / n_groups), g = (int)(unit % n_groups);
        const int ch0 = g * a.group, ch1 = min(a.n_chunks, ch0 + a.group);
        const int k0 = __ldg(a.strip_off + s), k1 = __ldg(a.strip_off + s + 1);
        if (k0 >= k1) continue;
        // the unit's steps (row k, chunk ch) in its order
        auto adv = [&](int &k, int &ch) {
            if (cm) { if (++k == k1) { k = k0; ++ch; } }
            else { if (++ch == ch1) { ch = ch0; ++k; } }
        };
        auto valid = [&](int k, int ch) { return cm ? ch < ch1 : k < k1; };
        int k2 = k0, ch2 = ch0;
        adv(k2, ch2);
        int ch = ch0;
        int4 mr = __ldg(a.mrows + k0);
        int4 mr2 = valid(k2, ch2) ? __ldg(a.mrows + k2) : make_int4(-1, 0, 0, 0);
        MomSample cs = mom_load<CW, OK>(a, mr, ch, lane_ch);
        while (true) {
            if (__any_sync(FULL_MASK, cs.key != cur)) {
                mom_flush<NW, LPS>(acc, cur, lane, a.mom, stride, Word());
                cur = cs.key;
            }
            const bool more = valid(k2, ch2);
            int k3 = k2, ch3 = ch2;
            adv(k3, ch3);
            int4 mr3 = make_int4(-1, 0, 0, 0);
            MomSample ns;
            if (more) {
                if (valid(k3, ch3)) mr3 = __ldg(a.mrows + k3);
                ns = mom_load<CW, OK>(a, mr2, ch2, lane_ch);
            }
            if (cs.w.x != 0.f || cs.w.y != 0.f || cs.w.z != 0.f || cs.w.w != 0.f) {
                J2 D = j_from(cs.d0, cs.d1), M = j_from(cs.m0, cs.m1);
                float4 w = cs.w;
                if (mr.z < 0) {                  // the conjugate baseline: D -> D^H, M -> M^H, w permuted
                    D = j_herm(D);
                    M = j_herm(M);
                    w = make_float4(w.x, w.z, w.y, w.w);
                }
                if constexpr (FORM == FORM_FULL) {
                    if constexpr (OK == KIND_DIAG)
                        M = j_muld(j_dmul(make_float2(cs.o[0].x, cs.o[0].y), make_float2(cs.o[0].z, cs.o[0].w), M),
                                   make_float2(cs.o[2].x, -cs.o[2].y), make_float2(cs.o[2].z, -cs.o[2].w));
                    else if constexpr (OK == KIND_FULL)
                        M = j_mul_h(j_mul(fac_jones<OK>(cs.o), M), fac_jones<OK>(cs.o + 2));
                    mom_add(acc, D, M, w, lane & 1);
                } else {
                    mom_add_e<OK>(acc, D, M, fac_jones<OK>(cs.o), fac_jones<OK>(cs.o + 2), w);
                }
            }
            if (!more) break;
            cs = ns;
            mr = mr2;
            mr2 = mr3;
            k2 = k3;
            ch2 = ch3;
        }
    }
    mom_flush<NW, LPS>(acc, cur, lane, a.mom, stride, Word());
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
// element (u, v) of the Hermitian S block kj of a slot, in FP32 (u, v compile-time after unrolling)
__device__ __forceinline__ float2 slot_S(const double *Mo, int kj, int u, int v)
{
    const double *s = Mo + 16 * kj;
    if (u == v) return make_float2((float)__ldg(s + u), 0.f);
    const int i = u < v ? mom_pair(u, v) : mom_pair(v, u);
    const double2 x = __ldg(reinterpret_cast<const double2 *>(s + 4 + 2 * i));
    return u < v ? make_float2((float)x.x, (float)x.y) : make_float2((float)x.x, -(float)x.y);
}

__device__ __forceinline__ float2 slot_T(const double *Mo, int kj, int u)
{
    const double2 x = __ldg(reinterpret_cast<const double2 *>(Mo + MOM_T + 8 * kj + 2 * u));
    return make_float2((float)x.x, (float)x.y);
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
        const double *Mo = A.mom + ((size_t)bin * A.n_up + up) * MOM_N;
        double2 Gd[4];
        gains_of(A, bin, o, Gd);
        float2 G[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) G[e] = f2(Gd[e]);
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
                const int kj = p_side ? 2 * k + j : 2 * j + k;
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
                                const float2 sv = p_side ? slot_S(Mo, kj, 2 * l + m, 2 * l2 + m2)
                                                         : cconj(slot_S(Mo, kj, 2 * m + l, 2 * m2 + l2));
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
                        const float2 tv = p_side ? slot_T(Mo, kj, 2 * l + m) : cconj(slot_T(Mo, kj, 2 * m + l));
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
        const double *Mo = A.mom + ((size_t)bin * A.n_up + up) * MOM_E;
        double2 Gd[4];
        gains_of(A, bin, o, Gd);
        const float2 g[2] = { f2(Gd[0]), f2(Gd[3]) };
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
                        const float2 sv = p_side ? slot_S(Mo, 0, 2 * x + y, 2 * x2 + y2)
                                                 : cconj(slot_S(Mo, 0, 2 * y + x, 2 * y2 + x2));
                        const float2 t = cmul(gg, sv);
                        hh[x + x2].x += t.x;
                        hh[x + x2].y += t.y;
                    }
#pragma unroll
            for (int y = 0; y < 2; ++y) {
                const double2 tv = __ldg(reinterpret_cast<const double2 *>(Mo + MOM_ET) + (p_side ? 2 * x + y : 2 * y + x));
                const float2 tf = p_side ? make_float2((float)tv.x, (float)tv.y) : make_float2((float)tv.x, -(float)tv.y);
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
cudaError_t mom_launch_pass(const qc::MomArgs &a, int form, int ok, int sm_count, cudaStream_t st)
{
    using namespace qc;
    const int block = 128;                       // two or three CTAs per SM (register-bound)
    const int n_groups = (a.n_chunks + a.group - 1) / a.group;
    const long units = (long)a.n_strips * n_groups;
    auto grid = [&](int per_sm) {
        return (int)std::max(1L, std::min((long)sm_count * per_sm, (units * 32 + block - 1) / block));
    };
    if (form == FORM_FULL) {
        if (ok == KIND_NONE)
            mom_pass_kernel<FORM_FULL, KIND_NONE><<<grid(mom_pass_ctas<FORM_FULL, KIND_NONE>()), block, 0, st>>>(a);
        else if (ok == KIND_DIAG)
            mom_pass_kernel<FORM_FULL, KIND_DIAG><<<grid(mom_pass_ctas<FORM_FULL, KIND_DIAG>()), block, 0, st>>>(a);
        else
            mom_pass_kernel<FORM_FULL, KIND_FULL><<<grid(mom_pass_ctas<FORM_FULL, KIND_FULL>()), block, 0, st>>>(a);
    } else {
        if (ok == KIND_DIAG)
            mom_pass_kernel<FORM_E, KIND_DIAG><<<grid(mom_pass_ctas<FORM_E, KIND_DIAG>()), block, 0, st>>>(a);
        else if (ok == KIND_FULL)
            mom_pass_kernel<FORM_E, KIND_FULL><<<grid(mom_pass_ctas<FORM_E, KIND_FULL>()), block, 0, st>>>(a);
        else
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
