// qc_moments.cu -- sufficient statistics for a single-term chain (the solve from per-baseline
// sums; not in the paper).
//
// When the solved term is the only term of the chain, its gains are constant over each
// solution interval, so every sample of a baseline (p, q) in an interval enters J^H W J and
// J^H W r (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified) through gain-free sums of that
// (interval, baseline).  With the weight index kj = 2k + j of correlation (k, j) and the
// row-major index u = 2l + m of the model entry M_lm (rows with p > q through their conjugate
// baseline, so the sums are kept per unordered pair p < q):
//     S[kj][u][v] = sum w_kj conj(M_u) M_v   (Hermitian; 16 reals per kj)
//     T[kj][u]    = sum w_kj conj(M_u) D_kj   (16 complex)
//     U[kj]       = sum w_kj |D_kj|^2          (4 reals)
// one pass over the data forms them (mom_pass_kernel: FP32 per lane, FP64 sums), and every
// iteration forms each antenna's 4x4 block from them and the current gains in FP32, with
// JHr = b - JHJ vec(G) and everything after it in FP64 (mom_normal_kernel):
//     JHJ_p[(k,l),(k,l')] += sum_j sum_m sum_m' G_q,jm conj(G_q,jm') S[kj][(l,m)][(l',m')]
//     b_p[(k,l)]          += sum_j sum_m G_q,jm T[kj][(l,m)]
//     JHJ_q[(k,l),(k,l')] += sum_j sum_m sum_m' G_p,jm conj(G_p,jm') conj(S[jk][(m,l)][(m',l')])
//     b_q[(k,l)]          += sum_j sum_m G_p,jm conj(T[jk][(m,l)])
//     JHr = b - JHJ vec(G)
// written in the accumulator layout of the update kernel (a diagonal or phase-only term takes
// the (0, 3) rows and columns).  An iteration then reads 800 B per (interval, baseline)
// instead of 81 B per sample.
#include "qc_internal.h"

#include <algorithm>

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

// One sample's terms for correlation row k added to a lane's register sums (all indices
// compile-time constants after unrolling; k selects the data row and the weights).
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

// Add the warp's register sums to the FP64 sums of each lane pair's key (-1: nothing) and zero
// them.  Lanes of one parity hold the same words, so every reduction runs over lane offsets
// 2, 4, 8, 16:
//  - one key for the warp (an interval at least 16 channels wide): a reduce-scatter (words
//    padded to 64; after halving at offsets 16, 8, 4, 2 lane L holds words 4 (L >> 1) .. + 3),
//    then one atomic per word;
//  - 16 distinct keys: each lane adds its own words;
//  - otherwise: a segmented reduction per word over the run of equal keys (channel intervals
//    are contiguous, so a run is a range of lanes), added by the run's first lane pair.
__device__ __forceinline__ void mom_flush(float (&acc)[MOM_H], int key, int lane, double *mom)
{
    const int k = lane & 1;
    const int k0 = __shfl_sync(FULL_MASK, key, 0);
    if (__all_sync(FULL_MASK, key == k0)) {
        if (k0 >= 0) {
            // in place: after the halving at offset o the live words are acc[0 .. h)
#pragma unroll
            for (int h = 32, o = 16; h >= 4; h >>= 1, o >>= 1) {
                const bool up = (lane & o) != 0;
#pragma unroll
                for (int i = 0; i < h; ++i) {
                    const float lo = acc[i];
                    const float hi = i + h < MOM_H ? acc[i + h] : 0.f;
                    const float send = up ? lo : hi;
                    const float keep = up ? hi : lo;
                    acc[i] = keep + __shfl_xor_sync(FULL_MASK, send, o);
                }
            }
            double *dst = mom + (size_t)k0 * MOM_N;
            const int base = 4 * (lane >> 1);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (base + j < MOM_H) atomicAdd(dst + mom_word(base + j, k), (double)acc[j]);
        }
    } else {
        const unsigned m = __match_any_sync(FULL_MASK, key);
        if (__all_sync(FULL_MASK, m == (3u << (lane & ~1)))) {
            if (key >= 0) {
                double *dst = mom + (size_t)key * MOM_N;
#pragma unroll
                for (int v = 0; v < MOM_H; ++v) atomicAdd(dst + mom_word(v, k), (double)acc[v]);
            }
        } else {
            const int seg_end = 32 - __clz(m);
            const bool head = (lane >> 1) == ((__ffs(m) - 1) >> 1);
            double *dst = mom + (size_t)(key >= 0 ? key : 0) * MOM_N;
#pragma unroll
            for (int v = 0; v < MOM_H; ++v) {
                float x = acc[v];
#pragma unroll
                for (int d = 2; d < 32; d <<= 1) {
                    const float o = __shfl_down_sync(FULL_MASK, x, d);
                    if (lane + d < seg_end) x += o;
                }
                if (head && key >= 0) atomicAdd(dst + mom_word(v, k), (double)x);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < MOM_H; ++v) acc[v] = 0.f;
}

// The rows of the baseline strips in strip order, as the pass reads them: {row (-1: no usable
// sample), first bin of the row's time interval, unordered pair, 1 if ant1 > ant2}.
static __global__ void mom_rows_kernel(long n, const int *strip_rows, const int4 *rows, const uint8_t *row_live,
                                       const int *t_map, int n_fint, const int *up_of_bl, int4 *out)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int row = strip_rows[k];
    const int4 r = rows[row];
    out[k] = make_int4(row_live[row] ? row : -1, t_map[r.z] * n_fint, up_of_bl[r.w], r.x > r.y ? 1 : 0);
}

// a streamed 16-byte load: read-only for the kernel's lifetime, not kept in L1
__device__ __forceinline__ float4 ld_stream(const float4 *p)
{
    float4 r;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}

// one sample as loaded: its key, folded weights and the raw data and model quads
struct MomSample {
    int key;
    float4 w, d0, d1, m0, m1;
};

__device__ __forceinline__ MomSample mom_load(const MomArgs &a, const int4 &mr, int ch, int lane)
{
    MomSample x;
    const int c = ch * 16 + (lane >> 1);
    x.key = c < a.n_chan ? (mr.y + __ldg(a.tn.f_map + c)) * a.n_up + mr.z : -1;
    if (c < a.n_chan && mr.x >= 0) {
        const size_t i = (size_t)mr.x * a.n_chan + c;
        x.w = ld_stream(a.wf + i);
        x.d0 = ld_stream(a.vis + 2 * i);
        x.d1 = ld_stream(a.vis + 2 * i + 1);
        x.m0 = ld_stream(a.model + 2 * i);
        x.m1 = ld_stream(a.model + 2 * i + 1);
    } else {
        x.w = make_float4(0.f, 0.f, 0.f, 0.f);
        x.d0 = x.d1 = x.m0 = x.m1 = x.w;
    }
    return x;
}

// One pass: warps walk units of a baseline strip (the rows of one ordered baseline in time
// order) x a group of 16-channel chunks, row by row and chunk by chunk within a row, with the
// next sample's loads in flight while the current one is added to the lane's register sums.
// The sums are flushed when any lane's (interval, pair) key changes, so an interval that spans
// the group's chunks is flushed once per row.
static __global__ void __launch_bounds__(128, 3) mom_pass_kernel(const MomArgs a)
{
    if (__ldg(a.n_active) == 0) return;
    const int lane = threadIdx.x & 31;
    float acc[MOM_H];
#pragma unroll
    for (int v = 0; v < MOM_H; ++v) acc[v] = 0.f;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long n_warps = ((long)gridDim.x * blockDim.x) >> 5;
    const int n_groups = (a.n_chunks + a.group - 1) / a.group;
    const long n_units = (long)a.n_strips * n_groups;
    int cur = -1;
    for (long unit = warp; unit < n_units; unit += n_warps) {
        const int s = (int)(unit / n_groups), g = (int)(unit % n_groups);
        const int ch0 = g * a.group, ch1 = min(a.n_chunks, ch0 + a.group);
        const int k1 = __ldg(a.strip_off + s + 1);
        int k = __ldg(a.strip_off + s), ch = ch0;
        if (k >= k1) continue;
        int4 mr = __ldg(a.mrows + k);
        int4 mr_next = k + 1 < k1 ? __ldg(a.mrows + k + 1) : make_int4(-1, 0, 0, 0);
        MomSample cs = mom_load(a, mr, ch, lane);
        int conj = mr.w;
        while (true) {
            // the next step (chunk by chunk, then the next row) and its loads
            int k2 = k, ch2 = ch + 1;
            int4 mr2 = mr;
            if (ch2 == ch1) {
                ch2 = ch0;
                ++k2;
                mr2 = mr_next;
                if (k2 + 1 < k1) mr_next = __ldg(a.mrows + k2 + 1);
            }
            if (__any_sync(FULL_MASK, cs.key != cur)) {
                mom_flush(acc, cur, lane, a.mom);
                cur = cs.key;
            }
            const bool more = k2 < k1;
            MomSample ns;
            if (more) ns = mom_load(a, mr2, ch2, lane);
            if (cs.w.x != 0.f || cs.w.y != 0.f || cs.w.z != 0.f || cs.w.w != 0.f) {
                J2 D = j_from(cs.d0, cs.d1), M = j_from(cs.m0, cs.m1);
                float4 w = cs.w;
                if (conj) {                      // the conjugate baseline: D -> D^H, M -> M^H, w permuted
                    D = j_herm(D);
                    M = j_herm(M);
                    w = make_float4(w.x, w.z, w.y, w.w);
                }
                mom_add(acc, D, M, w, lane & 1);
            }
            if (!more) break;
            cs = ns;
            k = k2;
            ch = ch2;
            mr = mr2;
            conj = mr.w;
        }
    }
    mom_flush(acc, cur, lane, a.mom);
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

cudaError_t mom_launch_pass(const qc::MomArgs &a, int sm_count, cudaStream_t st)
{
    const int block = 128;                       // three CTAs per SM (register-bound)
    const int n_groups = (a.n_chunks + a.group - 1) / a.group;
    const long units = (long)a.n_strips * n_groups;
    const int grid = (int)std::max(1L, std::min((long)sm_count * 3, (units * 32 + block - 1) / block));
    qc::mom_pass_kernel<<<grid, block, 0, st>>>(a);
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
    qc::mom_normal_kernel<<<(int)((warps + 3) / 4), 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t mom_launch_rows(long n, const int *strip_rows, const int4 *rows, const uint8_t *row_live, const int *t_map,
                            int n_fint, const int *up_of_bl, int4 *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    qc::mom_rows_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(n, strip_rows, rows, row_live, t_map, n_fint,
                                                                 up_of_bl, out);
    return cudaGetLastError();
}

size_t mom_words() { return qc::MOM_N; }
