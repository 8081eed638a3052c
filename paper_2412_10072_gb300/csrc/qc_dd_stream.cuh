// qc_dd_stream.cuh -- streaming accumulate kernel for chains of one or two terms with
// directions (N_D > 1, at most DDS_MAX_DIR).
//
// The arithmetic of dd_acc_kernel (Eq. baselinemodel with directions: the residual over all
// directions; Eq. g_derivative_dd for a direction-dependent solved term, one block per
// (interval, antenna, direction); Eq. g_derivative_di for a direction-independent one, the
// Jacobian summed over directions; the q side through the conjugate baseline, Eq.
// gct_derivative_dd) on the skeleton of acc_stream_kernel:
//  * row tiles: a warp walks the 32-channel chunks of one row after the other, so the
//    antenna pair is fixed for a row and the register sums are flushed only when it or a
//    lane's bin changes;
//  * d, w and the N_D model words of each step are copied DEPTH - 1 steps ahead into the
//    warp's cp.async ring (stage layout [d0][d1][w][m_{0,0}][m_{0,1}] .. [m_{N_D-1,1}], 32
//    lanes each), zero-filled where there is nothing to read;
//  * the entries of a direction-independent term are read once per step (the solved term's
//    stay in registers while unchanged); a direction-dependent term's entries are read per
//    direction from its small table (L1/L2);
//  * a direction-dependent solved term: a CTA forms the blocks of SD of its directions (grid
//    dimension y), two for a diagonal term; every CTA forms the whole residual;
//  * a solved delay term (direction-independent by construction) adds to its parameter sums
//    per (interval, antenna) through the chain rule, as acc_delay_kernel does.
#pragma once
#include <type_traits>

#include "qc_stream_delay.cuh"

namespace qc {

constexpr int DDS_MAX_DIR = 4;   // directions the streaming kernel takes (more: dd_acc_kernel)
constexpr int DDS_DEPTH = 3;     // ring depth (steps): two CTAs of 8 warps per SM at N_D = 2

struct DDStreamArgs {
    StreamArgs s;           // row tiles (s.order 0); s.model: [n_row][n_chan][n_dir] x 2 float4
    int n_dir;
    int nd_n, nd_o;         // directions in the solved / other term's table (1: direction-independent)
    const float *omega;     // solved delay term: [n_chan] 2 pi nu - omega_ref
};

__host__ __device__ constexpr int dds_smem_per_warp(int n_dir)
{
    return DDS_DEPTH * ((3 + 2 * n_dir) * 32 * 16 + 2 * 16);
}

__device__ __forceinline__ J2 dds_zero()
{
    J2 r;
    r.a = r.b = r.c = r.d = make_float2(0.f, 0.f);
    return r;
}

__device__ __forceinline__ void dds_add(J2 &A, const J2 &B)
{
    A.a = cadd(A.a, B.a); A.b = cadd(A.b, B.b); A.c = cadd(A.c, B.c); A.d = cadd(A.d, B.d);
}

// A B for Jones matrices of kinds KA and KB (a diagonal one keeps its zeros out of the products)
template <int KA, int KB> __device__ __forceinline__ J2 kprod(const J2 &A, const J2 &B)
{
    if constexpr (KA == KIND_DIAG && KB == KIND_DIAG) {
        J2 r;
        r.a = cmul(A.a, B.a);
        r.b = r.c = make_float2(0.f, 0.f);
        r.d = cmul(A.d, B.d);
        return r;
    } else if constexpr (KA == KIND_DIAG) {
        return j_dmul(A.a, A.d, B);
    } else if constexpr (KB == KIND_DIAG) {
        return j_muld(A, B.a, B.d);
    } else {
        return j_mul(A, B);
    }
}

// Weights and weighted residual of one side seen through a diagonal left factor L: the
// Jacobian of V = L G X with respect to G is that of G X with row i scaled by l_i, so the
// blocks of G are those of the unscaled problem with w_ij -> |l_i|^2 w_ij and
// wr_ij -> conj(l_i) wr_ij (and no coupling between the rows).
__device__ __forceinline__ void dds_left_diag(const J2 &L, float4 &w, J2 &wr)
{
    const float n0 = cnorm2(L.a), n1 = cnorm2(L.d);
    w = make_float4(n0 * w.x, n0 * w.y, n1 * w.z, n1 * w.w);
    wr.a = cmulc(wr.a, L.a);
    wr.b = cmulc(wr.b, L.a);
    wr.c = cmulc(wr.c, L.d);
    wr.d = cmulc(wr.d, L.d);
}

// One direction of a sample of baseline (p, q): with the solved term G and the other term O
// (to the left of G when OLEFT, else to the right; absent when OK is KIND_NONE), the chain
// C_{a,d} = O G or G O.  WV: adds C_{p,d} M_d C_{q,d}^H to V.  XY = 1 adds, XY = 2 writes the
// solved term's X_d = R_{p,d} M_d C_{q,d}^H and Y_d = R_{q,d} M_d^H C_{p,d}^H (Eq. chain_trick
// per direction; R is O when O is to the right, else the identity).
template <int GK, int OK, bool OLEFT, bool WV, int XY>
__device__ __forceinline__ void dds_direction(const J2 &Gp, const J2 &Gq, const J2 &Op, const J2 &Oq, const J2 &M,
                                              J2 &V, J2 &X, J2 &Y)
{
    if constexpr (OK == KIND_NONE || OLEFT) {
        constexpr int CK = (GK == KIND_FULL || OK == KIND_FULL) ? KIND_FULL : KIND_DIAG;
        J2 Cp = Gp, Cq = Gq;
        if constexpr (OK != KIND_NONE) {
            Cp = kprod<OK, GK>(Op, Gp);
            Cq = kprod<OK, GK>(Oq, Gq);
        }
        const J2 A = lmulk<CK>(Cp, M);                 // C_p M
        if constexpr (WV) dds_add(V, rmulk_h<CK>(A, Cq));   // C_p M C_q^H
        if constexpr (XY == 1) {
            dds_add(X, rmulk_h<CK>(M, Cq));            // M C_q^H
            dds_add(Y, j_herm(A));                     // M^H C_p^H
        } else if constexpr (XY == 2) {
            X = rmulk_h<CK>(M, Cq);
            Y = j_herm(A);
        }
    } else {
        J2 Z;                                          // O_p M O_q^H
        if constexpr (OK == KIND_DIAG) Z = j_muld(j_dmul(Op.a, Op.d, M), cconj(Oq.a), cconj(Oq.d));
        else Z = j_mul_h(j_mul(Op, M), Oq);
        const J2 Xd = rmulk_h<GK>(Z, Gq);              // O_p M C_q^H
        if constexpr (WV) dds_add(V, lmulk<GK>(Gp, Xd));
        if constexpr (XY == 1) {
            dds_add(X, Xd);
            dds_add(Y, j_herm(lmulk<GK>(Gp, Z)));      // O_q M^H C_p^H
        } else if constexpr (XY == 2) {
            X = Xd;
            Y = j_herm(lmulk<GK>(Gp, Z));
        }
    }
}

// SD = 0: a direction-independent solved term (one pass over the directions sums V, X and Y);
// SD > 0: a direction-dependent solved term, SD of its directions per CTA (grid dimension y:
// directions SD y .. SD y + SD - 1), V over every direction first, then X_d and Y_d of each of
// the CTA's directions straight into its register sums.
template <int GK, int OK, bool OLEFT, bool DSUMS, int SD, int DEPTH>
__global__ void __launch_bounds__(256, 2) dd_stream_kernel(const DDStreamArgs da)
{
    const StreamArgs &a = da.s;
    if (__ldg(a.n_active) == 0) return;
    constexpr int TS = GK == KIND_FULL ? TS_FULL : TS_DIAG;
    // a full left factor enters the blocks (HAS_L); a diagonal one only scales the weights
    // of its side (dds_left_diag), so the blocks keep the layout without a left factor
    constexpr bool HAS_L = OLEFT && OK == KIND_FULL;
    constexpr bool LDIAG = OLEFT && OK == KIND_DIAG;
    using Lay = typename std::conditional<DSUMS, DelayLayout<HAS_L>, AccLayout<TS, HAS_L>>::type;
    constexpr int KR = Lay::KR, KG = Lay::KG;
    static_assert(DEPTH >= 3, "the entry of the next step must be in the ring");
    static_assert(!DSUMS || GK == KIND_DIAG, "a delay term is diagonal");
    extern __shared__ float4 s_stream[];
    const int n_dir = da.n_dir, n_mw = 2 * n_dir, v4 = 3 + n_mw;
    constexpr int NA = SD > 0 ? SD : 1;                    // register sums: one set per direction
    const int ndn = da.nd_n, ndo = da.nd_o, d0 = blockIdx.y * NA;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float4 *ring = s_stream + (size_t)wib * DEPTH * v4 * 32;                          // [DEPTH][v4][32]
    int4 *meta = reinterpret_cast<int4 *>(s_stream + (size_t)nw * DEPTH * v4 * 32) + (size_t)wib * DEPTH * 2;
    const int W = (int)((gridDim.x * blockDim.x) >> 5);
    const int n_chan = a.n_chan, n_ant = a.n_ant;

    StreamCursor<false> cur;
    cur.start(a, lane, (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), W);
    int stage_i = 0;
    auto issue = [&]() {
        cur.issue_dd(a, lane, ring, meta, stage_i, n_mw);
        if (++stage_i == DEPTH) stage_i = 0;
    };
#pragma unroll
    for (int d = 0; d < DEPTH - 1; ++d) issue();
    __syncwarp();

    Acc<KR, false> Ap[NA], Aq[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        Ap[j].zero();
        Aq[j].zero();
    }
    int stage = 0, cur_key = -1, cur_pq = -1;
    auto read_map = [&](const int4 &m0, const int4 &m1) {
        const int c = m1.x + lane;
        return (m0.x != STREAM_END && m0.z >= 0 && c < n_chan) ? __ldg(a.fmap2 + c) : make_int2(0, 0);
    };
    // accumulator antenna pair of the solved term in direction d: (antenna, d) -> a N_D + d
    auto pq_acc = [&](int pq, int d) {
        return SD > 0 ? ((pq & 0xffff) * ndn + d) | (((pq >> 16) * ndn + d) << 16) : pq;
    };
    auto flush_all = [&]() {
#pragma unroll
        for (int j = 0; j < NA; ++j)
            if (SD == 0 || d0 + j < n_dir)
                flush_pair<KR, KG, Lay>(Ap[j], Aq[j], cur_key, pq_acc(cur_pq, d0 + j), lane, a.active, a.acc,
                                        n_ant * ndn);
    };
    int4 eA0 = meta[0], eA1 = meta[1];
    int2 fmA = read_map(eA0, eA1);
    int ci_p = -1, ci_q = -1, act_key = -1;
    bool act_val = false;
    J2 cGp = j_identity(), cGq = j_identity(), Op = j_identity(), Oq = j_identity();
    // a step in two parts, as in acc_stream_kernel: (A) entries, the direction-independent
    // gains, the issue ahead, the wait and the lane's key; (B) the arithmetic over the
    // directions and the advance.  Steps that need no flush stay in an inner loop that only
    // adds; the flush runs outside it.
    int4 e = eA0, e1 = eA1, eB0 = eA0, eB1 = eA1;
    int2 fm = fmA, fmB = fmA;
    int nst = 0, key = -1;
    bool in = false, live = false;
    float om = 0.f;
    auto part_a = [&]() -> bool {
        e = eA0;
        e1 = eA1;
        if (e.x == STREAM_END) return false;
        fm = fmA;
        nst = stage + 1 == DEPTH ? 0 : stage + 1;
        eB0 = meta[2 * nst];
        eB1 = meta[2 * nst + 1];
        fmB = read_map(eB0, eB1);
        const int c = e1.x + lane;
        if (e.z >= 0) {
            const int p = e.y & 0xffff, q = e.y >> 16;
            if constexpr (OK != KIND_NONE) {
                if (ndo == 1) {
                    Op = fetch_k<OK>(a.to, n_ant, e.w, fm.y, p);
                    Oq = fetch_k<OK>(a.to, n_ant, e.w, fm.y, q);
                }
            }
            if constexpr (SD == 0) {
                // the solved term's entries stay in registers while the lane's table index is unchanged
                const bool inr = c < n_chan;
                int ip, iq;
                if constexpr (DSUMS) {
                    // the delay term's gains at the lane's channel: table [n_tint][n_ant][n_chan]
                    om = inr ? __ldg(da.omega + c) : 0.f;
                    ip = inr ? (e.z * n_ant + p) * n_chan + c : ci_p;
                    iq = inr ? (e.z * n_ant + q) * n_chan + c : ci_q;
                } else {
                    ip = inr ? (e.z * n_ant + p) * a.tn.n_fint + fm.x : ci_p;
                    iq = inr ? (e.z * n_ant + q) * a.tn.n_fint + fm.x : ci_q;
                }
                if (__any_sync(0xffffffffu, ip != ci_p || iq != ci_q)) {
                    if constexpr (DSUMS) {
                        if (ip != ci_p) { cGp = j_diag(__ldg(a.tn.tab + ip)); ci_p = ip; }
                        if (iq != ci_q) { cGq = j_diag(__ldg(a.tn.tab + iq)); ci_q = iq; }
                    } else {
                        if (ip != ci_p) { cGp = fetch_k<GK>(a.tn, n_ant, e.z, fm.x, p); ci_p = ip; }
                        if (iq != ci_q) { cGq = fetch_k<GK>(a.tn, n_ant, e.z, fm.x, q); ci_q = iq; }
                    }
                }
            }
        }
        issue();
        cp_async_wait<DEPTH - 1>();
        __syncwarp();
        live = e.z >= 0;                            // warp-uniform
        in = live && c < n_chan;
        key = in ? e.z * a.tn.n_fint + fm.x : -1;
        return true;
    };
    auto part_b = [&]() {
        const float4 *slot = ring + (size_t)stage * v4 * 32 + lane;
        const float4 w = slot[64];
        bool ok = in && (w.x != 0.f || w.y != 0.f || w.z != 0.f || w.w != 0.f);
        if (ok && key != act_key) {          // activity of the lane's bin, read when the bin changes
            act_key = key;
            act_val = __ldg(a.active + key) != 0;
        }
        ok = ok && act_val;
        if (ok) {
            const int p = e.y & 0xffff, q = e.y >> 16;
            const J2 Dm = j_from(slot[0], slot[32]);
            const float4 wq = make_float4(w.x, w.z, w.y, w.w);
            // the other term's entries in direction d (a direction-dependent one from its table)
            auto other_at = [&](int d, J2 &Opd, J2 &Oqd) {
                Opd = Op;
                Oqd = Oq;
                if constexpr (OK != KIND_NONE) {
                    if (ndo > 1) {
                        Opd = fetch_k<OK>(a.to, n_ant * ndo, e.w, fm.y, p * ndo + d);
                        Oqd = fetch_k<OK>(a.to, n_ant * ndo, e.w, fm.y, q * ndo + d);
                    }
                }
            };
            J2 V = dds_zero();
            if constexpr (SD == 0) {
                // direction-independent solved term: its Jacobian is summed over the directions
                // (a term to its left is direction-independent too, so L is O)
                J2 X = dds_zero(), Y = dds_zero();
                for (int d = 0; d < n_dir; ++d) {
                    J2 Opd, Oqd;
                    other_at(d, Opd, Oqd);
                    const J2 M = j_from(slot[96 + 64 * d], slot[128 + 64 * d]);
                    dds_direction<GK, OK, OLEFT, true, 1>(cGp, cGq, Opd, Oqd, M, V, X, Y);
                }
                J2 wr;
                wr.a = cscale(csub(Dm.a, V.a), w.x); wr.b = cscale(csub(Dm.b, V.b), w.y);
                wr.c = cscale(csub(Dm.c, V.c), w.z); wr.d = cscale(csub(Dm.d, V.d), w.w);
                float4 wp = w, wqq = wq;
                J2 wrp = wr, wrq = j_herm(wr);
                if constexpr (LDIAG) {
                    dds_left_diag(Op, wp, wrp);
                    dds_left_diag(Oq, wqq, wrq);
                }
                if constexpr (DSUMS) {
                    delay_side<HAS_L>(Ap[0], Op, X, wp, wrp, cGp.a, cGp.d, om);
                    delay_side<HAS_L>(Aq[0], Oq, Y, wqq, wrq, cGq.a, cGq.d, om);
                } else {
                    accumulate_side<TS, HAS_L, false>(Ap[0], Op, X, wp, wrp);
                    accumulate_side<TS, HAS_L, false>(Aq[0], Oq, Y, wqq, wrq);
                }
            } else {
                // direction-dependent solved term: the residual over every direction first
                auto solved_at = [&](int d, J2 &Gp, J2 &Gq) {
                    Gp = fetch_k<GK>(a.tn, n_ant * ndn, e.z, fm.x, p * ndn + d);
                    Gq = fetch_k<GK>(a.tn, n_ant * ndn, e.z, fm.x, q * ndn + d);
                };
                for (int d = 0; d < n_dir; ++d) {
                    J2 Gp, Gq, Opd, Oqd, X_, Y_;
                    solved_at(d, Gp, Gq);
                    other_at(d, Opd, Oqd);
                    const J2 M = j_from(slot[96 + 64 * d], slot[128 + 64 * d]);
                    dds_direction<GK, OK, OLEFT, true, 0>(Gp, Gq, Opd, Oqd, M, V, X_, Y_);
                }
                J2 wr;
                wr.a = cscale(csub(Dm.a, V.a), w.x); wr.b = cscale(csub(Dm.b, V.b), w.y);
                wr.c = cscale(csub(Dm.c, V.c), w.z); wr.d = cscale(csub(Dm.d, V.d), w.w);
                const J2 wrh = j_herm(wr);
#pragma unroll
                for (int j = 0; j < NA; ++j) {
                    const int d = d0 + j;
                    if (d < n_dir) {
                        J2 Gp, Gq, Opd, Oqd, X, Y;
                        solved_at(d, Gp, Gq);
                        other_at(d, Opd, Oqd);
                        const J2 M = j_from(slot[96 + 64 * d], slot[128 + 64 * d]);
                        dds_direction<GK, OK, OLEFT, false, 2>(Gp, Gq, Opd, Oqd, M, V, X, Y);
                        if constexpr (LDIAG) {
                            float4 wp = w, wqq = wq;
                            J2 wrp = wr, wrq = wrh;
                            dds_left_diag(Opd, wp, wrp);
                            dds_left_diag(Oqd, wqq, wrq);
                            accumulate_side<TS, false, false>(Ap[j], Opd, X, wp, wrp);
                            accumulate_side<TS, false, false>(Aq[j], Oqd, Y, wqq, wrq);
                        } else {
                            accumulate_side<TS, HAS_L, false>(Ap[j], Opd, X, w, wr);
                            accumulate_side<TS, HAS_L, false>(Aq[j], Oqd, Y, wq, wrh);
                        }
                    }
                }
            }
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
                const bool change = e.y != cur_pq || key != cur_key;
                if (__any_sync(0xffffffffu, change && cur_key >= 0)) break;
                cur_key = key;
                cur_pq = e.y;
            }
            part_b();
        }
        if (ended) break;
        flush_all();
        cur_key = key;
        cur_pq = e.y;
        part_b();
    }
    if (__any_sync(0xffffffffu, cur_key >= 0)) flush_all();
    cp_async_wait<0>();
}

} // namespace qc
