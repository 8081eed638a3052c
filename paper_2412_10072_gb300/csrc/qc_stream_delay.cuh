// qc_stream_delay.cuh -- streaming accumulate kernel of a solved delay term (QC_TERM_DELAY).
//
// Same ring, cursor and flushes as acc_stream_kernel, for chains of one or two terms.
// The difference is what a sample adds.  The delay term's gains change from channel to
// channel, g_c(nu) = exp(i (phi_c + 2 pi tau_c nu)), while its parameters are shared by
// every sample of a solution interval (Scenario 2 of Section 2.4).  Each sample first
// forms the blocks of a diagonal term at its own channel: JHJ_g over (g_X, g_Y) and JHr_g.
// It then applies the chain rule with dg_c/dphi_c = i g_c and dg_c/dtau_c = i omega g_c,
// omega = 2 pi nu, and adds the real products (Eq. jhj_case2, Eq. jhwr_case2, without
// their factor 2, which the update applies) to register sums per (interval, antenna), with
// omega taken relative to the centre of the band, omega' = omega - omega_ref (the update
// shifts the sums back in FP64; centred sums keep FP32 rounding small and a band of one
// frequency exactly degenerate):
//   [0..2]   sum h_XX (1, omega', omega'^2)     [3..5]   sum h_YY (1, omega', omega'^2)
//   [6, 7]   sum r_X (1, omega')                [8, 9]   sum r_Y (1, omega')
//   [10..12] sum h_XY (1, omega', omega'^2)  (left factor only: X and Y couple through L)
// with h_cc = JHJ_g[c][c], h_XY = Re(conj(g_X) JHJ_g[X][Y] g_Y), r_c = Im(conj(g_c) JHr_g[c]).
// The keys of the flushes are the term's parameter intervals, so a row tile of an interval
// wider than 32 channels flushes once per row, as the other diagonal and full solves do.
#pragma once
#include "qc_delay.cuh"
#include "qc_stream.cuh"

namespace qc {

// register sums of one side, flushed to KG_SUMS FP64 words per (interval, antenna)
template <bool HAS_L> struct DelayLayout {
    static constexpr int KR = HAS_L ? 13 : 10, KG = KG_SUMS;
    __device__ static constexpr int g(int i) { return i; }
};

struct DelayStreamArgs {
    StreamArgs s;          // s.tn: the delay term's parameter intervals (n_fint, f_map), with
                           // s.tn.tab its channel table [n_tint][n_ant][n_chan] of (g_X, g_Y)
    const float *omega;    // [n_chan] 2 pi nu - omega_ref of each channel
};

// One side (antenna) of a sample: diagonal-term quantities at the sample's channel, then
// the chain rule into the register sums.  X, w in the orientation of this side, and wd its
// weighted residual w * (D - V), or (WD) its weighted data w * D: the model of the sample is
// V = E g with g = (g_X, g_Y) at this channel, so conj(g_X) JHr_g[X] = conj(g_X) (J^H W d)[X]
// - h_00 |g_X|^2 - conj(g_X) h_01 g_Y, whose imaginary part lacks the real h_00 |g_X|^2
// (likewise for Y with conj(h_01)); without a left factor h_01 = 0.
template <bool HAS_L, bool WD = false>
__device__ __forceinline__ void delay_side(Acc<DelayLayout<HAS_L>::KR, false> &A, const J2 &L, const J2 &X,
                                           float4 w, const J2 &wd, float2 gx, float2 gy, float om)
{
    const float wv[4] = { w.x, w.y, w.z, w.w };
    const float2 wrv[4] = { wd.a, wd.b, wd.c, wd.d };
    const float2 Xv[4] = { X.a, X.b, X.c, X.d };            // X[l][j] = Xv[2l+j]
    float h00, h11;
    float2 j0, j1, h01 = make_float2(0.f, 0.f);
    if constexpr (!HAS_L) {
        // parameter k in {XX, YY} touches row k of V: E[(k,j), k] = X[k][j]
        h00 = fmaf(wv[0], cnorm2(Xv[0]), wv[1] * cnorm2(Xv[1]));
        h11 = fmaf(wv[2], cnorm2(Xv[2]), wv[3] * cnorm2(Xv[3]));
        j0 = cfma_conj(Xv[1], wrv[1], cfma_conj(Xv[0], wrv[0], make_float2(0.f, 0.f)));
        j1 = cfma_conj(Xv[3], wrv[3], cfma_conj(Xv[2], wrv[2], make_float2(0.f, 0.f)));
    } else {
        // free columns (0,0) and (1,1): E[(i,j), k] = L[i][k] X[k][j]
        const float2 Lv[4] = { L.a, L.b, L.c, L.d };
        float2 E0[4], E1[4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                E0[2 * i + j] = cmul(Lv[2 * i + 0], Xv[0 + j]);
                E1[2 * i + j] = cmul(Lv[2 * i + 1], Xv[2 + j]);
            }
        h00 = 0.f;
        h11 = 0.f;
        j0 = make_float2(0.f, 0.f);
        j1 = j0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            h00 = fmaf(wv[m], cnorm2(E0[m]), h00);
            h11 = fmaf(wv[m], cnorm2(E1[m]), h11);
            h01 = cfma_conj(E0[m], cscale(E1[m], wv[m]), h01);
            j0 = cfma_conj(E0[m], wrv[m], j0);
            j1 = cfma_conj(E1[m], wrv[m], j1);
        }
    }
    float rx = gx.x * j0.y - gx.y * j0.x;                 // Im(conj(g_X) JHr_g[X])
    float ry = gy.x * j1.y - gy.y * j1.x;                 // Im(conj(g_Y) JHr_g[Y])
    const float om2 = om * om;
    float xy = 0.f;
    if constexpr (HAS_L) {
        const float2 t = make_float2(fmaf(gx.x, h01.x, gx.y * h01.y), fmaf(gx.x, h01.y, -gx.y * h01.x));
        xy = fmaf(t.x, gy.x, -t.y * gy.y);                 // Re(conj(g_X) JHJ_g[X][Y] g_Y)
        if constexpr (WD) {
            const float yi = fmaf(t.x, gy.y, t.y * gy.x);  // Im(conj(g_X) JHJ_g[X][Y] g_Y)
            rx -= yi;
            ry += yi;
        }
    }
    A.s[0] += h00;
    A.s[1] = fmaf(h00, om, A.s[1]);
    A.s[2] = fmaf(h00, om2, A.s[2]);
    A.s[3] += h11;
    A.s[4] = fmaf(h11, om, A.s[4]);
    A.s[5] = fmaf(h11, om2, A.s[5]);
    A.s[6] += rx;
    A.s[7] = fmaf(rx, om, A.s[7]);
    A.s[8] += ry;
    A.s[9] = fmaf(ry, om, A.s[9]);
    if constexpr (HAS_L) {
        A.s[10] += xy;
        A.s[11] = fmaf(xy, om, A.s[11]);
        A.s[12] = fmaf(xy, om2, A.s[12]);
    }
}

// One unflagged sample of baseline (p, q): chain factors around the delay term G (diagonal
// at this channel) and both sides' sums (the conjugate baseline for q), as in sample_math for
// a diagonal term; the sides take the weighted data, so the sample forms neither V nor the
// residual (delay_side).
template <int LK, int RK>
__device__ __forceinline__ void delay_sample_math(const J2 &Lp, const J2 &Gp, const J2 &Rp, const J2 &Lq, const J2 &Gq,
                                                  const J2 &Rq, const J2 &Dm, const J2 &M, float4 w, float om,
                                                  Acc<DelayLayout<LK != KIND_NONE>::KR, false> &Ap,
                                                  Acc<DelayLayout<LK != KIND_NONE>::KR, false> &Aq)
{
    constexpr bool HAS_L = LK != KIND_NONE;
    J2 X, Y;
    if constexpr (RK == KIND_NONE) {
        const J2 Cp = HAS_L ? rmulk<KIND_DIAG>(Lp, Gp) : Gp;
        const J2 Cq = HAS_L ? rmulk<KIND_DIAG>(Lq, Gq) : Gq;
        constexpr int CK = HAS_L ? KIND_FULL : KIND_DIAG;
        const J2 A = lmulk<CK>(Cp, M);                 // C_p M
        X = rmulk_h<CK>(M, Cq);                        // M C_q^H
        Y = j_herm(A);                                 // M^H C_p^H
    } else {
        J2 Z;
        if constexpr (RK == KIND_DIAG) Z = j_muld(j_dmul(Rp.a, Rp.d, M), cconj(Rq.a), cconj(Rq.d));
        else Z = j_mul_h(j_mul(Rp, M), Rq);
        X = rmulk_h<LK>(rmulk_h<KIND_DIAG>(Z, Gq), Lq);
        const J2 W = lmulk<LK>(Lp, lmulk<KIND_DIAG>(Gp, Z));
        Y = j_herm(W);
    }
    J2 wd;
    wd.a = cscale(Dm.a, w.x); wd.b = cscale(Dm.b, w.y);
    wd.c = cscale(Dm.c, w.z); wd.d = cscale(Dm.d, w.w);
    delay_side<HAS_L, true>(Ap, Lp, X, w, wd, Gp.a, Gp.d, om);
    delay_side<HAS_L, true>(Aq, Lq, Y, make_float4(w.x, w.z, w.y, w.w), j_herm(wd), Gq.a, Gq.d, om);
}

template <int LK, int RK, bool M16, int DEPTH>
__global__ void __launch_bounds__(256, 2) acc_delay_kernel(const DelayStreamArgs da)
{
    const StreamArgs &a = da.s;
    if (__ldg(a.n_active) == 0) return;
    constexpr bool HAS_L = LK != KIND_NONE;
    constexpr int FLUSH_EVERY = M16 ? 16 : (1 << 30);
    using Lay = DelayLayout<HAS_L>;
    constexpr int KR = Lay::KR, KG = Lay::KG;
    constexpr int V4 = M16 ? 4 : 5;
    static_assert(DEPTH >= 3, "the entry of the next step must be in the ring");
    extern __shared__ float4 s_stream[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float4 *ring = s_stream + (size_t)wib * DEPTH * V4 * 32;
    int4 *meta = reinterpret_cast<int4 *>(s_stream + (size_t)nw * DEPTH * V4 * 32) + (size_t)wib * DEPTH * 2;
    const int W = (int)((gridDim.x * blockDim.x) >> 5);
    const int n_chan = a.n_chan, n_ant = a.n_ant;

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

    Acc<KR, false> Ap, Aq;
    Ap.zero();
    Aq.zero();
    int stage = 0, cur_key = -1, cur_pq = -1;
    auto read_map = [&](const int4 &m0, const int4 &m1) {
        const int c = m1.x + lane;
        return (m0.x != STREAM_END && m0.z >= 0 && c < n_chan) ? __ldg(a.fmap2 + c) : make_int2(0, 0);
    };
    int4 eA0 = meta[0], eA1 = meta[1];
    int2 fmA = read_map(eA0, eA1);
    int ci_p = -1, ci_q = -1, act_key = -1, since_flush = 0;
    bool act_val = false;
    J2 cGp = j_identity(), cGq = j_identity();
    // a step in two parts, as in acc_stream_kernel: (A) entries, gains, the issue ahead, the wait
    // and the lane's key; (B) the arithmetic and the advance.  Steps that need no flush stay in an
    // inner loop that only adds; the flush runs outside it.
    int4 e = eA0, e1 = eA1, eB0 = eA0, eB1 = eA1;
    int2 fm = fmA, fmB = fmA;
    int nst = 0, key = -1;
    bool in = false, live = false;
    float om = 0.f;
    J2 Lp, Lq, Rp, Rq;
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
        // this step's gain entries and the lane's omega, loaded before the issue below
        om = 0.f;
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
            const bool inr = c < n_chan;
            if (inr) om = __ldg(da.omega + c);
            // the delay term's gains at the lane's channel: table [n_tint][n_ant][n_chan]
            const int ip = inr ? (e.z * n_ant + p) * n_chan + c : ci_p;
            const int iq = inr ? (e.z * n_ant + q) * n_chan + c : ci_q;
            if (__any_sync(0xffffffffu, ip != ci_p || iq != ci_q)) {
                if (ip != ci_p) { cGp = j_diag(__ldg(a.tn.tab + ip)); ci_p = ip; }
                if (iq != ci_q) { cGq = j_diag(__ldg(a.tn.tab + iq)); ci_q = iq; }
            }
        }
        issue();
        cp_async_wait<DEPTH - 1>();
        __syncwarp();
        live = e.z >= 0;
        in = live && c < n_chan;
        key = in ? e.z * a.tn.n_fint + fm.x : -1;
        return true;
    };
    auto part_b = [&]() {
        const float4 *slot = ring + (size_t)stage * V4 * 32 + lane;
        const float4 w = slot[M16 ? 96 : 128];
        bool ok = in && (w.x != 0.f || w.y != 0.f || w.z != 0.f || w.w != 0.f);
        if (ok && key != act_key) {
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
            delay_sample_math<LK, RK>(Lp, Gp, Rp, Lq, Gq, Rq, Dm, M, w, om, Ap, Aq);
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

} // namespace qc
