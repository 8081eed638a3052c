// qc_dd.cu -- chains with direction-dependent terms (N_D > 1 directions).
//
// The model of Eq. baselinemodel with directions: V_pq = sum_d C_{p,d} M_{pq,d} C_{q,d}^H,
// C_{p,d} the product of the chain's Jones terms (Eq. joneschain), each term either
// direction-dependent (its own gains per direction) or direction-independent (the same
// gains in every direction).  The derivative with respect to the solved term n
// (Eq. chain_trick) is, for a direction-dependent term, per direction
//     dv/dg_{p,d} = L_{p,d} (x) (R_{p,d} M_d C_{q,d}^H)^T          (Eq. g_derivative_dd)
// and, for a direction-independent term, the sum of the same over directions
// (Eq. g_derivative_di); the q side goes through the conjugate baseline (Eq.
// gct_derivative_dd).  The AllJones approximation keeps one block per (interval, antenna)
// and, for a direction-dependent term, per direction.
//
// A direction-dependent term is stored as a term over n_ant * N_D "antennas" (a, d) ->
// a N_D + d (its gains are laid out [n_tint][n_fint][n_ant][N_D][4], which is that), so the
// FP64 block solve, update and convergence test of the one-direction path apply unchanged.
// A direction-independent solved term must have no direction-dependent term to its left:
// then L_{p,d} = L_p and its Jacobian is L_p (x) (sum_d X_d)^T, accumulated in one pass.
//
// Kernels: dd_acc_kernel (one pass per iteration: the residual of every sample over all
// directions and its contributions to the blocks of the solved term; for a
// direction-dependent term, grid dimension y is the direction whose blocks a CTA forms)
// and dd_residual_kernel (chi^2 of Eq. min and, optionally, the residual).
#include "qc_internal.h"

namespace qc {

// Jones matrix of term T (nd directions in its table) at (tint, fint) for antenna a, direction d
__device__ __forceinline__ J2 dd_jones(const DevTerm &T, int nd, int n_ant, int tint, int fint, int a, int d)
{
    return fetch_jones(T, n_ant * nd, tint, fint, nd > 1 ? a * nd + d : a);
}

// Chain factors around the solved term n for antenna a in direction d: L = prod_{j<n},
// G = term n, R = prod_{j>n} (n = -1: everything in L).
__device__ __forceinline__ void dd_factors(const DDArgs &A, const int *tint, const int *fint, int a, int d, J2 &L,
                                           J2 &G, J2 &R)
{
    const Chain &C = A.C;
    L = j_identity();
    G = j_identity();
    R = j_identity();
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {
        if (j >= C.n_terms) break;
        const J2 J = dd_jones(C.t[j], A.nd[j], C.n_ant, tint[j], fint[j], a, d);
        if (j < C.n || C.n < 0) L = j_mul(L, J);
        else if (j == C.n) G = J;
        else R = j_mul(R, J);
    }
}

__device__ __forceinline__ J2 j_add(const J2 &A, const J2 &B)
{
    J2 r;
    r.a = cadd(A.a, B.a); r.b = cadd(A.b, B.b); r.c = cadd(A.c, B.c); r.d = cadd(A.d, B.d);
    return r;
}

__device__ __forceinline__ J2 j_zero()
{
    J2 r;
    r.a = r.b = r.c = r.d = make_float2(0.f, 0.f);
    return r;
}

template <int TS>
__global__ void __launch_bounds__(256) dd_acc_kernel(const DDArgs A)
{
    if (__ldg(A.n_active) == 0) return;
    using Lay = AccLayout<TS, true>;
    constexpr int KR = Lay::KR, KG = Lay::KG;
    const Data &D = A.D;
    const Chain &C = A.C;
    const int n = C.n, n_chan = D.n_chan, n_dir = A.n_dir;
    const DevTerm &Tn = C.t[n];
    const int ndn = A.nd[n];
    const int nat = C.n_ant * ndn;                       // accumulator antennas of the solved term
    const int dsel = blockIdx.y;                         // direction of the blocks this CTA forms
    const bool dd = A.dd_solved != 0;
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long n_warps = ((long)gridDim.x * blockDim.x) >> 5;
    const int n_chunks = (n_chan + 31) / 32;
    Acc<KR, false> Ap, Aq;
    Ap.zero();
    Aq.zero();
    int cur_key = -1, cur_pq = -1;
    for (long u = warp; u < (long)D.n_row * n_chunks; u += n_warps) {
        const int row = (int)(u / n_chunks);
        const int c = (int)(u % n_chunks) * 32 + lane;
        if (!__ldg(A.row_live + row)) continue;          // warp-uniform
        const bool in = c < n_chan;
        const int4 meta = __ldg(D.rows + row);
        const int tn = __ldg(Tn.t_map + meta.z);
        const int key = in ? tn * Tn.n_fint + __ldg(Tn.f_map + c) : -1;
        const int pv = ndn > 1 ? meta.x * ndn + dsel : meta.x;
        const int qv = ndn > 1 ? meta.y * ndn + dsel : meta.y;
        const int pq = pv | (qv << 16);
        if (__any_sync(0xffffffffu, (pq != cur_pq || key != cur_key) && cur_key >= 0))
            flush_pair<KR, KG, Lay>(Ap, Aq, cur_key, cur_pq, lane, A.active, A.acc, nat);
        cur_key = key;
        cur_pq = pq;
        const size_t s = (size_t)row * n_chan + (in ? c : 0);
        const float4 w = in ? __ldg(A.wf + s) : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool ok = in && (w.x != 0.f || w.y != 0.f || w.z != 0.f || w.w != 0.f) && __ldg(A.active + key);
        if (!ok) continue;
        int tint[MAXT], fint[MAXT];
#pragma unroll
        for (int j = 0; j < MAXT; ++j) {
            tint[j] = j < C.n_terms ? __ldg(C.t[j].t_map + meta.z) : 0;
            fint[j] = j < C.n_terms ? __ldg(C.t[j].f_map + c) : 0;
        }
        J2 V = j_zero(), X = j_zero(), Y = j_zero(), Lp = j_identity(), Lq = j_identity();
        for (int d = 0; d < n_dir; ++d) {
            J2 Lpd, Gpd, Rpd, Lqd, Gqd, Rqd;
            dd_factors(A, tint, fint, meta.x, d, Lpd, Gpd, Rpd);
            dd_factors(A, tint, fint, meta.y, d, Lqd, Gqd, Rqd);
            const J2 Cp = j_mul(j_mul(Lpd, Gpd), Rpd), Cq = j_mul(j_mul(Lqd, Gqd), Rqd);
            const size_t mi = 2 * (s * n_dir + d);
            const J2 M = j_from(__ldg(D.model + mi), __ldg(D.model + mi + 1));
            const J2 CpM = j_mul(Cp, M);
            V = j_add(V, j_mul_h(CpM, Cq));
            if (!dd || d == dsel) {
                X = j_add(X, j_mul_h(j_mul(Rpd, M), Cq));        // R_p M C_q^H
                Y = j_add(Y, j_mul_h(j_mul(Rqd, j_herm(M)), Cp)); // R_q M^H C_p^H
                Lp = Lpd;
                Lq = Lqd;
            }
        }
        const J2 Dm = j_from(__ldg(D.vis + 2 * s), __ldg(D.vis + 2 * s + 1));
        J2 wr;
        wr.a = cscale(csub(Dm.a, V.a), w.x); wr.b = cscale(csub(Dm.b, V.b), w.y);
        wr.c = cscale(csub(Dm.c, V.c), w.z); wr.d = cscale(csub(Dm.d, V.d), w.w);
        accumulate_side<TS, true, false>(Ap, Lp, X, w, wr);
        accumulate_side<TS, true, false>(Aq, Lq, Y, make_float4(w.x, w.z, w.y, w.w), j_herm(wr));
    }
    if (__any_sync(0xffffffffu, cur_key >= 0)) flush_pair<KR, KG, Lay>(Ap, Aq, cur_key, cur_pq, lane, A.active, A.acc, nat);
}

// chi^2 = sum over unflagged cross-correlation samples of w |D - V|^2 (FP64 sum of FP32
// terms), and the residual when requested
__global__ void __launch_bounds__(256) dd_residual_kernel(const DDArgs A)
{
    const Data &D = A.D;
    const Chain &C = A.C;
    const int n_chan = D.n_chan, n_dir = A.n_dir;
    const long n = (long)D.n_row * n_chan;
    double tot = 0.0;
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long)gridDim.x * blockDim.x) {
        const int row = (int)(s / n_chan), c = (int)(s % n_chan);
        const int4 meta = __ldg(D.rows + row);
        bool ok = meta.x != meta.y;
        if (ok && D.flag) ok = __ldg(D.flag + s) == 0;
        if (!ok) {
            if (A.resid) { A.resid[2 * s] = make_float4(0, 0, 0, 0); A.resid[2 * s + 1] = make_float4(0, 0, 0, 0); }
            continue;
        }
        int tint[MAXT], fint[MAXT];
#pragma unroll
        for (int j = 0; j < MAXT; ++j) {
            tint[j] = j < C.n_terms ? __ldg(C.t[j].t_map + meta.z) : 0;
            fint[j] = j < C.n_terms ? __ldg(C.t[j].f_map + c) : 0;
        }
        J2 V = j_zero();
        for (int d = 0; d < n_dir; ++d) {
            J2 Cp, Cq, G_, R_;
            dd_factors(A, tint, fint, meta.x, d, Cp, G_, R_);
            dd_factors(A, tint, fint, meta.y, d, Cq, G_, R_);
            const size_t mi = 2 * ((size_t)s * n_dir + d);
            const J2 M = j_from(__ldg(D.model + mi), __ldg(D.model + mi + 1));
            V = j_add(V, j_mul_h(j_mul(Cp, M), Cq));
        }
        const J2 Dm = j_from(__ldg(D.vis + 2 * s), __ldg(D.vis + 2 * s + 1));
        J2 r;
        r.a = csub(Dm.a, V.a); r.b = csub(Dm.b, V.b); r.c = csub(Dm.c, V.c); r.d = csub(Dm.d, V.d);
        const float4 w = __ldg(D.weight + s);
        tot += (double)(w.x * cnorm2(r.a)) + (double)(w.y * cnorm2(r.b)) + (double)(w.z * cnorm2(r.c)) +
               (double)(w.w * cnorm2(r.d));
        if (A.resid) {
            A.resid[2 * s] = make_float4(r.a.x, r.a.y, r.b.x, r.b.y);
            A.resid[2 * s + 1] = make_float4(r.c.x, r.c.y, r.d.x, r.d.y);
        }
    }
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < (int)blockDim.x / 32; ++i) t += red[i];
        atomicAdd(A.chi2, t);
    }
}

} // namespace qc

cudaError_t dd_launch_acc(const qc::DDArgs &a, int ts, int grid_x, cudaStream_t st)
{
    const dim3 grid(grid_x, a.dd_solved ? a.n_dir : 1);
    if (ts == qc::TS_FULL) qc::dd_acc_kernel<qc::TS_FULL><<<grid, 256, 0, st>>>(a);
    else qc::dd_acc_kernel<qc::TS_DIAG><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t dd_launch_residual(const qc::DDArgs &a, int grid, cudaStream_t st)
{
    qc::dd_residual_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}
