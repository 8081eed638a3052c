// qc_delay.cuh -- delay terms (QC_TERM_DELAY): gains parameterised per solution interval by
// a phase and a delay per correlation, evaluated at every channel,
//   g_c(nu) = exp(i (phi_c + 2 pi tau_c nu)),  parameters u = (phi_X, tau_X, phi_Y, tau_Y)
// (Scenario 2 of Section 2.4: each gain g_{n,s,a} is tied to a parameter u_{n,a} and the
// normal equations sum over samples, Eq. jhj_case2 and Eq. jhwr_case2).
//
// The accumulate kernels see a delay term as a diagonal term with one bin per (time
// interval, channel): its Jones table is evaluated at every channel, and they form the
// complex blocks JHJ_g, JHr_g of the diagonal entries per channel bin.  Within one channel
// bin the derivative dg/du is constant, so the chain rule of Eq. cp_jacobian applies to
// the per-channel sums exactly:
//   JHJ_u = sum over channels of 2 Re(J2^H JHJ_g J2),  JHr_u = sum of 2 Re(J2^H JHr_g),
//   J2 = d(g_X, g_Y)/du = [[i g_X, 2 pi nu i g_X, 0, 0], [0, 0, i g_Y, 2 pi nu i g_Y]].
// delay_update_kernel forms these 4x4 real blocks in FP64, solves them, updates the
// parameters, re-evaluates the channel table and tests convergence on the gains.
#pragma once
#include "qc_kernels.cuh"

namespace qc {

constexpr double DELAY_TWO_PI = 6.283185307179586476925286766559;

struct DelayArgs {
    int n_tint, n_fint, n_ant, n_chan;   // n_fint: parameter intervals along frequency
    const int *fmap;          // [n_chan] parameter interval of each channel
    const int2 *frange;       // [n_fint] first and last channel of each interval (x < 0: none)
    const double *nu;         // [n_chan] channel frequencies
    double *params;           // FP64 master [n_tint][n_fint][n_ant][4]
    float4 *tab;              // FP32 channel table [n_tint][n_ant][n_chan]: (g_X, g_Y)
    double omega_ref;         // 2 pi nu of the centre of the band: the streaming kernel's sums use
                              // omega' = 2 pi nu - omega_ref
};

// float32 parameters [n_tint][n_fint][n_ant][4] -> FP64 master copy
static __global__ void delay_params_in_kernel(long n, const float *src, double *params)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        params[i] = (double)src[i];
}

__device__ __forceinline__ double2 delay_gain(double phi, double tau, double w)
{
    double s, c;
    sincos(phi + tau * w, &s, &c);
    return make_double2(c, s);
}

// Gain of one correlation, exp(i (phi + tau w)), in float: the phase is formed and reduced to
// [-pi, pi] in FP64, split into a float head and tail, and the head's sine and cosine
// (sincosf) corrected to first order by the tail, which keeps the float table within about
// one float rounding of the exact gain at FP32 cost (FP64 sincos is slow on this part).
__device__ __forceinline__ float2 delay_gain_f32(double phi, double tau, double w)
{
    const double th = phi + tau * w;
    const double r = th - DELAY_TWO_PI * rint(th * (1.0 / DELAY_TWO_PI));
    const float hi = (float)r, lo = (float)(r - (double)hi);
    float s, c;
    sincosf(hi, &s, &c);
    return make_float2(fmaf(-s, lo, c), fmaf(c, lo, s));
}

// |exp(i a) - exp(i b)|^2 = 4 sin^2((a - b) / 2), from the phase change d = a - b (formed in
// FP64 from the parameter changes; the sine of the reduced half angle in float)
__device__ __forceinline__ double delay_change2(double d)
{
    const double h = 0.5 * d;
    const double r = h - 0.5 * DELAY_TWO_PI * rint(h * (2.0 / DELAY_TWO_PI));
    const double sn = (double)sinf((float)r);
    return 4.0 * sn * sn;
}

// channel table from the FP64 parameters, one entry per (time interval, antenna, channel)
static __global__ void delay_tab_kernel(const DelayArgs a)
{
    const long n = (long)a.n_tint * a.n_ant * a.n_chan;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % a.n_chan);
        const long ta = i / a.n_chan;
        const int ant = (int)(ta % a.n_ant), tint = (int)(ta / a.n_ant);
        const double *u = a.params + (((size_t)tint * a.n_fint + a.fmap[c]) * a.n_ant + ant) * 4;
        const double w = DELAY_TWO_PI * a.nu[c];
        const float2 gx = delay_gain_f32(u[0], u[1], w), gy = delay_gain_f32(u[2], u[3], w);
        a.tab[i] = make_float4(gx.x, gx.y, gy.x, gy.y);
    }
}

// FP64 master -> float32 parameters in the public layout
static __global__ void delay_params_out_kernel(long n, const double *params, float *dst)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = (float)params[i];
}

struct DelayUpdArgs {
    DelayArgs d;
    double *acc;              // diagonal accumulators [n_tint * n_chan][n_ant][KG_DIAG] (read, then zeroed)
    int8_t *gain_flags;       // [n_tint][n_fint][n_ant]
    int *iters;               // [n_tint][n_fint]
    uint8_t *active;          // [n_tint * n_chan] channel bins
    const int *n_active_prev; // intervals active entering this iteration (0: nothing to do)
    int *n_active_next;       // incremented for every interval still active after it
    const long long *bin_nvis, *bin_nbytes;   // per channel bin
    unsigned long long *vis_iters, *acc_bytes;
    int k;                    // iteration (1-based)
    double alpha, tol;
};

// One block per parameter interval (time interval x frequency interval), threads over antennas.
// SUMS = false: the accumulators are the complex diagonal blocks of every channel bin
// [n_tint * n_chan][n_ant][KG_DIAG] and activity is kept per channel bin; the chain rule is
// applied here, channel by channel.  SUMS = true: the streaming delay kernel has applied it
// per sample and left the 13 real sums of each (interval, antenna) [bins][n_ant][KG_SUMS]
// (h_XX, h_YY, h_XY times 1, omega', omega'^2; r_X, r_Y times 1, omega') with the centred
// omega' = omega - omega_ref; they are shifted back to omega here in FP64, so that a band of
// one frequency gives the exactly proportional phase and delay columns of the oracle (a
// singular block) rather than FP32 rounding; activity per interval.
constexpr int KG_SUMS = 16;

template <bool SUMS>
static __global__ void __launch_bounds__(128) delay_update_kernel(const DelayUpdArgs u)
{
    if (*u.n_active_prev == 0) return;
    const DelayArgs &d = u.d;
    const int bin = blockIdx.x;
    const int tint = bin / d.n_fint, fu = bin % d.n_fint;
    const int2 fr = d.frange[fu];
    const size_t cb0 = (size_t)tint * d.n_chan;            // first channel bin of the time interval
    if (fr.x < 0) {
        // no channel maps to this interval: no data, the parameters stay as they are
        if (u.k == 1) {
            for (int ant = threadIdx.x; ant < d.n_ant; ant += blockDim.x)
                if (u.gain_flags) u.gain_flags[(size_t)bin * d.n_ant + ant] = 1;
            if (threadIdx.x == 0 && u.iters) u.iters[bin] = 1;
        }
        return;
    }
    if (!u.active[SUMS ? (size_t)bin : cb0 + fr.x]) return;
    double num = 0, den = 0;
    for (int ant = threadIdx.x; ant < d.n_ant; ant += blockDim.x) {
        double *P = d.params + ((size_t)bin * d.n_ant + ant) * 4;
        const double u0 = P[0], u1 = P[1], u2 = P[2], u3 = P[3];
        double2 M[4][4], b[4], x[4];
        for (int i = 0; i < 4; ++i) {
            b[i] = make_double2(0.0, 0.0);
            for (int j = 0; j < 4; ++j) M[i][j] = make_double2(0.0, 0.0);
        }
        if (SUMS) {
            double *A = u.acc + ((size_t)bin * d.n_ant + ant) * KG_SUMS;
            double S[13];
            for (int i = 0; i < 13; ++i) { S[i] = A[i]; A[i] = 0.0; }
            // sum h w^k with w = w' + w0:  h w = h w' + w0 h,  h w^2 = h w'^2 + 2 w0 h w' + w0^2 h
            const double w0 = d.omega_ref;
            for (int base = 0; base <= 10; base += (base == 3 ? 7 : 3)) {
                const double s0 = S[base], s1 = S[base + 1], s2 = S[base + 2];
                S[base + 1] = s1 + w0 * s0;
                S[base + 2] = s2 + 2.0 * w0 * s1 + w0 * w0 * s0;
            }
            S[7] += w0 * S[6];
            S[9] += w0 * S[8];
            const int o2[2][2] = { { 0, 1 }, { 1, 2 } };    // power of omega of block entry (i, j)
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    M[i][j].x = 2.0 * S[o2[i][j]];
                    M[2 + i][2 + j].x = 2.0 * S[3 + o2[i][j]];
                    M[i][2 + j].x = 2.0 * S[10 + o2[i][j]];
                    M[2 + j][i].x = 2.0 * S[10 + o2[i][j]];
                }
            b[0].x = 2.0 * S[6];
            b[1].x = 2.0 * S[7];
            b[2].x = 2.0 * S[8];
            b[3].x = 2.0 * S[9];
        }
        for (int c = fr.x; !SUMS && c <= fr.y; ++c) {
            double *A = u.acc + ((cb0 + c) * d.n_ant + ant) * KG_DIAG;
            const double h00 = A[0], h11 = A[1];
            const double2 h01 = make_double2(A[2], A[3]), j0 = make_double2(A[4], A[5]), j1 = make_double2(A[6], A[7]);
            for (int i = 0; i < KG_DIAG; ++i) A[i] = 0.0;
            const double w = DELAY_TWO_PI * d.nu[c];
            const double2 gx = delay_gain(u0, u1, w), gy = delay_gain(u2, u3, w);
            const double f[2] = { 1.0, w };
            // Re(conj(g_X) JHJ_g[X][Y] g_Y): the X-Y coupling (zero without a left factor)
            const double2 t = make_double2(gx.x * h01.x + gx.y * h01.y, gx.x * h01.y - gx.y * h01.x);
            const double xy = t.x * gy.x - t.y * gy.y;
            // Im(conj(g_c) JHr_g[c]) of each correlation
            const double rx = gx.x * j0.y - gx.y * j0.x, ry = gy.x * j1.y - gy.y * j1.x;
            for (int i = 0; i < 2; ++i) {
                for (int j = 0; j < 2; ++j) {
                    M[i][j].x += 2.0 * h00 * f[i] * f[j];
                    M[2 + i][2 + j].x += 2.0 * h11 * f[i] * f[j];
                    M[i][2 + j].x += 2.0 * xy * f[i] * f[j];
                    M[2 + j][i].x += 2.0 * xy * f[i] * f[j];
                }
                b[i].x += 2.0 * rx * f[i];
                b[2 + i].x += 2.0 * ry * f[i];
            }
        }
        const int singular = block_solve<4>(M, b, x);
        if (!singular)
            for (int e = 0; e < 4; ++e) P[e] += u.alpha * x[e].x;
        if (u.gain_flags) u.gain_flags[(size_t)bin * d.n_ant + ant] = (int8_t)singular;
        if (SUMS) {
            // the parameter change, kept in the (already read) sums for the channel pass below
            double *A = u.acc + ((size_t)bin * d.n_ant + ant) * KG_SUMS;
            A[0] = P[0] - u0;
            A[1] = P[1] - u1;
            A[2] = P[2] - u2;
            A[3] = P[3] - u3;
            continue;
        }
        // re-evaluate the channel table; relative change of the gains over the interval's channels
        // (the gains have unit modulus: |g_new - g_old|^2 = 4 sin^2 of half the phase change,
        // |g_new|^2 = 1 per correlation)
        const double d0 = P[0] - u0, d1 = P[1] - u1, d2 = P[2] - u2, d3 = P[3] - u3;
        for (int c = fr.x; c <= fr.y; ++c) {
            const double w = DELAY_TWO_PI * d.nu[c];
            const float2 nx = delay_gain_f32(P[0], P[1], w), ny = delay_gain_f32(P[2], P[3], w);
            d.tab[((size_t)tint * d.n_ant + ant) * d.n_chan + c] = make_float4(nx.x, nx.y, ny.x, ny.y);
            num += delay_change2(d0 + d1 * w) + delay_change2(d2 + d3 * w);
            den += 2.0;
        }
    }
    if (SUMS) {
        // the channel table and the change of the gains, spread over the block's threads by
        // (antenna, channel)
        __syncthreads();
        const int nch = fr.y - fr.x + 1;
        const long n = (long)d.n_ant * nch;
        for (long i = threadIdx.x; i < n; i += blockDim.x) {
            const int ant = (int)(i / nch), c = fr.x + (int)(i - (long)ant * nch);
            const double *P = d.params + ((size_t)bin * d.n_ant + ant) * 4;
            const double *A = u.acc + ((size_t)bin * d.n_ant + ant) * KG_SUMS;
            const double w = DELAY_TWO_PI * d.nu[c];
            const float2 nx = delay_gain_f32(P[0], P[1], w), ny = delay_gain_f32(P[2], P[3], w);
            d.tab[((size_t)tint * d.n_ant + ant) * d.n_chan + c] = make_float4(nx.x, nx.y, ny.x, ny.y);
            num += delay_change2(A[0] + A[1] * w) + delay_change2(A[2] + A[3] * w);
            den += 2.0;
        }
        __syncthreads();
        for (int ant = threadIdx.x; ant < d.n_ant; ant += blockDim.x) {
            double *A = u.acc + ((size_t)bin * d.n_ant + ant) * KG_SUMS;
            A[0] = A[1] = A[2] = A[3] = 0.0;
        }
    }
    __shared__ double s_num[4], s_den[4];
    for (int dd = 16; dd > 0; dd >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, dd);
        den += __shfl_down_sync(0xffffffffu, den, dd);
    }
    const int wi = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_num[wi] = num; s_den[wi] = den; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tn = 0, td = 0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) { tn += s_num[i]; td += s_den[i]; }
        const double delta = td > 0 ? sqrt(tn / td) : 0.0;
        if (u.iters) u.iters[bin] = u.k;
        unsigned long long nv = 0, nb = 0;
        for (int c = fr.x; c <= fr.y; ++c) {
            nv += (unsigned long long)u.bin_nvis[cb0 + c];
            nb += (unsigned long long)u.bin_nbytes[cb0 + c];
        }
        atomicAdd(u.vis_iters, nv);
        atomicAdd(u.acc_bytes, nb);
        if (delta < u.tol) {
            if (SUMS) u.active[bin] = 0;
            else
                for (int c = fr.x; c <= fr.y; ++c) u.active[cb0 + c] = 0;
        } else {
            atomicAdd(u.n_active_next, 1);
        }
    }
}

} // namespace qc

namespace qc {

// ---------------------------------------------------------------------------
// initial estimate of a delay term (Section 4.3, "Initial estimates"): the peak of the
// Fourier transform along frequency of the baselines that include the reference antenna
// ---------------------------------------------------------------------------

struct DelayInitArgs {
    int n_row, n_chan, n_ant, ref, n_tint, n_fint;
    const int4 *rows;          // [n_row] {ant1, ant2, time, baseline}
    const float4 *vis;         // [n_row][n_chan] x 2
    const float4 *model;       // [n_row][n_chan] x 2, or nullptr (FP16 model)
    const uint4 *model16;      // [n_row][n_chan], or nullptr
    const float *bl_scale;     // [n_bl] FP16 model scales
    const float4 *wf;          // [n_row][n_chan] weights, zero where flagged or autocorrelation
    const int *t_map;          // [n_time] time interval of each data time
    float2 *x;                 // [n_tint][n_ant][2][n_chan] spectra (zeroed before)
    const int4 *fint_info;     // [n_fint] {first channel, channels, N, log2 N}
    const double *fint_dnu;    // [n_fint] channel spacing
    const double *fint_nu0;    // [n_fint] frequency of the first channel
    float *params;             // [n_tint][n_fint][n_ant][4] out
};

// x[t][a][c][chan] += w d conj(m) of correlation c (XX, YY) over the rows on baselines with
// the reference antenna, conjugated for rows (ref, a).  One warp per row, lanes over channels.
static __global__ void delay_gather_kernel(const DelayInitArgs a)
{
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long n_warps = ((long)gridDim.x * blockDim.x) >> 5;
    for (long row = warp; row < a.n_row; row += n_warps) {
        const int4 r = a.rows[row];
        if (r.x == r.y || (r.x != a.ref && r.y != a.ref)) continue;
        const int ant = r.x == a.ref ? r.y : r.x;
        const bool flip = r.x == a.ref;
        float2 *xa = a.x + ((size_t)a.t_map[r.z] * a.n_ant + ant) * 2 * a.n_chan;
        for (int c = lane; c < a.n_chan; c += 32) {
            const size_t s = (size_t)row * a.n_chan + c;
            const float4 w = a.wf[s];
            if (w.x == 0.f && w.y == 0.f && w.z == 0.f && w.w == 0.f) continue;
            const J2 D = j_from(a.vis[2 * s], a.vis[2 * s + 1]);
            const J2 M = a.model ? j_from(a.model[2 * s], a.model[2 * s + 1]) : load_model16(a.model16[s], a.bl_scale[r.w]);
            float2 zx = cscale(cmulc(D.a, M.a), w.x), zy = cscale(cmulc(D.d, M.d), w.w);
            if (flip) { zx = cconj(zx); zy = cconj(zy); }
            atomicAdd(&xa[c].x, zx.x);
            atomicAdd(&xa[c].y, zx.y);
            atomicAdd(&xa[a.n_chan + c].x, zy.x);
            atomicAdd(&xa[a.n_chan + c].y, zy.y);
        }
    }
}

// One block per (time interval, frequency interval, antenna, correlation): the spectrum over
// the interval's channels, zero-padded to N (a power of two), transformed by a radix-2 FFT in
// shared memory, X_k = sum_c x_c exp(-2 pi i k c / N); the peak |X_k| (lowest signed k
// among equal values) gives tau = k / (N dnu) and phi = arg X_k - 2 pi tau nu_0.
static __global__ void __launch_bounds__(256) delay_peak_kernel(const DelayInitArgs a)
{
    extern __shared__ float2 fbuf[];
    const int corr = blockIdx.x & 1;
    const int rest = blockIdx.x >> 1;
    const int ant = rest % a.n_ant;
    const int bin = rest / a.n_ant;                         // tint * n_fint + fint
    const int fi = bin % a.n_fint, tint = bin / a.n_fint;
    float *out = a.params + ((size_t)bin * a.n_ant + ant) * 4 + 2 * corr;
    const int4 info = a.fint_info[fi];
    const int c0 = info.x, n_c = info.y, N = info.z, lg = info.w;
    const float2 *xs = a.x + (((size_t)tint * a.n_ant + ant) * 2 + corr) * a.n_chan + c0;
    if (ant == a.ref || n_c == 0) {
        if (threadIdx.x == 0) { out[0] = 0.f; out[1] = 0.f; }
        return;
    }
    if (n_c == 1) {
        if (threadIdx.x == 0) {
            const float2 v = xs[0];
            out[0] = (v.x != 0.f || v.y != 0.f) ? atan2f(v.y, v.x) : 0.f;
            out[1] = 0.f;
        }
        return;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) fbuf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int c = threadIdx.x; c < n_c; c += blockDim.x) fbuf[__brev((unsigned)c) >> (32 - lg)] = xs[c];
    __syncthreads();
    for (int len = 2, lh = 0; len <= N; len <<= 1, ++lh) {
        const int half = len >> 1;
        for (int j = threadIdx.x; j < N / 2; j += blockDim.x) {
            const int grp = j >> lh, pos = j & (half - 1);
            const int i0 = grp * len + pos, i1 = i0 + half;
            float sn, cs;
            sincospif(-2.0f * (float)pos / (float)len, &sn, &cs);
            const float2 u = fbuf[i0], v = cmul(fbuf[i1], make_float2(cs, sn));
            fbuf[i0] = cadd(u, v);
            fbuf[i1] = csub(u, v);
        }
        __syncthreads();
    }
    float best = -1.f;
    int bk = 1 << 30;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int ks = i < N / 2 ? i : i - N;
        const float m = cnorm2(fbuf[i]);
        if (m > best || (m == best && ks < bk)) { best = m; bk = ks; }
    }
    for (int d = 16; d > 0; d >>= 1) {
        const float om = __shfl_down_sync(0xffffffffu, best, d);
        const int ok = __shfl_down_sync(0xffffffffu, bk, d);
        if (om > best || (om == best && ok < bk)) { best = om; bk = ok; }
    }
    __shared__ float s_best[8];
    __shared__ int s_k[8];
    const int wi = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_best[wi] = best; s_k[wi] = bk; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
            if (s_best[i] > best || (s_best[i] == best && s_k[i] < bk)) { best = s_best[i]; bk = s_k[i]; }
        if (!(best > 0.f)) { out[0] = 0.f; out[1] = 0.f; return; }
        const float2 X = fbuf[bk >= 0 ? bk : bk + N];
        const double tau = (double)bk / ((double)N * a.fint_dnu[fi]);
        double phi = atan2((double)X.y, (double)X.x) - DELAY_TWO_PI * tau * a.fint_nu0[fi];
        phi -= DELAY_TWO_PI * floor(phi / DELAY_TWO_PI + 0.5);
        out[0] = (float)phi;
        out[1] = (float)tau;
    }
}

} // namespace qc
