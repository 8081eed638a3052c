// qc_robust.cuh -- robust reweighting between solver epochs (Section 4.3, "Robust
// reweighting", after Sob et al. 2020).
//
// The noise is read as complex Student's t with nu degrees of freedom, a scale mixture of
// complex Gaussians, and one expectation-maximisation step reweights the samples between
// epochs from the residual r of the current chain:
//   z_s      = sum_c w_c |r_c|^2 over the k_s correlations with w_c > 0 (the caller's weights,
//              flags and autocorrelations folded in as w = 0);
//   sigma^2  = sum_s lambda_s z_s / sum_s k_s        (M step, the previous factors);
//   lambda_s = (nu + 2 k_s) / (nu + 2 z_s / sigma^2)  (E step, the posterior mean of the
//              mixing variable);
// and the next epoch's weights are w_c lambda_s.  Two passes over the residual: the sums of
// the M step (FP64), then the factors and the weights.
#pragma once
#include <stdint.h>

namespace qc {

__device__ __forceinline__ void robust_power(const float4 w, const float4 a, const float4 b, int &k, float &z)
{
    k = (w.x > 0.f) + (w.y > 0.f) + (w.z > 0.f) + (w.w > 0.f);
    z = w.x * fmaf(a.x, a.x, a.y * a.y) + w.y * fmaf(a.z, a.z, a.w * a.w) + w.z * fmaf(b.x, b.x, b.y * b.y) +
        w.w * fmaf(b.z, b.z, b.w * b.w);
}

// sums[0] += sum_s lambda_s z_s, sums[1] += sum_s k_s (FP64; block partials then one atomic each)
static __global__ void __launch_bounds__(256) robust_sum_kernel(long n_vis, const float4 *resid, const float4 *w0,
                                                                const float *lam, double *sums)
{
    double s_lz = 0.0, s_k = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_vis; i += (long)gridDim.x * blockDim.x) {
        int k;
        float z;
        robust_power(__ldg(w0 + i), __ldg(resid + 2 * i), __ldg(resid + 2 * i + 1), k, z);
        if (!k) continue;
        s_lz += (double)__ldg(lam + i) * (double)z;
        s_k += (double)k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s_lz += __shfl_down_sync(0xffffffffu, s_lz, o);
        s_k += __shfl_down_sync(0xffffffffu, s_k, o);
    }
    __shared__ double r_lz[8], r_k[8];
    if ((threadIdx.x & 31) == 0) { r_lz[threadIdx.x >> 5] = s_lz; r_k[threadIdx.x >> 5] = s_k; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int i = 0; i < (int)blockDim.x / 32; ++i) { a += r_lz[i]; b += r_k[i]; }
        atomicAdd(sums, a);
        atomicAdd(sums + 1, b);
    }
}

// lambda_s and the next epoch's weights w_c lambda_s (unusable samples keep factor 1)
static __global__ void __launch_bounds__(256) robust_apply_kernel(long n_vis, const float4 *resid, const float4 *w0,
                                                                  float *lam, float4 *wf, const double *sums,
                                                                  double nu)
{
    const double sigma2 = sums[1] > 0 ? sums[0] / sums[1] : 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_vis; i += (long)gridDim.x * blockDim.x) {
        const float4 w = __ldg(w0 + i);
        int k;
        float z;
        robust_power(w, __ldg(resid + 2 * i), __ldg(resid + 2 * i + 1), k, z);
        float l = 1.f;
        if (k && sigma2 > 0) l = (float)((nu + 2.0 * k) / (nu + 2.0 * (double)z / sigma2));
        lam[i] = l;
        wf[i] = make_float4(w.x * l, w.y * l, w.z * l, w.w * l);
    }
}

static __global__ void robust_fill_kernel(long n, float *x, float v)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] = v;
}

} // namespace qc
