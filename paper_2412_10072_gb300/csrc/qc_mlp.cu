// qc_mlp.cu -- learned warm start for the batched solver: per-antenna features,
// a 3 x 128 GELU multilayer perceptron (forward, backward, Adam) and the
// selection of initial gains.
//
// The paper's solvers start from initial estimates where a term allows it
// (Section 4.3, "Initial estimates"); here a small network predicts each
// interval's diagonal gains from per-antenna summaries of its data, and
// Algorithm 1 still iterates to tolerance from there.  All arithmetic is
// FP32 on the CUDA cores (the layers are 128 wide: tensor cores would not be
// fed), with exact-erf GELU.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "../../include/qc.h"
#include "qc_jones.cuh"

namespace {

using namespace qc;

constexpr int IN = QC_MLP_IN, HID = QC_MLP_HIDDEN, OUT = QC_MLP_OUT;
constexpr int SKIP = 6;           // first input feature passed straight to the outputs
// parameter offsets inside the flat float buffer
constexpr int W1 = 0, B1 = W1 + HID * IN, W2 = B1 + HID, B2 = W2 + HID * HID, W3 = B2 + HID, B3 = W3 + HID * HID,
              W4 = B3 + HID, B4 = W4 + OUT * HID, NPARAM = B4 + OUT;
static_assert(NPARAM == QC_MLP_NPARAM, "parameter count");

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ---------------------------------------------------------------------------
// forward: y = x[6..9] + W4 g(W3 g(W2 g(W1 x + b1) + b2) + b3) + b4,  g = GELU
// (the skip term passes the previous-interval gain features straight through,
// so the layers learn the correction to them)
// ---------------------------------------------------------------------------

constexpr int FR = 64;            // rows per CTA tile
constexpr int FT = 256;           // threads

// out[r][j] = sum_k in[r][k] W[j][k] + b[j] for a tile of FR rows and HID outputs;
// thread t computes rows 8*(t/32) .. +8 and outputs 4*(t%32) .. +4.
__device__ __forceinline__ void dense_tile(const float *in, int in_dim, int in_ld, const float *W, const float *b,
                                           float *out, int out_ld, int n_rows, float *z_store, size_t z_ld,
                                           long row0, bool act)
{
    static_assert(FR == 8 * (FT / 32) && HID == 4 * 32, "thread tile covers the CTA tile");
    const int t = threadIdx.x;
    const int r0 = 8 * (t >> 5), j0 = 4 * (t & 31);
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = b[j0 + j];
    for (int k = 0; k < in_dim; ++k) {
        float xv[8], wv[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) xv[i] = in[(r0 + i) * in_ld + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) wv[j] = W[(j0 + j) * in_dim + k];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], wv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = r0 + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (z_store && r < n_rows) z_store[(size_t)(row0 + r) * z_ld + j0 + j] = acc[i][j];
            out[r * out_ld + j0 + j] = act ? gelu(acc[i][j]) : acc[i][j];
        }
    }
}

__global__ void __launch_bounds__(FT) mlp_forward_kernel(const float *__restrict__ P, const float *__restrict__ x,
                                                         long n, float *__restrict__ y, float *__restrict__ z)
{
    extern __shared__ float sm[];
    float *w = sm;                                   // all parameters
    float *h0 = w + NPARAM;                          // [FR][HID]
    float *h1 = h0 + FR * HID;                       // [FR][HID]
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) w[i] = P[i];
    for (long row0 = (long)blockIdx.x * FR; row0 < n; row0 += (long)gridDim.x * FR) {
        const int nr = (int)min((long)FR, n - row0);
        __syncthreads();
        for (int i = threadIdx.x; i < FR * IN; i += blockDim.x) {
            const int r = i / IN, k = i % IN;
            h1[r * IN + k] = r < nr ? x[(row0 + r) * IN + k] : 0.f;
        }
        __syncthreads();
        dense_tile(h1, IN, IN, w + W1, w + B1, h0, HID, nr, z, 3 * HID, row0, true);
        __syncthreads();
        dense_tile(h0, HID, HID, w + W2, w + B2, h1, HID, nr, z ? z + HID : nullptr, 3 * HID, row0, true);
        __syncthreads();
        dense_tile(h1, HID, HID, w + W3, w + B3, h0, HID, nr, z ? z + 2 * HID : nullptr, 3 * HID, row0, true);
        __syncthreads();
        for (int i = threadIdx.x; i < FR * OUT; i += blockDim.x) {
            const int r = i / OUT, j = i % OUT;
            if (r >= nr) continue;
            float s = w[B4 + j] + x[(row0 + r) * IN + SKIP + j];
            for (int k = 0; k < HID; ++k) s = fmaf(h0[r * HID + k], w[W4 + j * HID + k], s);
            y[(row0 + r) * OUT + j] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// backward of the mean squared error over n rows x OUT outputs
// ---------------------------------------------------------------------------

constexpr int BR = 32;            // rows per CTA tile

// dW[j][k] += sum_r d[r][j] a[r][k] over the tile (rows r < nr), db[j] += sum_r d[r][j]
__device__ __forceinline__ void grad_tile(const float *d, int out_dim, const float *a, int in_dim, int in_ld, int nr,
                                          float *dW, float *db)
{
    for (int i = threadIdx.x; i < out_dim * in_dim; i += blockDim.x) {
        const int j = i / in_dim, k = i % in_dim;
        float s = 0.f;
        for (int r = 0; r < nr; ++r) s = fmaf(d[r * HID + j], a[r * in_ld + k], s);
        atomicAdd(dW + i, s);
    }
    for (int j = threadIdx.x; j < out_dim; j += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < nr; ++r) s += d[r * HID + j];
        atomicAdd(db + j, s);
    }
}

__global__ void __launch_bounds__(FT) mlp_backward_kernel(const float *__restrict__ P, const float *__restrict__ x,
                                                          const float *__restrict__ z, const float *__restrict__ y,
                                                          const float *__restrict__ target, long n,
                                                          float *__restrict__ G, double *__restrict__ loss)
{
    extern __shared__ float sm[];
    float *w2 = sm, *w3 = w2 + HID * HID, *w4 = w3 + HID * HID;
    float *xa = w4 + OUT * HID;                      // [BR][IN]
    float *a1 = xa + BR * IN, *a2 = a1 + BR * HID, *a3 = a2 + BR * HID;   // activations [BR][HID]
    float *dA = a3 + BR * HID, *dB = dA + BR * HID;  // deltas [BR][HID]
    __shared__ double red[FT / 32];
    for (int i = threadIdx.x; i < HID * HID; i += blockDim.x) { w2[i] = P[W2 + i]; w3[i] = P[W3 + i]; }
    for (int i = threadIdx.x; i < OUT * HID; i += blockDim.x) w4[i] = P[W4 + i];
    const float scale = 2.f / (float)((double)n * OUT);
    double lsum = 0;
    for (long row0 = (long)blockIdx.x * BR; row0 < n; row0 += (long)gridDim.x * BR) {
        const int nr = (int)min((long)BR, n - row0);
        __syncthreads();
        for (int i = threadIdx.x; i < BR * HID; i += blockDim.x) {
            const int r = i / HID, k = i % HID;
            const bool ok = r < nr;
            const float *zr = z + (size_t)(row0 + r) * 3 * HID;
            a1[i] = ok ? gelu(zr[k]) : 0.f;
            a2[i] = ok ? gelu(zr[HID + k]) : 0.f;
            a3[i] = ok ? gelu(zr[2 * HID + k]) : 0.f;
        }
        for (int i = threadIdx.x; i < BR * IN; i += blockDim.x) {
            const int r = i / IN;
            xa[i] = r < nr ? x[row0 * IN + i] : 0.f;
        }
        // output deltas (in dB, columns 0..OUT-1)
        for (int i = threadIdx.x; i < BR * OUT; i += blockDim.x) {
            const int r = i / OUT, j = i % OUT;
            float d = 0.f;
            if (r < nr) {
                const float e = y[(row0 + r) * OUT + j] - target[(row0 + r) * OUT + j];
                lsum += (double)e * e;
                d = scale * e;
            }
            dB[r * HID + j] = d;
        }
        __syncthreads();
        grad_tile(dB, OUT, a3, HID, HID, nr, G + W4, G + B4);
        // delta of layer 3: (d_out W4) * g'(z3)
        for (int i = threadIdx.x; i < BR * HID; i += blockDim.x) {
            const int r = i / HID, k = i % HID;
            float s = 0.f;
            for (int j = 0; j < OUT; ++j) s = fmaf(dB[r * HID + j], w4[j * HID + k], s);
            dA[i] = r < nr ? s * gelu_d(z[(size_t)(row0 + r) * 3 * HID + 2 * HID + k]) : 0.f;
        }
        __syncthreads();
        grad_tile(dA, HID, a2, HID, HID, nr, G + W3, G + B3);
        for (int i = threadIdx.x; i < BR * HID; i += blockDim.x) {
            const int r = i / HID, k = i % HID;
            float s = 0.f;
            for (int j = 0; j < HID; ++j) s = fmaf(dA[r * HID + j], w3[j * HID + k], s);
            dB[i] = r < nr ? s * gelu_d(z[(size_t)(row0 + r) * 3 * HID + HID + k]) : 0.f;
        }
        __syncthreads();
        grad_tile(dB, HID, a1, HID, HID, nr, G + W2, G + B2);
        for (int i = threadIdx.x; i < BR * HID; i += blockDim.x) {
            const int r = i / HID, k = i % HID;
            float s = 0.f;
            for (int j = 0; j < HID; ++j) s = fmaf(dB[r * HID + j], w2[j * HID + k], s);
            dA[i] = r < nr ? s * gelu_d(z[(size_t)(row0 + r) * 3 * HID + k]) : 0.f;
        }
        __syncthreads();
        grad_tile(dA, HID, xa, IN, IN, nr, G + W1, G + B1);
    }
    for (int d = 16; d > 0; d >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < (int)blockDim.x / 32; ++i) t += red[i];
        atomicAdd(loss, t / ((double)n * OUT));
    }
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

thread_local std::string g_mlp_error;

int cerr(cudaError_t e, const char *what)
{
    g_mlp_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? QC_ENOMEM : QC_ECUDA;
}

size_t fwd_smem() { return sizeof(float) * (NPARAM + 2 * FR * HID); }
size_t bwd_smem() { return sizeof(float) * (2 * HID * HID + OUT * HID + BR * IN + 5 * BR * HID); }

int sm_count()
{
    int dev = 0, n = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

} // namespace

extern "C" int qc_mlp_forward(const float *params, const float *x, int64_t n, float *y, float *z, void *stream)
{
    g_mlp_error.clear();
    if (!params || !x || !y || n < 0) { g_mlp_error = "invalid arguments"; return QC_EINVAL; }
    if (n == 0) return QC_OK;
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
    if (e != cudaSuccess) return cerr(e, "cudaFuncSetAttribute");
    const long tiles = (n + FR - 1) / FR;
    const int grid = (int)std::min<long>(tiles, (long)sm_count());
    mlp_forward_kernel<<<grid, FT, fwd_smem(), (cudaStream_t)stream>>>(params, x, n, y, z);
    e = cudaGetLastError();
    return e == cudaSuccess ? QC_OK : cerr(e, "mlp forward");
}

extern "C" int qc_mlp_backward(const float *params, const float *x, const float *z, const float *y, const float *target,
                               int64_t n, float *grad, double *loss, void *stream)
{
    g_mlp_error.clear();
    if (!params || !x || !z || !y || !target || !grad || !loss || n < 1) { g_mlp_error = "invalid arguments"; return QC_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), st);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem());
    if (e != cudaSuccess) return cerr(e, "mlp backward setup");
    const long tiles = (n + BR - 1) / BR;
    const int grid = (int)std::min<long>(tiles, 2L * sm_count());
    mlp_backward_kernel<<<grid, FT, bwd_smem(), st>>>(params, x, z, y, target, n, grad, loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? QC_OK : cerr(e, "mlp backward");
}

extern "C" int qc_mlp_adam(float *params, const float *grad, float *m, float *v, float lr, float beta1, float beta2,
                           float eps, int32_t step, void *stream)
{
    g_mlp_error.clear();
    if (!params || !grad || !m || !v || step < 1) { g_mlp_error = "invalid arguments"; return QC_EINVAL; }
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, NPARAM, lr, beta1, beta2,
                                                                         eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QC_OK : cerr(e, "adam");
}

extern "C" const char *qc_mlp_last_error(void) { return g_mlp_error.c_str(); }
