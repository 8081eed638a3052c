// qc_noalloc.cu -- chi^2 of a one-term problem without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a real-time pipeline whose
// device memory is planned and reserved up front (an unplanned allocation can
// fail, fragment the budget or stall the stream), or a host framework that owns
// every device buffer through its own pool and forbids foreign allocations.
// qc_residual_noalloc serves them: the caller passes every input and the output
// as device pointers, and the only scratch the computation needs -- the gain
// table rearranged for the kernel and the per-CTA partial sums -- lives in the
// file-scope array below, which the module reserves once on every device that
// loads it and keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/qc.h"
#include "qc_kernels.cuh"

void qc_internal_set_error(const char *msg);

namespace {

using namespace qc;

constexpr size_t TAB_BYTES = (size_t)QC_NOALLOC_MAX_GAINS * 2 * sizeof(float4);
constexpr int MAX_PARTS = QC_NOALLOC_MAX_BLOCKS;
constexpr size_t PARTS_BYTES = MAX_PARTS * sizeof(double);

// The scratch: [gain table (up to 2 float4 per entry) | per-CTA partial sums | bad-index word].
static __device__ __align__(256) unsigned char g_noalloc_scratch[TAB_BYTES + PARTS_BYTES + 256];

std::mutex g_mutex;
void *g_scratch_addr[256] = { nullptr };   // device address of g_noalloc_scratch, per device ordinal

// public layout [n_tint][n_fint][n_ant][4] (phase: [..][2]) -> kernel table [n_tint][n_ant][n_fint]
// (also clears the bad-index word of this call: the kernels after it run on the same stream)
__global__ void noalloc_table_kernel(int type, int n_tint, int n_fint, int n_ant, const void *src, float4 *tab,
                                     int *bad)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *bad = 0;
    const long n = (long)n_tint * n_fint * n_ant;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int ant = (int)(i % n_ant);
        const long bin = i / n_ant;
        const int tint = (int)(bin / n_fint), fint = (int)(bin % n_fint);
        const size_t t = ((size_t)tint * n_ant + ant) * n_fint + fint;
        if (type == QC_TERM_PHASE) {
            const float *ph = (const float *)src + 2 * i;
            float s0, c0, s1, c1;
            sincosf(ph[0], &s0, &c0);
            sincosf(ph[1], &s1, &c1);
            tab[t] = make_float4(c0, s0, c1, s1);
        } else {
            const float2 *g = (const float2 *)src + 4 * i;
            if (type == QC_TERM_FULL) {
                tab[2 * t] = make_float4(g[0].x, g[0].y, g[1].x, g[1].y);
                tab[2 * t + 1] = make_float4(g[2].x, g[2].y, g[3].x, g[3].y);
            } else {
                tab[t] = make_float4(g[0].x, g[0].y, g[3].x, g[3].y);
            }
        }
    }
}

// per-CTA partial sums of w |d - G_p M G_q^H|^2 over unflagged cross-correlation samples.
// The index arrays live in device memory, where the host cannot check them: every index
// is checked here before it is used, and a sample with an antenna, time or interval index
// out of range is skipped and recorded in *bad (the sum kernel then reports NaN).
__global__ void __launch_bounds__(256) noalloc_chi2_kernel(int n_row, int n_chan, int n_ant, int n_time,
                                                           const float4 *vis, const float4 *model,
                                                           const float4 *weight, const uint8_t *flag, const int *ant1,
                                                           const int *ant2, const int *time_idx, DevTerm term,
                                                           double *parts, int *bad)
{
    const long n = (long)n_row * n_chan;
    double tot = 0.0;
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long)gridDim.x * blockDim.x) {
        const int row = (int)(s / n_chan), c = (int)(s % n_chan);
        const int p = __ldg(ant1 + row), q = __ldg(ant2 + row);
        const int t = __ldg(time_idx + row);
        if (p < 0 || p >= n_ant || q < 0 || q >= n_ant || t < 0 || t >= n_time) {
            atomicOr(bad, 1);
            continue;
        }
        if (p == q || (flag && __ldg(flag + s))) continue;
        const int tint = __ldg(term.t_map + t), fint = __ldg(term.f_map + c);
        if (tint < 0 || tint >= term.n_tint || fint < 0 || fint >= term.n_fint) {
            atomicOr(bad, 1);
            continue;
        }
        const J2 Gp = fetch_jones(term, n_ant, tint, fint, p);
        const J2 Gq = fetch_jones(term, n_ant, tint, fint, q);
        const J2 M = j_from(__ldg(model + 2 * s), __ldg(model + 2 * s + 1));
        const J2 V = j_mul_h(j_mul(Gp, M), Gq);
        const J2 D = j_from(__ldg(vis + 2 * s), __ldg(vis + 2 * s + 1));
        const float4 w = __ldg(weight + s);
        tot += (double)(w.x * cnorm2(csub(D.a, V.a))) + (double)(w.y * cnorm2(csub(D.b, V.b))) +
               (double)(w.z * cnorm2(csub(D.c, V.c))) + (double)(w.w * cnorm2(csub(D.d, V.d)));
    }
    for (int d = 16; d > 0; d >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, d);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < (int)blockDim.x / 32; ++i) t += red[i];
        parts[blockIdx.x] = t;          // every CTA overwrites its own slot: nothing to clear
    }
}

// fixed-order sum of the partials (the result does not depend on CTA scheduling); NaN when
// the chi^2 kernel met an index out of range
__global__ void noalloc_sum_kernel(const double *parts, int n, const int *bad, double *out)
{
    __shared__ double red[32];
    double t = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += parts[i];
    for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int i = 0; i < (int)blockDim.x / 32; ++i) s += red[i];
        *out = *bad ? __longlong_as_double(0x7ff8000000000000ll) : s;
    }
}

int fail(int code, const char *msg)
{
    qc_internal_set_error(msg);
    return code;
}

} // namespace

extern "C" int qc_residual_noalloc(int32_t n_row, int32_t n_chan, int32_t n_ant, int32_t n_time, const void *data,
                                   const void *model,
                                   const float *weight, const uint8_t *flag, const int32_t *ant1, const int32_t *ant2,
                                   const int32_t *time_idx, int32_t type, int32_t n_tint, int32_t n_fint,
                                   const int32_t *t_map, const int32_t *f_map, const void *gains, double *chi2,
                                   void *stream)
{
    qc_internal_set_error("");
    if (n_row < 0 || n_chan < 1 || n_ant < 2 || n_time < 1 || n_tint < 1 || n_fint < 1)
        return fail(QC_EINVAL, "qc_residual_noalloc: invalid sizes");
    if (type != QC_TERM_DIAG && type != QC_TERM_FULL && type != QC_TERM_PHASE)
        return fail(QC_EINVAL, "qc_residual_noalloc: unknown term type");
    if ((long long)n_tint * n_fint * n_ant > QC_NOALLOC_MAX_GAINS)
        return fail(QC_EINVAL, "qc_residual_noalloc: n_tint * n_fint * n_ant exceeds QC_NOALLOC_MAX_GAINS "
                               "(the fixed scratch of this entry point); use qc_residual instead");
    if (!data || !model || !weight || !ant1 || !ant2 || !time_idx || !t_map || !f_map || !gains || !chi2)
        return fail(QC_EINVAL, "qc_residual_noalloc: a required pointer is NULL");
    for (const void *ptr : { data, model, (const void *)weight })
        if ((uintptr_t)ptr % 16) return fail(QC_EINVAL, "qc_residual_noalloc: data/model/weight must be 16-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) return fail(QC_ECUDA, "qc_residual_noalloc: no current device");
    void *scratch;
    {
        // first call on this device: look up the device address of the static scratch
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_scratch_addr[dev] = nullptr;
                return fail(QC_ECUDA, "qc_residual_noalloc: cudaGetSymbolAddress of the scratch failed");
            }
        }
        scratch = g_scratch_addr[dev];
    }
    float4 *tab = (float4 *)scratch;
    double *parts = (double *)((unsigned char *)scratch + TAB_BYTES);
    int *bad = (int *)((unsigned char *)scratch + TAB_BYTES + PARTS_BYTES);
    cudaStream_t st = (cudaStream_t)stream;
    const long n_gain = (long)n_tint * n_fint * n_ant;
    noalloc_table_kernel<<<(int)std::min<long>((n_gain + 255) / 256, 1024), 256, 0, st>>>(type, n_tint, n_fint, n_ant,
                                                                                       gains, tab, bad);
    DevTerm term;
    term.type = type;
    term.n_tint = n_tint;
    term.n_fint = n_fint;
    term.t_map = t_map;
    term.f_map = f_map;
    term.tab = tab;
    const long n = (long)n_row * n_chan;
    const int grid = (int)std::max(1L, std::min<long>((n + 255) / 256, (long)MAX_PARTS));
    noalloc_chi2_kernel<<<grid, 256, 0, st>>>(n_row, n_chan, n_ant, n_time, (const float4 *)data,
                                             (const float4 *)model, (const float4 *)weight, flag, ant1, ant2, time_idx,
                                             term, parts, bad);
    noalloc_sum_kernel<<<1, 256, 0, st>>>(parts, grid, bad, chi2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(QC_ECUDA, "qc_residual_noalloc: kernel launch failed");
    return QC_OK;
}
