// qc_api.cu -- host side of libqc: validation, device staging, the chain
// schedule of epochs x terms x iterations (Section 4.3 of arxiv 2412.10072)
// and CUDA-graph replay of each term's iteration loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/qc.h"
#include "qc_internal.h"
#include "qc_kernels.cuh"

using namespace qc;

namespace {

thread_local std::string g_create_error;

__global__ void bl_scale_kernel(const float4 *model, const int4 *rows, int n_row, int n_chan, unsigned *scale_bits)
{
    const long n = (long)n_row * n_chan;
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long)gridDim.x * blockDim.x) {
        const int row = (int)(s / n_chan);
        const int4 meta = rows[row];
        if (meta.x == meta.y) continue;
        const float4 a = model[2 * s], b = model[2 * s + 1];
        float m = fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))),
                        fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w))));
        if (!(m <= 3.0e38f)) m = 0.f;           // non-finite (flagged garbage) does not set the scale
        atomicMax(scale_bits + meta.w, __float_as_uint(m));
    }
}

__global__ void pack16_kernel(const float4 *model, const int4 *rows, int n_row, int n_chan, const float *scale,
                              uint4 *out)
{
    const long n = (long)n_row * n_chan;
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long)gridDim.x * blockDim.x) {
        const int row = (int)(s / n_chan);
        const int4 meta = rows[row];
        const float sc = meta.x == meta.y ? 1.f : scale[meta.w];
        const float inv = sc > 0.f ? 1.f / sc : 0.f;
        const float4 a = model[2 * s], b = model[2 * s + 1];
        __half2 h0 = __floats2half2_rn(a.x * inv, a.y * inv), h1 = __floats2half2_rn(a.z * inv, a.w * inv);
        __half2 h2 = __floats2half2_rn(b.x * inv, b.y * inv), h3 = __floats2half2_rn(b.z * inv, b.w * inv);
        uint4 o;
        o.x = *reinterpret_cast<unsigned *>(&h0);
        o.y = *reinterpret_cast<unsigned *>(&h1);
        o.z = *reinterpret_cast<unsigned *>(&h2);
        o.w = *reinterpret_cast<unsigned *>(&h3);
        out[s] = o;
    }
}

__global__ void fix_scale_kernel(unsigned *bits, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float v = __uint_as_float(bits[i]);
        reinterpret_cast<float *>(bits)[i] = v > 0.f ? v : 1.f;
    }
}

// user gains [n_tint][n_fint][n_ant][4] (complex64) or phases [..][2] (float32)
// -> FP64 master parameters and FP32 kernel table [n_tint][n_ant][n_fint]
__global__ void gains_in_kernel(int type, int n_tint, int n_fint, int n_ant, const void *src, double *params,
                                float4 *tab)
{
    const long n = (long)n_tint * n_fint * n_ant;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int ant = (int)(i % n_ant);
        const long bin = i / n_ant;
        const int tint = (int)(bin / n_fint), fint = (int)(bin % n_fint);
        const size_t t = ((size_t)tint * n_ant + ant) * n_fint + fint;
        if (type == 2) {
            const float *ph = (const float *)src + 2 * i;
            params[2 * i] = ph[0];
            params[2 * i + 1] = ph[1];
            double s0, c0, s1, c1;
            sincos((double)ph[0], &s0, &c0);
            sincos((double)ph[1], &s1, &c1);
            tab[t] = make_float4((float)c0, (float)s0, (float)c1, (float)s1);
            continue;
        }
        const float2 *g = (const float2 *)src + 4 * i;
        double2 *P = reinterpret_cast<double2 *>(params) + 4 * i;
        for (int e = 0; e < 4; ++e) P[e] = make_double2(g[e].x, g[e].y);
        if (type == 0) { P[1] = make_double2(0, 0); P[2] = make_double2(0, 0); }
        if (type == 1) {
            tab[2 * t] = make_float4(g[0].x, g[0].y, g[1].x, g[1].y);
            tab[2 * t + 1] = make_float4(g[2].x, g[2].y, g[3].x, g[3].y);
        } else {
            tab[t] = make_float4(g[0].x, g[0].y, g[3].x, g[3].y);
        }
    }
}

__global__ void gains_out_kernel(int type, long n, const double *params, void *dst)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        if (type == 2) {
            float *ph = (float *)dst + 2 * i;
            ph[0] = (float)params[2 * i];
            ph[1] = (float)params[2 * i + 1];
            continue;
        }
        float2 *g = (float2 *)dst + 4 * i;
        const double2 *P = reinterpret_cast<const double2 *>(params) + 4 * i;
        for (int e = 0; e < 4; ++e) g[e] = make_float2((float)P[e].x, (float)P[e].y);
        if (type == 0) { g[1] = make_float2(0.f, 0.f); g[2] = make_float2(0.f, 0.f); }
    }
}

__global__ void bin_bytes_kernel(int n, const long long *nvis, const long long *nunflag, long long b_flag,
                                 long long b_unflag, long long *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = nvis[i] * b_flag + nunflag[i] * b_unflag;
}

__global__ void init_term_kernel(int n_bins, uint8_t *active, int *cnt, int n_cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_bins) active[i] = 1;
    if (i < n_cnt) cnt[i] = i == 0 ? n_bins : 0;
}

template <typename T> size_t nbytes(size_t n) { return n * sizeof(T); }

int grid_for(long n, int block, int sm)
{
    long g = (n + block - 1) / block;
    return (int)std::max(1L, std::min(g, (long)sm * 32));
}

} // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

qc_ctx::~qc_ctx()
{
    for (auto &b : tb) if (b.exec) cudaGraphExecDestroy(b.exec);
    for (void *p : owned) qc_dev_free(p);
    for (auto e : events) cudaEventDestroy(e);
    if (own_stream) cudaStreamDestroy(own_stream);
}

int qc_ctx::fail(int code, const std::string &msg)
{
    err = msg;
    return code;
}

int qc_ctx::cuda_fail(cudaError_t e, const char *what)
{
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? QC_ENOMEM : QC_ECUDA;
}

namespace {
std::atomic<long long> g_alloc_countdown{0};   // > 0: the allocation that brings it to 0 fails
std::atomic<long long> g_live_allocs{0};
std::atomic<unsigned long long> g_wait_limit_ns{2000000000ull};
std::atomic<int> g_wait_stall{-1};
} // namespace

cudaError_t qc_dev_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    long long c = g_alloc_countdown.load();
    while (c > 0 && !g_alloc_countdown.compare_exchange_weak(c, c - 1)) {}
    if (c == 1) return cudaErrorMemoryAllocation;      // injected on the host: cudaMalloc is not called
    const cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) ++g_live_allocs;
    return e;
}

void qc_dev_free(void *p)
{
    if (!p) return;
    cudaFree(p);
    --g_live_allocs;
}

uint64_t qc_wait_limit_ns() { return g_wait_limit_ns.load(); }
int qc_wait_stall_stage() { return g_wait_stall.load(); }

extern "C" void qc_test_fail_alloc(int64_t n) { g_alloc_countdown.store(n > 0 ? n : 0); }
extern "C" int64_t qc_test_live_allocs(void) { return g_live_allocs.load(); }
extern "C" void qc_test_wait_limit(int64_t limit_ns, int32_t stall_stage)
{
    g_wait_limit_ns.store(limit_ns > 0 ? (unsigned long long)limit_ns : 2000000000ull);
    g_wait_stall.store(stall_stage >= 0 ? stall_stage : -1);
}

void *qc_ctx::alloc(size_t bytes, cudaError_t *e)
{
    void *p = nullptr;
    *e = qc_dev_malloc(&p, bytes);
    if (*e == cudaSuccess) owned.push_back(p);
    return p;
}

void qc_ctx::release(void *p)
{
    auto it = std::find(owned.begin(), owned.end(), p);
    if (it != owned.end()) { qc_dev_free(p); owned.erase(it); }
}

int qc_ctx::ensure(Buf &b, size_t bytes)
{
    if (b.bytes >= bytes && b.ptr) return QC_OK;
    if (b.ptr) release(b.ptr);
    cudaError_t e;
    b.ptr = alloc(bytes, &e);
    b.bytes = b.ptr ? std::max<size_t>(bytes, 16) : 0;
    if (e != cudaSuccess) { b.ptr = nullptr; return cuda_fail(e, "cudaMalloc"); }
    return QC_OK;
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return c->cuda_fail(e_, #call); \
    } while (0)

extern "C" int qc_create(const qc_problem *p, qc_ctx **out)
{
    g_create_error.clear();
    if (!out) { g_create_error = "out is NULL"; return QC_EINVAL; }
    *out = nullptr;
    auto bad = [](const char *m) { g_create_error = m; return QC_EINVAL; };
    if (!p) return bad("problem is NULL");
    if (p->n_corr != 4) return bad("n_corr must be 4");
    if (p->n_dir < 1 || p->n_dir > QC_MAX_DIRS) return bad("n_dir must be in [1, QC_MAX_DIRS]");
    if (p->n_dir > 1 && p->model_fp16) return bad("the float16 model takes one direction (n_dir = 1)");
    if (p->n_row < 0 || p->n_chan < 1 || p->n_ant < 2 || p->n_time < 1) return bad("invalid sizes");
    if ((long long)p->n_row * p->n_chan > (1LL << 40)) return bad("problem too large");
    if (!p->data || !p->model || !p->weight) return bad("data, model and weight are required");
    if (!p->ant1 || !p->ant2 || !p->time_idx) return bad("ant1, ant2 and time_idx are required (host arrays)");
    if (p->memory != QC_MEM_HOST && p->memory != QC_MEM_DEVICE) return bad("memory must be QC_MEM_HOST or QC_MEM_DEVICE");
    for (int r = 0; r < p->n_row; ++r) {
        if (p->ant1[r] < 0 || p->ant1[r] >= p->n_ant || p->ant2[r] < 0 || p->ant2[r] >= p->n_ant)
            return bad("antenna index out of range");
        if (p->time_idx[r] < 0 || p->time_idx[r] >= p->n_time) return bad("time index out of range");
    }
    if (p->memory == QC_MEM_DEVICE) {
        for (const void *ptr : { p->data, p->model, (const void *)p->weight })
            if (((uintptr_t)ptr) % 16) return bad("device data/model/weight must be 16-byte aligned");
    }

    std::unique_ptr<qc_ctx> c(new qc_ctx());
    c->n_row = p->n_row;
    c->n_chan = p->n_chan;
    c->n_ant = p->n_ant;
    c->n_time = p->n_time;
    c->n_dir = p->n_dir;
    c->m16 = p->model_fp16 != 0;
    c->has_flag = p->flag != nullptr;
    {
        cudaError_t e = cudaGetDevice(&c->dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->dev);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { g_create_error = std::string("CUDA init: ") + cudaGetErrorString(e); return QC_ECUDA; }
    }
    // rows {ant1, ant2, time, baseline id}; strips: rows of one (ant1, ant2) pair in time order
    const int na = p->n_ant;
    std::vector<int> bl_of_pair((size_t)na * na, -1);
    std::vector<int4> rows(p->n_row);
    int n_bl = 0;
    for (int r = 0; r < p->n_row; ++r) {
        const int a1 = p->ant1[r], a2 = p->ant2[r];
        int bl = 0;
        if (a1 != a2) {
            int &slot = bl_of_pair[(size_t)a1 * na + a2];
            if (slot < 0) slot = n_bl++;
            bl = slot;
        }
        rows[r] = make_int4(a1, a2, p->time_idx[r], bl);
    }
    c->n_bl = n_bl;
    std::vector<int> strip_off(n_bl + 1, 0), strip_rows;
    for (int r = 0; r < p->n_row; ++r) if (rows[r].x != rows[r].y) strip_off[rows[r].w + 1]++;
    for (int b = 0; b < n_bl; ++b) strip_off[b + 1] += strip_off[b];
    strip_rows.resize(strip_off[n_bl]);
    {
        std::vector<int> fill(strip_off.begin(), strip_off.end() - 1);
        for (int r = 0; r < p->n_row; ++r) if (rows[r].x != rows[r].y) strip_rows[fill[rows[r].w]++] = r;
        for (int b = 0; b < n_bl; ++b)
            std::stable_sort(strip_rows.begin() + strip_off[b], strip_rows.begin() + strip_off[b + 1],
                             [&](int x, int y) { return rows[x].z < rows[y].z; });
    }
    c->n_strips = n_bl;
    c->n_strip_rows = (long)strip_rows.size();
    for (int b = 0; b < n_bl; ++b) c->max_strip_rows = std::max(c->max_strip_rows, strip_off[b + 1] - strip_off[b]);
    cudaError_t e;
    qc_ctx *cc = c.get();
    auto dalloc = [&](size_t bytes) -> void * { return cc->alloc(bytes, &e); };
#define DALLOC(dst, T, n)                                                                    \
    do {                                                                                     \
        dst = (T *)dalloc(nbytes<T>(n));                                                     \
        if (e != cudaSuccess) { g_create_error = "cudaMalloc failed"; return e == cudaErrorMemoryAllocation ? QC_ENOMEM : QC_ECUDA; } \
    } while (0)
#define HCOPY(dst, src, bytes)                                                               \
    do {                                                                                     \
        e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);                             \
        if (e != cudaSuccess) { g_create_error = std::string("H2D copy: ") + cudaGetErrorString(e); return QC_ECUDA; } \
    } while (0)
    DALLOC(c->d_rows, int4, std::max(1, p->n_row));
    if (p->n_row) HCOPY(c->d_rows, rows.data(), nbytes<int4>(p->n_row));
    DALLOC(c->d_strip_off, int, n_bl + 1);
    HCOPY(c->d_strip_off, strip_off.data(), nbytes<int>(n_bl + 1));
    DALLOC(c->d_strip_rows, int, std::max<size_t>(1, strip_rows.size()));
    if (!strip_rows.empty()) HCOPY(c->d_strip_rows, strip_rows.data(), nbytes<int>(strip_rows.size()));
    {
        // unordered antenna pairs: both orientations of a baseline share one slot of the sums
        // of a term solved from sums (qc_opts.moments)
        std::vector<int> upair((size_t)na * na, -1), up_of_bl(std::max(1, n_bl), 0);
        int n_up = 0;
        for (int a1 = 0; a1 < na; ++a1)
            for (int a2 = 0; a2 < na; ++a2) {
                const int bl = bl_of_pair[(size_t)a1 * na + a2];
                if (bl < 0) continue;
                const int lo = std::min(a1, a2), hi = std::max(a1, a2);
                int &slot = upair[(size_t)lo * na + hi];
                if (slot < 0) { slot = n_up++; upair[(size_t)hi * na + lo] = slot; }
                up_of_bl[bl] = slot;
            }
        c->n_up = n_up;
        DALLOC(c->d_upair, int, std::max<size_t>(1, upair.size()));
        if (!upair.empty()) HCOPY(c->d_upair, upair.data(), nbytes<int>(upair.size()));
        DALLOC(c->d_up_of_bl, int, up_of_bl.size());
        HCOPY(c->d_up_of_bl, up_of_bl.data(), nbytes<int>(up_of_bl.size()));
    }

    const size_t n_vis = (size_t)p->n_row * p->n_chan;
    const float4 *model32 = nullptr;
    if (p->memory == QC_MEM_DEVICE) {
        c->d_vis = (const float4 *)p->data;
        model32 = (const float4 *)p->model;
        c->d_weight = (const float4 *)p->weight;
        c->d_flag = p->flag;
    } else {
        float4 *v, *w;
        DALLOC(v, float4, 2 * n_vis);
        HCOPY(v, p->data, nbytes<float4>(2 * n_vis));
        DALLOC(w, float4, n_vis);
        HCOPY(w, p->weight, nbytes<float4>(n_vis));
        c->d_vis = v;
        c->d_weight = w;
        float4 *m;
        DALLOC(m, float4, 2 * n_vis * p->n_dir);
        HCOPY(m, p->model, nbytes<float4>(2 * n_vis * p->n_dir));
        model32 = m;
        if (p->flag) {
            uint8_t *f;
            DALLOC(f, uint8_t, n_vis);
            HCOPY(f, p->flag, n_vis);
            c->d_flag = f;
        }
    }
    if (c->m16) {
        unsigned *bits;
        uint4 *m16;
        DALLOC(bits, unsigned, std::max(1, n_bl));
        DALLOC(m16, uint4, n_vis);
        e = cudaMemsetAsync(bits, 0, nbytes<unsigned>(std::max(1, n_bl)), c->own_stream);
        if (e == cudaSuccess && n_vis) {
            bl_scale_kernel<<<grid_for((long)n_vis, 256, c->sm_count), 256, 0, c->own_stream>>>(
                model32, c->d_rows, p->n_row, p->n_chan, bits);
            fix_scale_kernel<<<(n_bl + 255) / 256 + 1, 256, 0, c->own_stream>>>(bits, n_bl);
            pack16_kernel<<<grid_for((long)n_vis, 256, c->sm_count), 256, 0, c->own_stream>>>(
                model32, c->d_rows, p->n_row, p->n_chan, (const float *)bits, m16);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->own_stream);
        if (e != cudaSuccess) { g_create_error = std::string("fp16 model packing: ") + cudaGetErrorString(e); return QC_ECUDA; }
        c->d_model16 = m16;
        c->d_bl_scale = (const float *)bits;
        if (p->memory == QC_MEM_HOST) c->release((void *)model32);
        model32 = nullptr;
    }
    c->d_model = model32;
    {
        // weights with flags and autocorrelations folded in (w = 0), read by the streaming
        // kernel instead of the flags; the owned host-mode copy is folded in place
        float4 *wf = nullptr;
        if (p->memory == QC_MEM_HOST) wf = const_cast<float4 *>(c->d_weight);
        else DALLOC(wf, float4, std::max<size_t>(1, n_vis));
        if (n_vis) {
            fold_flags_kernel<<<grid_for((long)n_vis, 256, c->sm_count), 256, 0, c->own_stream>>>(
                c->d_weight, c->d_flag, c->d_rows, p->n_row, p->n_chan, wf);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->own_stream);
            if (e != cudaSuccess) { g_create_error = std::string("weights: ") + cudaGetErrorString(e); return QC_ECUDA; }
        }
        c->d_wf = wf;
    }
    DALLOC(c->d_row_live, uint8_t, std::max(1, p->n_row));
    DALLOC(c->d_err, int, 1);
    e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->own_stream);
    if (e == cudaSuccess && p->n_row) {
        row_live_kernel<<<grid_for((long)p->n_row * 32, 256, c->sm_count), 256, 0, c->own_stream>>>(c->data_desc(),
                                                                                                     c->d_row_live);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->own_stream);
    if (e != cudaSuccess) { g_create_error = std::string("row flags: ") + cudaGetErrorString(e); return QC_ECUDA; }
#undef DALLOC
#undef HCOPY
    *out = c.release();
    return QC_OK;
}

extern "C" void qc_destroy(qc_ctx *c) { delete c; }

// lets the allocation-free entry point report through qc_last_error(NULL)
void qc_internal_set_error(const char *msg) { g_create_error = msg; }

extern "C" const char *qc_last_error(const qc_ctx *c)
{
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

extern "C" const char *qc_version(void) { return "qc-gb300 1.0 (sm_103a)"; }

// ---------------------------------------------------------------------------
// term staging
// ---------------------------------------------------------------------------

static size_t term_nbins(const qc_term &t) { return (size_t)t.n_tint * t.n_fint; }

int qc_ctx::validate_terms(const qc_term *terms, int n_terms, bool need_solve_fields)
{
    if (!terms) return fail(QC_EINVAL, "terms is NULL");
    if (n_terms < 1 || n_terms > QC_MAX_TERMS) return fail(QC_EINVAL, "n_terms must be in [1, QC_MAX_TERMS]");
    for (int j = 0; j < n_terms; ++j) {
        const qc_term &t = terms[j];
        if (t.type < 0 || t.type > 3) return fail(QC_EINVAL, "unknown term type");
        if (t.type == QC_TERM_DELAY) {
            if (!t.chan_freq) return fail(QC_EINVAL, "a delay term needs chan_freq");
            for (int i = 0; i < n_chan; ++i)
                if (!std::isfinite(t.chan_freq[i])) return fail(QC_EINVAL, "chan_freq must be finite");
            if ((long long)t.n_tint * n_chan * n_ant > (1LL << 31)) return fail(QC_EINVAL, "delay term too large");
        }
        if (t.n_tint < 1 || t.n_fint < 1) return fail(QC_EINVAL, "n_tint and n_fint must be >= 1");
        if ((long long)t.n_tint * t.n_fint * n_ant > (1LL << 31)) return fail(QC_EINVAL, "term too large");
        if (!t.t_map || !t.f_map || !t.gains) return fail(QC_EINVAL, "t_map, f_map and gains are required");
        if (t.memory != QC_MEM_HOST && t.memory != QC_MEM_DEVICE) return fail(QC_EINVAL, "term memory invalid");
        for (int i = 0; i < n_time; ++i)
            if (t.t_map[i] < 0 || t.t_map[i] >= t.n_tint) return fail(QC_EINVAL, "t_map value out of range");
        for (int i = 0; i < n_chan; ++i) {
            if (t.f_map[i] < 0 || t.f_map[i] >= t.n_fint) return fail(QC_EINVAL, "f_map value out of range");
            if (i && t.f_map[i] < t.f_map[i - 1]) return fail(QC_EINVAL, "f_map must be non-decreasing");
        }
        if (need_solve_fields && t.solve) {
            if (t.max_iter < 1) return fail(QC_EINVAL, "max_iter must be >= 1 for a solved term");
            if (!(t.tol >= 0)) return fail(QC_EINVAL, "tol must be >= 0");
        }
        if (n_dir > 1) {
            if (t.type == QC_TERM_PHASE)
                return fail(QC_EUNSUPPORTED, "chains with directions take diagonal, full and delay terms");
            if (t.type == QC_TERM_DELAY && t.dd)
                return fail(QC_EUNSUPPORTED, "a delay term is direction-independent");
            if (need_solve_fields && t.solve && !t.dd)
                for (int i = 0; i < j; ++i)
                    if (terms[i].dd)
                        return fail(QC_EUNSUPPORTED, "a solved direction-independent term must not have a "
                                                     "direction-dependent term to its left");
        }
    }
    return QC_OK;
}

// The kernels' view of the chain: a delay term becomes a diagonal term with one bin per
// (time interval, channel) and the identity channel map, its table evaluated at every
// channel from the interval's parameters (the channel ranges, maps and frequencies of its
// intervals are uploaded here).  Other terms are unchanged.
int qc_ctx::expand_terms(const qc_term *terms, int n_terms, std::vector<qc_term> &xt, cudaStream_t st)
{
    qc_ctx *c = this;
    xt.assign(terms, terms + n_terms);
    if ((int)fid.size() != n_chan) {
        fid.resize(n_chan);
        for (int i = 0; i < n_chan; ++i) fid[i] = i;
    }
    for (int j = 0; j < n_terms; ++j) {
        delay[j] = terms[j].type == QC_TERM_DELAY;
        if (!delay[j]) continue;
        const qc_term &t = terms[j];
        TermBufs &B = tb[j];
        B.hfr.assign(t.n_fint, make_int2(-1, -2));
        for (int ch = 0; ch < n_chan; ++ch) {
            int2 &r = B.hfr[t.f_map[ch]];
            if (r.x < 0) r.x = ch;
            r.y = ch;
        }
        int rc;
        if ((rc = ensure(B.dfmap, nbytes<int>(std::max(1, n_chan))))) return rc;
        if ((rc = ensure(B.dfr, nbytes<int2>(t.n_fint)))) return rc;
        if ((rc = ensure(B.dnu, nbytes<double>(std::max(1, n_chan))))) return rc;
        if ((rc = ensure(B.domega, nbytes<float>(std::max(1, n_chan))))) return rc;
        B.hufmap.assign(t.f_map, t.f_map + n_chan);
        double mean_nu = 0;
        for (int ch = 0; ch < n_chan; ++ch) mean_nu += t.chan_freq[ch];
        B.omega_ref = n_chan ? DELAY_TWO_PI * (mean_nu / n_chan) : 0.0;
        std::vector<float> om(n_chan);
        for (int ch = 0; ch < n_chan; ++ch) om[ch] = (float)(DELAY_TWO_PI * t.chan_freq[ch] - B.omega_ref);
        if (n_chan) {
            CK(cudaMemcpyAsync(B.dfmap.ptr, t.f_map, nbytes<int>(n_chan), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(B.dnu.ptr, t.chan_freq, nbytes<double>(n_chan), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(B.domega.ptr, om.data(), nbytes<float>(n_chan), cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));      // om is a local staging vector
        }
        CK(cudaMemcpyAsync(B.dfr.ptr, B.hfr.data(), nbytes<int2>(t.n_fint), cudaMemcpyHostToDevice, st));
        xt[j].type = QC_TERM_DIAG;
        xt[j].n_fint = n_chan;
        xt[j].f_map = fid.data();
    }
    return QC_OK;
}

DelayArgs qc_ctx::delay_args(int j, const qc_term &xt_j)
{
    TermBufs &B = tb[j];
    DelayArgs d;
    d.n_tint = xt_j.n_tint;
    d.n_fint = (int)B.hfr.size();
    d.n_ant = n_ant;
    d.n_chan = n_chan;
    d.fmap = (const int *)B.dfmap.ptr;
    d.frange = (const int2 *)B.dfr.ptr;
    d.nu = (const double *)B.dnu.ptr;
    d.params = (double *)B.params.ptr;
    d.tab = (float4 *)B.tab.ptr;
    d.omega_ref = B.omega_ref;
    return d;
}

// Upload maps and gains of every term; fills chain (device descriptors).
int qc_ctx::stage_terms(const qc_term *terms, int n_terms, cudaStream_t st, Chain &chain)
{
    qc_ctx *c = this;
    chain.n_terms = n_terms;
    chain.n = -1;
    chain.n_ant = n_ant;
    for (int j = 0; j < n_terms; ++j) {
        const qc_term &t = terms[j];
        TermBufs &B = tb[j];
        cur_nd[j] = term_nd(t);
        const size_t nb = term_nbins(t);
        const size_t nent = nb * term_nat(t);
        const size_t tab_f4 = nent * (t.type == 1 ? 2 : 1);
        int rc;
        if ((rc = ensure(B.maps, nbytes<int>(n_time + n_chan)))) return rc;
        if ((rc = ensure(B.tab, nbytes<float4>(tab_f4)))) return rc;
        if ((rc = ensure(B.params, nbytes<double>(nent * (t.type == 2 ? 2 : 8))))) return rc;
        if ((rc = ensure(B.stage, nent * (t.type == 2 ? 8 : 32)))) return rc;
        B.hmaps.assign(t.t_map, t.t_map + n_time);
        B.hmaps.insert(B.hmaps.end(), t.f_map, t.f_map + n_chan);
        CK(cudaMemcpyAsync(B.maps.ptr, B.hmaps.data(), nbytes<int>(n_time + n_chan), cudaMemcpyHostToDevice, st));
        if (delay[j]) {
            // parameters [n_tint][n_fint][n_ant][4] (float32) -> FP64 master; table per channel
            const DelayArgs da = delay_args(j, t);
            const size_t nvals = (size_t)da.n_tint * da.n_fint * n_ant * 4;
            const void *src = t.gains;
            if (t.memory == QC_MEM_HOST) {
                CK(cudaMemcpyAsync(B.stage.ptr, t.gains, nbytes<float>(nvals), cudaMemcpyHostToDevice, st));
                src = B.stage.ptr;
            }
            delay_params_in_kernel<<<grid_for((long)nvals, 256, sm_count), 256, 0, st>>>((long)nvals, (const float *)src,
                                                                                        da.params);
            CK(cudaGetLastError());
            delay_tab_kernel<<<grid_for((long)nent, 256, sm_count), 256, 0, st>>>(da);
            CK(cudaGetLastError());
            launches += 2;
        } else {
            const void *src = t.gains;
            if (t.memory == QC_MEM_HOST) {
                CK(cudaMemcpyAsync(B.stage.ptr, t.gains, nent * (t.type == 2 ? 8 : 32), cudaMemcpyHostToDevice, st));
                src = B.stage.ptr;
            }
            gains_in_kernel<<<grid_for((long)nent, 256, sm_count), 256, 0, st>>>(t.type, t.n_tint, t.n_fint, term_nat(t), src,
                                                                                (double *)B.params.ptr,
                                                                                (float4 *)B.tab.ptr);
            CK(cudaGetLastError());
            ++launches;
        }
        DevTerm &d = chain.t[j];
        d.type = t.type;
        d.n_tint = t.n_tint;
        d.n_fint = t.n_fint;
        d.t_map = (const int *)B.maps.ptr;
        d.f_map = (const int *)B.maps.ptr + n_time;
        d.tab = (const float4 *)B.tab.ptr;
    }
    return QC_OK;
}

Data qc_ctx::data_desc() const
{
    Data D;
    D.n_row = n_row;
    D.n_chan = n_chan;
    D.vis = d_vis;
    D.model = d_model;
    D.weight = d_weight_use ? d_weight_use : d_weight;
    D.model16 = d_model16;
    D.bl_scale = d_bl_scale;
    D.flag = d_flag;
    D.rows = d_rows;
    D.strip_rows = d_strip_rows;
    D.strip_off = d_strip_off;
    D.n_strips = n_strips;
    return D;
}

// ---------------------------------------------------------------------------
// residual / chi^2
// ---------------------------------------------------------------------------

extern "C" int qc_residual(qc_ctx *c, const qc_term *terms, int32_t n_terms, void *resid, int32_t resid_memory,
                           double *chi2)
{
    if (!c) return QC_EINVAL;
    c->err.clear();
    if (!chi2) return c->fail(QC_EINVAL, "chi2 is NULL");
    int rc = c->validate_terms(terms, n_terms, false);
    if (rc) return rc;
    cudaStream_t st = c->own_stream;
    std::vector<qc_term> xt;
    if ((rc = c->expand_terms(terms, n_terms, xt, st))) return rc;
    Chain chain;
    if ((rc = c->stage_terms(xt.data(), n_terms, st, chain))) return rc;
    if ((rc = c->ensure(c->scalars, 64))) return rc;
    double *d_chi2 = (double *)c->scalars.ptr;
    const size_t n_vis = (size_t)c->n_row * c->n_chan;
    float4 *dres = nullptr;
    if (resid) {
        if (resid_memory == QC_MEM_DEVICE) dres = (float4 *)resid;
        else {
            if ((rc = c->ensure(c->resid_stage, nbytes<float4>(2 * n_vis)))) return rc;
            dres = (float4 *)c->resid_stage.ptr;
        }
    }
    if ((rc = c->run_residual(chain, dres, d_chi2, st))) return rc;
    CK(cudaMemcpyAsync(chi2, d_chi2, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (resid && resid_memory != QC_MEM_DEVICE)
        CK(cudaMemcpyAsync(resid, dres, nbytes<float4>(2 * n_vis), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return QC_OK;
}

extern "C" int qc_delay_init(qc_ctx *c, qc_term *term, int32_t ref_ant, int32_t oversample)
{
    if (!c) return QC_EINVAL;
    c->err.clear();
    if (!term) return c->fail(QC_EINVAL, "term is NULL");
    if (term->type != QC_TERM_DELAY) return c->fail(QC_EINVAL, "qc_delay_init needs a QC_TERM_DELAY term");
    if (c->n_dir > 1) return c->fail(QC_EUNSUPPORTED, "qc_delay_init takes problems with one direction");
    int rc = c->validate_terms(term, 1, false);
    if (rc) return rc;
    if (ref_ant < 0 || ref_ant >= c->n_ant) return c->fail(QC_EINVAL, "ref_ant out of range");
    if (oversample < 0) return c->fail(QC_EINVAL, "oversample must be >= 0");
    if (oversample == 0) oversample = 4;
    const qc_term &t = *term;
    // per frequency interval: first channel, channels, transform length, spacing, first frequency
    std::vector<int4> info(t.n_fint, make_int4(0, 0, 1, 0));
    std::vector<double> dnu(t.n_fint, 0.0), nu0(t.n_fint, 0.0);
    int max_n = 1;
    for (int ch = 0; ch < c->n_chan; ++ch) {
        int4 &f = info[t.f_map[ch]];
        if (f.y == 0) f.x = ch;
        ++f.y;
    }
    for (int fi = 0; fi < t.n_fint; ++fi) {
        int4 &f = info[fi];
        if (f.y == 0) continue;
        nu0[fi] = t.chan_freq[f.x];
        if (f.y > 1) {
            const double d = (t.chan_freq[f.x + f.y - 1] - t.chan_freq[f.x]) / (f.y - 1);
            if (!(d != 0.0)) return c->fail(QC_EUNSUPPORTED, "an interval's channels have no frequency spread");
            for (int k = 0; k < f.y; ++k)
                if (std::fabs(t.chan_freq[f.x + k] - nu0[fi] - k * d) > 1e-6 * std::fabs(d))
                    return c->fail(QC_EUNSUPPORTED, "the delay estimate needs uniformly spaced channels");
            dnu[fi] = d;
        }
        long long N = 1;
        int lg = 0;
        while (N < (long long)oversample * f.y) { N *= 2; ++lg; }
        if (N > 16384) return c->fail(QC_EUNSUPPORTED, "transform longer than 16384 (reduce oversample)");
        f.z = (int)N;
        f.w = lg;
        max_n = std::max(max_n, (int)N);
    }
    cudaStream_t st = c->own_stream;
    // scratch of chain position 0: every qc_solve and qc_residual stages its buffers anew
    // (maps, accumulators, staging), and its graph is re-captured on every qc_solve
    TermBufs &B = c->tb[0];
    const size_t nx = (size_t)t.n_tint * c->n_ant * 2 * c->n_chan;
    const size_t npar = (size_t)t.n_tint * t.n_fint * c->n_ant * 4;
    if ((rc = c->ensure(B.maps, nbytes<int>(c->n_time + c->n_chan)))) return rc;
    if ((rc = c->ensure(B.acc, std::max(nbytes<float2>(nx), nbytes<float>(npar) + 64)))) return rc;
    if ((rc = c->ensure(B.stage, nbytes<float>(npar)))) return rc;
    if ((rc = c->ensure(B.dfr, nbytes<int4>(t.n_fint)))) return rc;
    if ((rc = c->ensure(B.dnu, nbytes<double>(2 * (size_t)t.n_fint)))) return rc;
    CK(cudaMemcpyAsync(B.maps.ptr, t.t_map, nbytes<int>(c->n_time), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.dfr.ptr, info.data(), nbytes<int4>(t.n_fint), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.dnu.ptr, dnu.data(), nbytes<double>(t.n_fint), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync((double *)B.dnu.ptr + t.n_fint, nu0.data(), nbytes<double>(t.n_fint), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(B.acc.ptr, 0, nbytes<float2>(nx), st));
    DelayInitArgs a;
    a.n_row = c->n_row;
    a.n_chan = c->n_chan;
    a.n_ant = c->n_ant;
    a.ref = ref_ant;
    a.n_tint = t.n_tint;
    a.n_fint = t.n_fint;
    a.rows = c->d_rows;
    a.vis = c->d_vis;
    a.model = c->m16 ? nullptr : c->d_model;
    a.model16 = c->d_model16;
    a.bl_scale = c->d_bl_scale;
    a.wf = c->d_wf;
    a.t_map = (const int *)B.maps.ptr;
    a.x = (float2 *)B.acc.ptr;
    a.fint_info = (const int4 *)B.dfr.ptr;
    a.fint_dnu = (const double *)B.dnu.ptr;
    a.fint_nu0 = (const double *)B.dnu.ptr + t.n_fint;
    float *dpar = t.memory == QC_MEM_DEVICE ? (float *)t.gains : (float *)B.stage.ptr;
    a.params = dpar;
    if (c->n_row) {
        delay_gather_kernel<<<grid_for((long)c->n_row * 32, 256, c->sm_count), 256, 0, st>>>(a);
        CK(cudaGetLastError());
    }
    const int smem = max_n * (int)sizeof(float2);
    if (smem > 48 * 1024) {
        if (smem > c->smem_optin) return c->fail(QC_EUNSUPPORTED, "transform does not fit in shared memory");
        CK(cudaFuncSetAttribute((const void *)delay_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    }
    const long blocks = (long)t.n_tint * t.n_fint * c->n_ant * 2;
    if (blocks > 0) {
        delay_peak_kernel<<<(unsigned)blocks, 256, smem, st>>>(a);
        CK(cudaGetLastError());
    }
    if (t.memory == QC_MEM_HOST)
        CK(cudaMemcpyAsync(t.gains, dpar, nbytes<float>(npar), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return QC_OK;
}

int qc_ctx::run_residual(const Chain &chain, float4 *dres, double *d_chi2, cudaStream_t st)
{
    qc_ctx *c = this;
    CK(cudaMemsetAsync(d_chi2, 0, sizeof(double), st));
    if (n_dir > 1) {
        DDArgs da;
        memset(&da, 0, sizeof da);
        da.D = data_desc();
        da.wf = d_wf;
        da.row_live = d_row_live;
        da.n_dir = n_dir;
        da.C = chain;
        da.C.n = -1;
        for (int j = 0; j < chain.n_terms; ++j) da.nd[j] = cur_nd[j];
        da.resid = dres;
        da.chi2 = d_chi2;
        CK(dd_launch_residual(da, grid_for((long)n_row * n_chan, 256, sm_count), st));
        ++launches;
        return QC_OK;
    }
    ResArgs ra;
    ra.D = data_desc();
    ra.C = chain;
    ra.resid = dres;
    ra.chi2 = d_chi2;
    const long warps = (long)n_row * ((n_chan + 31) / 32);
    const int grid = grid_for(warps * 32, 256, sm_count);
    if (m16) residual_kernel<true><<<grid, 256, 0, st>>>(ra);
    else residual_kernel<false><<<grid, 256, 0, st>>>(ra);
    CK(cudaGetLastError());
    ++launches;
    return QC_OK;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------

static int kind_of_range(const qc_term *terms, int lo, int hi)
{
    int k = KIND_NONE;
    for (int j = lo; j < hi; ++j) k = std::max(k, terms[j].type == 1 ? KIND_FULL : KIND_DIAG);
    return k;
}

int qc_ctx::pick_order(const qc_term &t, const qc_opts *o) const
{
    if (o && (o->order == 0 || o->order == 1)) return o->order;
    // mean interval extent along channels and along time (rows of one baseline)
    const double wf = (double)n_chan / t.n_fint;
    const double ht = (double)n_time / t.n_tint;
    return (wf >= 32.0 || wf >= ht) ? 0 : 1;
}

extern "C" int qc_solve(qc_ctx *c, qc_term *terms, int32_t n_terms, const qc_opts *o, qc_stats *stats)
{
    if (!c) return QC_EINVAL;
    c->err.clear();
    int rc = c->validate_terms(terms, n_terms, true);
    if (rc) return rc;
    qc_opts defaults;
    memset(&defaults, 0, sizeof defaults);
    defaults.n_epochs = 1;
    defaults.damping_mode = QC_DAMP_ALTERNATE;
    defaults.use_graph = 1;
    defaults.order = -1;
    if (!o) o = &defaults;
    if (o->n_epochs < 1) return c->fail(QC_EINVAL, "n_epochs must be >= 1");
    if (o->damping_mode != QC_DAMP_CONST && o->damping_mode != QC_DAMP_ALTERNATE)
        return c->fail(QC_EINVAL, "unknown damping_mode");
    for (int j = 0; j < n_terms; ++j)
        if (terms[j].solve && terms[j].reduce && !o->allreduce)
            return c->fail(QC_EINVAL, "a term with reduce = 1 needs opts.allreduce");
    cudaStream_t st = o->stream ? (cudaStream_t)o->stream : c->own_stream;
    c->launches = 0;
    qc_stats S;
    memset(&S, 0, sizeof S);

    cudaEvent_t ev0, ev1;
    if ((rc = c->get_event(0, ev0)) || (rc = c->get_event(1, ev1))) return rc;
    CK(cudaEventRecord(ev0, st));
    std::vector<qc_term> xt;     // the kernels' view of the terms (delay terms per channel)
    if ((rc = c->expand_terms(terms, n_terms, xt, st))) return rc;
    Chain chain;
    if ((rc = c->stage_terms(xt.data(), n_terms, st, chain))) return rc;
    if ((rc = c->ensure(c->scalars, 64))) return rc;
    unsigned long long *d_counters = (unsigned long long *)c->scalars.ptr;   // [0] vis_iters, [1] bytes
    double *d_chi2 = (double *)c->scalars.ptr + 4;
    CK(cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned long long), st));
    if (o->want_chi2) {
        if ((rc = c->run_residual(chain, nullptr, d_chi2, st))) return rc;
        CK(cudaMemcpyAsync(&S.chi2_before, d_chi2, sizeof(double), cudaMemcpyDeviceToHost, st));
    }

    // per solved term: bin counts and byte weights
    const long long b_flag = c->has_flag ? 1 : 0;
    const long long b_unflag = 32 + (c->m16 ? 16 : 32 * c->n_dir) + 16;
    for (int j = 0; j < n_terms; ++j) {
        if (!terms[j].solve) continue;
        const qc_term &t = xt[j];
        TermBufs &B = c->tb[j];
        const size_t nb = term_nbins(t);
        const size_t KG = t.type == 1 ? KG_FULL : KG_DIAG;
        const size_t nat = c->term_nat(t);
        if ((rc = c->ensure(B.acc, nbytes<double>(nb * nat * KG)))) return rc;
        if ((rc = c->ensure(B.active, nb))) return rc;
        if ((rc = c->ensure(B.cnt, nbytes<int>(t.max_iter + 1)))) return rc;
        if ((rc = c->ensure(B.nvis, nbytes<long long>(3 * nb)))) return rc;
        if ((rc = c->ensure(B.iters, nbytes<int>(nb)))) return rc;
        if ((rc = c->ensure(B.flags, nb * nat))) return rc;
        CK(cudaMemsetAsync(B.acc.ptr, 0, nbytes<double>(nb * nat * KG), st));
        CK(cudaMemsetAsync(B.iters.ptr, 0, nbytes<int>(nb), st));
        CK(cudaMemsetAsync(B.flags.ptr, 0, nb * nat, st));
        // the counts of the previous call stand while the term's maps are the same (FNV-1a
        // over the kernels' view of them)
        uint64_t sig = 1469598103934665603ull;
        auto mix = [&](uint64_t v) { sig = (sig ^ v) * 1099511628211ull; };
        mix((uint64_t)t.type);
        mix((uint64_t)t.n_tint);
        mix((uint64_t)t.n_fint);
        mix((uint64_t)nat);
        for (int i = 0; i < c->n_time; ++i) mix((uint64_t)(uint32_t)t.t_map[i]);
        for (int i = 0; i < c->n_chan; ++i) mix((uint64_t)(uint32_t)t.f_map[i]);
        B.graph_valid = false;
        if (sig == B.count_sig && B.count_buf == B.nvis.ptr) continue;
        B.count_sig = 0;
        CK(cudaMemsetAsync(B.nvis.ptr, 0, nbytes<long long>(3 * nb), st));
        long long *nvis = (long long *)B.nvis.ptr;
        CountArgs ca;
        ca.D = c->data_desc();
        ca.t_map = chain.t[j].t_map;
        ca.f_map = chain.t[j].f_map;
        ca.n_fint = t.n_fint;
        ca.nvis = nvis;
        ca.nunflag = nvis + nb;
        if (c->n_row) {
            count_kernel<<<grid_for((long)c->n_row * 32, 256, c->sm_count), 256, 0, st>>>(ca);
            CK(cudaGetLastError());
            ++c->launches;
        }
        bin_bytes_kernel<<<((int)nb + 255) / 256, 256, 0, st>>>((int)nb, nvis, nvis + nb, b_flag, b_unflag, nvis + 2 * nb);
        CK(cudaGetLastError());
        ++c->launches;
        B.count_sig = sig;
        B.count_buf = B.nvis.ptr;
    }

    // robust reweighting between epochs: every kernel reads the context's folded weight copy,
    // reweighted in place; the weights before reweighting are kept and put back on return
    const bool robust = o->robust && o->n_epochs > 1;
    const double nu = o->robust_nu > 0 ? o->robust_nu : 5.0;
    const size_t n_vis = (size_t)c->n_row * c->n_chan;
    struct RobustGuard {
        qc_ctx *c = nullptr;
        cudaStream_t st = nullptr;
        size_t bytes = 0;
        ~RobustGuard()
        {
            if (!c) return;
            cudaMemcpyAsync(const_cast<float4 *>(c->d_wf), c->rob_w0.ptr, bytes, cudaMemcpyDeviceToDevice, st);
            c->d_weight_use = nullptr;
        }
    } guard;
    if (robust && n_vis) {
        if (!std::isfinite(nu)) return c->fail(QC_EINVAL, "robust_nu must be finite");
        if ((rc = c->ensure(c->rob_w0, nbytes<float4>(n_vis)))) return rc;
        if ((rc = c->ensure(c->rob_lam, nbytes<float>(n_vis)))) return rc;
        if ((rc = c->ensure(c->rob_res, nbytes<float4>(2 * n_vis)))) return rc;
        if ((rc = c->ensure(c->rob_sums, nbytes<double>(4)))) return rc;
        CK(cudaMemcpyAsync(c->rob_w0.ptr, c->d_wf, nbytes<float4>(n_vis), cudaMemcpyDeviceToDevice, st));
        robust_fill_kernel<<<grid_for((long)n_vis, 256, c->sm_count), 256, 0, st>>>((long)n_vis, (float *)c->rob_lam.ptr,
                                                                                     1.f);
        CK(cudaGetLastError());
        guard.c = c;
        guard.st = st;
        guard.bytes = nbytes<float4>(n_vis);
        c->d_weight_use = c->d_wf;
    }
    int n_iter_max = 0;
    for (int epoch = 0; epoch < o->n_epochs; ++epoch) {
        for (int n = 0; n < n_terms; ++n) {
            if (!terms[n].solve) continue;
            int it_max = 0;
            double acc_ms = 0, pass_ms = 0;
            long long acc_launches = 0;
            if ((rc = c->solve_term(xt.data(), n_terms, n, chain, o, st, &it_max, &acc_ms, &acc_launches, &pass_ms)))
                return rc;
            S.acc_ms += acc_ms;
            S.pass_ms += pass_ms;
            S.acc_launches += acc_launches;
            if (epoch == o->n_epochs - 1) n_iter_max = std::max(n_iter_max, it_max);
        }
        if (guard.c && epoch < o->n_epochs - 1) {
            // one EM step on the residual of the current chain (whitened by the original weights)
            double *sums = (double *)c->rob_sums.ptr;
            if ((rc = c->run_residual(chain, (float4 *)c->rob_res.ptr, sums + 2, st))) return rc;
            CK(cudaMemsetAsync(sums, 0, 2 * sizeof(double), st));
            const int g = grid_for((long)n_vis, 256, c->sm_count);
            robust_sum_kernel<<<g, 256, 0, st>>>((long)n_vis, (const float4 *)c->rob_res.ptr,
                                                 (const float4 *)c->rob_w0.ptr, (const float *)c->rob_lam.ptr, sums);
            robust_apply_kernel<<<g, 256, 0, st>>>((long)n_vis, (const float4 *)c->rob_res.ptr,
                                                   (const float4 *)c->rob_w0.ptr, (float *)c->rob_lam.ptr,
                                                   const_cast<float4 *>(c->d_wf), sums, nu);
            CK(cudaGetLastError());
            c->launches += 3;
        }
    }
    if (guard.c) {
        // the caller's weights again for chi2_after and for later calls
        CK(cudaMemcpyAsync(const_cast<float4 *>(c->d_wf), c->rob_w0.ptr, nbytes<float4>(n_vis),
                           cudaMemcpyDeviceToDevice, st));
        c->d_weight_use = nullptr;
        guard.c = nullptr;
    }
    if (o->want_chi2) {
        if ((rc = c->run_residual(chain, nullptr, d_chi2, st))) return rc;
        CK(cudaMemcpyAsync(&S.chi2_after, d_chi2, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    // write back solved gains, flags, iteration counts
    for (int j = 0; j < n_terms; ++j) {
        if (!terms[j].solve) continue;
        qc_term &t = terms[j];
        TermBufs &B = c->tb[j];
        const size_t nb = term_nbins(t), nent = nb * c->term_nat(t);
        const size_t gbytes = nent * (t.type == 2 ? 8 : (t.type == QC_TERM_DELAY ? 16 : 32));
        void *dst = t.memory == QC_MEM_DEVICE ? t.gains : B.stage.ptr;
        if (t.type == QC_TERM_DELAY)
            delay_params_out_kernel<<<grid_for((long)nent * 4, 256, c->sm_count), 256, 0, st>>>(
                (long)nent * 4, (const double *)B.params.ptr, (float *)dst);
        else
            gains_out_kernel<<<grid_for((long)nent, 256, c->sm_count), 256, 0, st>>>(t.type, (long)nent,
                                                                                   (const double *)B.params.ptr, dst);
        CK(cudaGetLastError());
        ++c->launches;
        if (t.memory == QC_MEM_HOST) {
            CK(cudaMemcpyAsync(t.gains, B.stage.ptr, gbytes, cudaMemcpyDeviceToHost, st));
            if (t.gain_flags) CK(cudaMemcpyAsync(t.gain_flags, B.flags.ptr, nent, cudaMemcpyDeviceToHost, st));
            if (t.iters) CK(cudaMemcpyAsync(t.iters, B.iters.ptr, nbytes<int>(nb), cudaMemcpyDeviceToHost, st));
        } else {
            if (t.gain_flags) CK(cudaMemcpyAsync(t.gain_flags, B.flags.ptr, nent, cudaMemcpyDeviceToDevice, st));
            if (t.iters) CK(cudaMemcpyAsync(t.iters, B.iters.ptr, nbytes<int>(nb), cudaMemcpyDeviceToDevice, st));
        }
    }
    unsigned long long hc[2];
    CK(cudaMemcpyAsync(hc, d_counters, sizeof hc, cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(ev1, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ev0, ev1));
    S.ms = ms;
    S.vis_iters = (int64_t)hc[0];
    S.acc_bytes = (int64_t)hc[1];
    S.n_iter_max = n_iter_max;
    S.launches = c->launches;
    if (stats) *stats = S;
    return QC_OK;
}

bool qc_ctx::configured(const void *fn) const
{
    return std::find(configured_fns.begin(), configured_fns.end(), fn) != configured_fns.end();
}

int qc_ctx::get_event(int i, cudaEvent_t &ev)
{
    while ((int)events.size() <= i) {
        cudaEvent_t e;
        cudaError_t err_ = cudaEventCreate(&e);
        if (err_ != cudaSuccess) return cuda_fail(err_, "cudaEventCreate");
        events.push_back(e);
    }
    ev = events[i];
    return QC_OK;
}

int qc_ctx::solve_term(const qc_term *terms, int n_terms, int n, Chain chain, const qc_opts *o, cudaStream_t st,
                       int *it_max, double *acc_ms, long long *acc_launches, double *pass_ms)
{
    *pass_ms = 0;
    qc_ctx *c = this;
    const qc_term &t = terms[n];
    TermBufs &B = tb[n];
    const int nb = (int)term_nbins(t);
    chain.n = n;
    const int ts = t.type == 1 ? TS_FULL : TS_DIAG;
    const int lk = kind_of_range(terms, 0, n);
    const int rk = kind_of_range(terms, n + 1, n_terms);
    // chains with directions: chains of one or two terms with at most DDS_MAX_DIR directions
    // take the streaming direction-dependent kernel (row tiles, qc_dd_stream.cuh), longer
    // chains the general one (qc_dd.cu)
    const bool ddp = n_dir > 1;
    DDSLaunch DS;
    if (ddp && n_terms <= 2 && n_dir <= DDS_MAX_DIR && (o->kernel == 0 || o->kernel == 3) &&
        (long long)n_ant * n_dir < 32768) {
        const int ok_ = n_terms == 2 ? (terms[1 - n].type == 1 ? KIND_FULL : KIND_DIAG) : KIND_NONE;
        DS = dds_launcher(t.type == 1 ? KIND_FULL : KIND_DIAG, ok_, n == 1, delay[n], cur_nd[n] > 1);
    }
    const bool dds = DS.fn != nullptr;
    const int order = dds ? 0 : pick_order(t, o);
    // the prefetching and streaming kernels are compiled for at most 256 threads per CTA
    // (the streaming kernel for two such CTAs per SM)
    const bool bt_ok = o->block_threads >= 32 && o->block_threads % 32 == 0;
    int block = (bt_ok && o->block_threads <= 256) ? o->block_threads : 256;
    const int block_stream = block;
    AccArgs aa;
    aa.D = data_desc();
    aa.C = chain;
    aa.tn = chain.t[n];
    aa.row_live = d_row_live;
    aa.to = n_terms == 2 ? chain.t[1 - n] : chain.t[n];
    aa.acc = (double *)B.acc.ptr;
    aa.active = (const uint8_t *)B.active.ptr;
    aa.order = order;
    aa.n_chunks = (n_chan + 31) / 32;
    const long units = order == 0 ? (long)n_row : (long)n_strips * aa.n_chunks;
    int per_sm = o->ctas_per_sm > 0 ? o->ctas_per_sm : 0;
    const bool simple = n_terms <= 2;
    AccLaunch L = acc_launcher(ts, simple, lk, rk, m16);
    const int nat = term_nat(t);
    if (!L.fn && !ddp) return fail(QC_EUNSUPPORTED, "no accumulate kernel for this chain");
    // the term from per-(interval, pair) sums (qc_moments.cu): one pass over the data, then
    // every iteration forms the blocks from the sums and the current gains.  No term to the
    // left: the full form, the term to the right folded into the model; a diagonal or phase-only
    // term with a term to its left: the diagonal form
    int mom_form = -1, mom_ok = KIND_NONE;
    if (o->moments && n_terms <= 2 && !delay[n] && !ddp && d_model != nullptr && n_up > 0 &&
        (size_t)nb * n_up < (size_t)INT32_MAX) {
        if (lk == KIND_NONE) { mom_form = FORM_FULL; mom_ok = rk; }
        else if (t.type != QC_TERM_FULL) { mom_form = FORM_E; mom_ok = lk; }
    }
    const bool mom = mom_form >= 0;
    // pipelined kernel: shared-memory layout of the per-warp rings for this chain
    PipeArgs pa;
    memset(&pa, 0, sizeof pa);
    int pipe_smem = 0;
    // auto and kernel 3: the streaming kernel (chains of one or two terms; antenna pairs are
    // packed as p | q << 16); kernels 1 and 2 on request, and for longer chains
    // kernel 4: the warp-specialised kernel (chains of one or two terms; a solved delay term
    // keeps its own streaming kernel)
    // kernel 5: the self-feeding variant (every warp issues its own bulk copies)
    bool ws = !mom && !ddp && L.ws_fn != nullptr && !delay[n] && n_ant < 32768 && (o->kernel == 4 || o->kernel == 5);
    const bool self_feed = o->kernel == 5;
    const void *ws_fn = self_feed ? (order == 0 ? L.wss_fn : L.wss_fn1) : L.ws_fn;
    const int ws_warps = self_feed ? L.wss_nw : L.ws_nc;     // warps that own a ring
    const bool streaming = !mom && !ddp && L.stream_fn != nullptr && n_ant < 32768 &&
                           (o->kernel == 3 || o->kernel == 0 || ((o->kernel == 4 || o->kernel == 5) && delay[n]));
    // a solved delay term under the streaming kernel: its own kernel, which applies the chain
    // rule per sample and keeps sums per parameter interval (else: the per-channel bins)
    DelayLaunch DL;
    if (delay[n] && streaming) DL = delay_launcher(lk, rk, m16);
    const bool ded = DL.fn != nullptr;
    // a solved delay term with sums per parameter interval (the streaming kernels), else
    // the per-channel bins
    const bool psums = ded || (dds && delay[n]);
    DevTerm tnu = chain.t[n];
    const int nbu = delay[n] ? t.n_tint * (int)B.hfr.size() : nb;
    if (psums) {
        tnu.n_fint = (int)B.hfr.size();
        tnu.f_map = (const int *)B.dfmap.ptr;
        aa.tn = tnu;
        int rc_;
        if ((rc_ = ensure(B.acc, nbytes<double>((size_t)nbu * n_ant * KG_SUMS)))) return rc_;
        CK(cudaMemsetAsync(B.acc.ptr, 0, nbytes<double>((size_t)nbu * n_ant * KG_SUMS), st));
        aa.acc = (double *)B.acc.ptr;
    }
    const void *stream_fn = dds ? DS.fn : (ded ? DL.fn : L.stream_fn);
    const int stream_smem_per_warp = dds ? dds_smem_per_warp(n_dir) : (ded ? DL.smem_per_warp : L.stream_smem_per_warp);
    bool pipelined = !mom && !ddp && !streaming && L.pipe_fn != nullptr && (o->kernel == 1 || (o->kernel == 0 && order == 1));
    const bool has_o = n_terms == 2;
    if (pipelined) {
        const int NW = L.pipe_nw;
        const int n_chunks = (n_chan + 31) / 32;
        std::vector<int4> ci(n_chunks);
        int capn = 1, capo = has_o ? 1 : 0;
        for (int ch = 0; ch < n_chunks; ++ch) {
            const int c0 = ch * 32, c1 = std::min(n_chan, c0 + 32) - 1;
            ci[ch].x = t.f_map[c0];
            ci[ch].y = t.f_map[c1] - t.f_map[c0] + 1;
            ci[ch].z = has_o ? terms[1 - n].f_map[c0] : 0;
            ci[ch].w = has_o ? terms[1 - n].f_map[c1] - terms[1 - n].f_map[c0] + 1 : 0;
            capn = std::max(capn, ci[ch].y);
            capo = std::max(capo, ci[ch].w);
        }
        const int esn = t.type == 1 ? 32 : 16;
        const int eso = has_o ? (terms[1 - n].type == 1 ? 32 : 16) : 16;
        pa.jn_cap = capn;
        pa.jo_cap = capo;
        const int mb = m16 ? 16 : 32;
        pa.off_m = 32 * 32;
        pa.off_w = pa.off_m + 32 * mb;
        pa.off_jn = pa.off_w + 32 * 16;
        pa.off_jo = pa.off_jn + 2 * pa.jn_cap * esn;
        pa.slot_bytes = pa.off_jo + 2 * pa.jo_cap * eso;
        pa.stage_fmap = n_chan <= 8192 ? 1 : 0;
        const int fmap_bytes = pa.stage_fmap ? ((2 * n_chan * 4 + 15) / 16) * 16 : 0;
        const int H = L.pipe_h;
        const int per_stage = H * (pa.slot_bytes + (int)sizeof(SlotDesc)) + 8;
        const int warp_budget = (smem_optin - fmap_bytes - 128) / NW;
        const int ns = std::min(8, warp_budget / per_stage);
        if (ns < 2) pipelined = false;
        else {
            pa.ns = ns;
            pa.desc_off = ns * H * pa.slot_bytes;
            pa.bar_off = pa.desc_off + ns * H * (int)sizeof(SlotDesc);
            pa.warp_bytes = ((pa.bar_off + ns * 8 + 15) / 16) * 16;
            pa.fmap_off = NW * pa.warp_bytes;
            pipe_smem = pa.fmap_off + fmap_bytes;
            if (!configured(L.pipe_fn)) {
                CK(cudaFuncSetAttribute(L.pipe_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin));
                configured_fns.push_back(L.pipe_fn);
            }
        }
    }
    int ws_cap = 1;            // warp-specialised kernel: other-term entries per 32-channel chunk (max)
    {
        // static per-row and per-chunk information of this term solve (both kernels)
        const int n_chunks = (n_chan + 31) / 32;
        std::vector<int4> ci(n_chunks);
        for (int ch = 0; ch < n_chunks; ++ch) {
            const int c0 = ch * 32, c1 = std::min(n_chan, c0 + 32) - 1;
            ci[ch].x = t.f_map[c0];
            ci[ch].y = t.f_map[c1] - t.f_map[c0] + 1;
            ci[ch].z = has_o ? terms[1 - n].f_map[c0] : 0;
            ci[ch].w = has_o ? terms[1 - n].f_map[c1] - terms[1 - n].f_map[c0] + 1 : 0;
            ws_cap = std::max(ws_cap, ci[ch].w);
        }
        int rc_;
        if ((rc_ = ensure(B.row_info, nbytes<int4>(std::max(1, n_row))))) return rc_;
        if ((rc_ = ensure(B.chunk_info, nbytes<int4>(n_chunks)))) return rc_;
        CK(cudaMemcpyAsync(B.chunk_info.ptr, ci.data(), nbytes<int4>(n_chunks), cudaMemcpyHostToDevice, st));
        if (n_row) {
            row_info_kernel<<<(n_row + 255) / 256, 256, 0, st>>>(data_desc(), d_row_live, chain.t[n],
                                                                has_o ? chain.t[1 - n] : chain.t[n], has_o ? 1 : 0,
                                                                (int4 *)B.row_info.ptr);
            CK(cudaGetLastError());
            ++launches;
        }
        pa.row_info = (const int4 *)B.row_info.ptr;
        pa.chunk_info = (const int4 *)B.chunk_info.ptr;
        aa.row_info = pa.row_info;
    }
    // warp-specialised kernel: shared-memory layout of one consumer's ring stage (d, m, folded
    // weights, the 32 channel maps, the other term's entries for p and q, a 32-byte header)
    // and the ring depth that two CTAs per SM leave room for
    WsArgs wa;
    memset(&wa, 0, sizeof wa);
    int ws_smem = 0, ws_grid = 0;
    if (ws) {
        const int ok_ = lk != KIND_NONE ? lk : rk;
        const int eso = ok_ == KIND_FULL ? 32 : 16;
        const int jo = has_o ? ((ws_cap * eso + 15) / 16) * 16 : 0;
        wa.off_m = 1024;
        wa.off_w = wa.off_m + 32 * (m16 ? 16 : 32);
        wa.off_fm = wa.off_w + 512;
        wa.off_jp = wa.off_fm + 256;
        wa.off_jq = wa.off_jp + jo;
        wa.off_h = wa.off_jq + jo;
        wa.stage_bytes = ((wa.off_h + 32 + 127) / 128) * 128;
        const int NC = ws_warps;
        const int nbar = self_feed ? 1 : 2;        // barriers per stage: full (and empty)
        const int budget = std::min(smem_optin, smem_per_sm / 2 - 1024) - 2560;
        wa.depth = std::min(6, budget / (NC * (wa.stage_bytes + 8 * nbar)));
        if (wa.depth < 2) ws = false;
        else ws_smem = NC * wa.depth * wa.stage_bytes + nbar * NC * wa.depth * 8;
    }
    StreamArgs sa;
    memset(&sa, 0, sizeof sa);
    int stream_smem = 0;
    const long n_rt = order == 0 ? (long)n_row : n_strip_rows;
    if (streaming || ws || dds) {
        // step-major row table in the tile order, and the channel maps of both terms (padded
        // to whole 32-channel chunks: the warp-specialised kernel copies them 32 at a time)
        const int n_chunks = (n_chan + 31) / 32;
        int rc_;
        if ((rc_ = ensure(B.rt, nbytes<int4>(std::max(1L, n_rt))))) return rc_;
        if (m16 && (rc_ = ensure(B.rt_scale, nbytes<float>(std::max(1L, n_rt))))) return rc_;
        if ((rc_ = ensure(B.fmap2, nbytes<int2>(32 * n_chunks)))) return rc_;
        std::vector<int2> fm(32 * n_chunks, make_int2(0, 0));
        for (int ch = 0; ch < n_chan; ++ch)
            fm[ch] = make_int2(psums ? B.hufmap[ch] : t.f_map[ch], has_o ? terms[1 - n].f_map[ch] : 0);
        CK(cudaMemcpyAsync(B.fmap2.ptr, fm.data(), nbytes<int2>(32 * n_chunks), cudaMemcpyHostToDevice, st));
        if (n_rt) {
            row_table_kernel<<<(int)((n_rt + 255) / 256), 256, 0, st>>>(
                (int)n_rt, order == 0 ? nullptr : d_strip_rows, (const int4 *)B.row_info.ptr, d_rows,
                m16 ? d_bl_scale : nullptr, (int4 *)B.rt.ptr, m16 ? (float *)B.rt_scale.ptr : nullptr);
            CK(cudaGetLastError());
            ++launches;
        }
    }
    if (ws) {
        const int n_chunks = (n_chan + 31) / 32;
        int rc_;
        wa.vis = d_vis;
        wa.model = d_model;
        wa.model16 = d_model16;
        wa.wf = d_wf;
        wa.n_chan = n_chan;
        wa.n_ant = n_ant;
        wa.order = order;
        wa.n_chunks = n_chunks;
        wa.nwr = (n_chunks + 31) / 32;
        wa.nwk = (int)((n_strip_rows + 31) / 32);
        if (order == 0) {
            if ((rc_ = ensure(B.ws_rl, nbytes<int4>(std::max(1, n_row))))) return rc_;
            if (m16 && (rc_ = ensure(B.ws_rls, nbytes<float>(std::max(1, n_row))))) return rc_;
            if ((rc_ = ensure(B.ws_rlb, nbytes<unsigned>((size_t)std::max(1, n_row) * wa.nwr)))) return rc_;
            if ((rc_ = ensure(B.ws_n, sizeof(int)))) return rc_;
            wa.rl = (const int4 *)B.ws_rl.ptr;
            wa.rl_scale = m16 ? (const float *)B.ws_rls.ptr : nullptr;
            wa.rl_bits = (const unsigned *)B.ws_rlb.ptr;
            wa.n_rl = (const int *)B.ws_n.ptr;
        } else {
            if ((rc_ = ensure(B.ws_sb, nbytes<unsigned>((size_t)n_chunks * std::max(1, wa.nwk))))) return rc_;
            if ((rc_ = ensure(B.units, sizeof(int)))) return rc_;
            wa.sbits = (const unsigned *)B.ws_sb.ptr;
            wa.unit_counter = (int *)B.units.ptr;
        }
        wa.rt = (const int4 *)B.rt.ptr;
        wa.rt_scale = m16 ? (const float *)B.rt_scale.ptr : nullptr;
        wa.unit_off = d_strip_off;
        wa.n_strips = n_strips;
        wa.tn = chain.t[n];
        wa.to = has_o ? chain.t[1 - n] : chain.t[n];
        wa.fmap2 = (const int2 *)B.fmap2.ptr;
        wa.chunk_info = (const int4 *)B.chunk_info.ptr;
        wa.active = (const uint8_t *)B.active.ptr;
        wa.acc = (double *)B.acc.ptr;
        wa.err = d_err;
        wa.wait_ns = qc_wait_limit_ns();
        wa.stall_fill = qc_wait_stall_stage();
        if (!configured(ws_fn)) {
            // the kernel's static shared memory (chunk table, abort flag) counts against the limit too
            cudaFuncAttributes fa;
            CK(cudaFuncGetAttributes(&fa, ws_fn));
            CK(cudaFuncSetAttribute(ws_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem_optin - (int)fa.sharedSizeBytes));
            configured_fns.push_back(ws_fn);
        }
        int occ = 0;
        const int ws_block = self_feed ? ws_warps * 32 : (ws_warps + 1) * 32;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ws_fn, ws_block, ws_smem);
        if (e != cudaSuccess || occ < 1) return fail(QC_EUNSUPPORTED, "warp-specialised kernel does not fit on an SM");
        per_sm = per_sm > 0 ? std::min(per_sm, occ) : occ;
        ws_grid = sm_count * per_sm;
    }
    if (streaming || dds) {
        int rc_;
        block = block_stream;
        sa.vis = d_vis;
        sa.model = d_model;
        sa.model16 = d_model16;
        sa.wf = d_wf;
        sa.n_chan = n_chan;
        sa.n_ant = n_ant;
        sa.rt = (const int4 *)B.rt.ptr;
        sa.rt_scale = m16 ? (const float *)B.rt_scale.ptr : nullptr;
        sa.unit_off = d_strip_off;
        sa.order = order;
        sa.n_chunks = (n_chan + 31) / 32;
        sa.n_units = order == 0 ? n_row : n_strips * sa.n_chunks;
        sa.tn = psums ? tnu : chain.t[n];
        sa.to = has_o ? chain.t[1 - n] : chain.t[n];
        sa.fmap2 = (const int2 *)B.fmap2.ptr;
        sa.acc = (double *)B.acc.ptr;
        sa.active = (const uint8_t *)B.active.ptr;
        if (order == 1) {
            if ((rc_ = ensure(B.units, sizeof(int)))) return rc_;
            sa.unit_counter = (int *)B.units.ptr;
        }
        stream_smem = (block / 32) * stream_smem_per_warp;
        if (stream_smem > smem_optin) return fail(QC_EUNSUPPORTED, "streaming kernel ring exceeds shared memory");
        if (!configured(stream_fn)) {
            CK(cudaFuncSetAttribute(stream_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin));
            configured_fns.push_back(stream_fn);
        }
    }
    int grid;
    DDArgs dda;
    memset(&dda, 0, sizeof dda);
    if (dds) {
        if (per_sm == 0) {
            int occ = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stream_fn, block, stream_smem);
            per_sm = (e == cudaSuccess && occ > 0) ? occ : 1;
        }
        const long warps_needed = std::max(1L, (long)n_row);
        grid = (int)std::max(1L, std::min((long)sm_count * per_sm, (warps_needed * 32 + block - 1) / block));
    } else if (ddp) {
        dda.D = data_desc();
        dda.wf = d_wf;
        dda.row_live = d_row_live;
        dda.n_dir = n_dir;
        dda.C = chain;
        for (int j = 0; j < n_terms; ++j) dda.nd[j] = cur_nd[j];
        dda.dd_solved = cur_nd[n] > 1;
        dda.acc = (double *)B.acc.ptr;
        dda.active = (const uint8_t *)B.active.ptr;
        grid = sm_count * 8;
    } else if (mom) {
        grid = 0;
    } else if (ws) {
        grid = ws_grid;
    } else if (streaming) {
        if (per_sm == 0) {
            int occ = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stream_fn, block, stream_smem);
            per_sm = (e == cudaSuccess && occ > 0) ? occ : 1;
        }
        const long warps_needed = std::max(1L, (long)sa.n_units);
        grid = (int)std::max(1L, std::min((long)sm_count * per_sm, (warps_needed * 32 + block - 1) / block));
    } else if (pipelined) {
        const int NW = L.pipe_nw;
        const long groups = (units + NW - 1) / NW;
        grid = (int)std::max(1L, std::min((long)sm_count, groups));
    } else {
        const int smem = (block / 32) * L.acc_smem_per_warp;
        if (!configured(L.fn)) {
            CK(cudaFuncSetAttribute(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin));
            configured_fns.push_back(L.fn);
        }
        if (per_sm == 0) {
            int occ = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, L.fn, block, smem);
            per_sm = (e == cudaSuccess && occ > 0) ? occ : 2;
        }
        const long warps_needed = std::max(1L, units);
        grid = (int)std::max(1L, std::min((long)sm_count * per_sm, (warps_needed * 32 + block - 1) / block));
    }
    int rc;
    if ((rc = ensure(B.chunk_act, (size_t)t.n_tint * aa.n_chunks))) return rc;
    aa.chunk_active = (const uint8_t *)B.chunk_act.ptr;
    sa.chunk_active = aa.chunk_active;
    pa.a = aa;
    pa.chunk_active = (const uint8_t *)B.chunk_act.ptr;
    pa.err = d_err;
    pa.wait_ns = qc_wait_limit_ns();
    pa.stall_issue = qc_wait_stall_stage();
    const int ca_threads = t.n_tint * aa.n_chunks;

    UpdArgs ua;
    ua.type = t.type;
    ua.n_bins = nb;
    ua.n_fint = t.n_fint;
    ua.n_ant = nat;
    ua.acc = (double *)B.acc.ptr;
    ua.params = (double *)B.params.ptr;
    ua.tab = (float4 *)B.tab.ptr;
    ua.gain_flags = (int8_t *)B.flags.ptr;
    ua.iters = (int *)B.iters.ptr;
    ua.active = (uint8_t *)B.active.ptr;
    ua.bin_nvis = (const long long *)B.nvis.ptr;
    ua.bin_nbytes = (const long long *)B.nvis.ptr + 2 * (size_t)nb;
    ua.vis_iters = (unsigned long long *)scalars.ptr;
    ua.acc_bytes = (unsigned long long *)scalars.ptr + 1;
    ua.tol = t.tol;
    // gain flagging on divergence: first / last relative updates and the parameters before the solve
    ua.div = (o->div_flag && !delay[n] && t.max_iter >= 4) ? 1 : 0;
    ua.max_iter = t.max_iter;
    ua.div_stats = nullptr;
    ua.params0 = nullptr;
    // the streaming kernel sums J^H W d in place of J^H W r (the update subtracts JHJ g)
    ua.b_form = (streaming && !dds && !delay[n]) ? 1 : 0;
    const size_t pbytes = nbytes<double>((size_t)nb * nat * (t.type == 2 ? 2 : 8));
    if (ua.div) {
        int rc_;
        if ((rc_ = ensure(B.div, nbytes<double>((size_t)nb * nat * 2)))) return rc_;
        if ((rc_ = ensure(B.params0, pbytes))) return rc_;
        ua.div_stats = (double *)B.div.ptr;
        ua.params0 = (const double *)B.params0.ptr;
    }
    int *cnt = (int *)B.cnt.ptr;
    const int upd_block = nat >= 128 ? 128 : (nat > 32 ? 64 : 32);
    // delay terms: the update reduces the channel bins of each parameter interval
    DelayUpdArgs dua;
    memset(&dua, 0, sizeof dua);
    if (delay[n]) {
        dua.d = delay_args(n, t);
        dua.acc = ua.acc;
        dua.gain_flags = ua.gain_flags;
        dua.iters = ua.iters;
        dua.active = ua.active;
        dua.bin_nvis = ua.bin_nvis;
        dua.bin_nbytes = ua.bin_nbytes;
        dua.vis_iters = ua.vis_iters;
        dua.acc_bytes = ua.acc_bytes;
        dua.tol = ua.tol;
    }

    // sums of the term solve: [bins][unordered pairs][MOM_N or MOM_E] FP32, the per-bin bytes of
    // one iteration for the byte counter, then the pass's row table
    MomArgs ma;
    MomNormArgs mn;
    memset(&ma, 0, sizeof ma);
    memset(&mn, 0, sizeof mn);
    const int mom_n = mom_form == FORM_E ? MOM_E : MOM_N;
    const size_t mom_words_all = mom ? (size_t)nb * n_up * mom_n : 0;
    const size_t mom_cnt_off = ((nbytes<float>(mom_words_all) + 15) / 16) * 16;
    const size_t mom_rows_off = ((mom_cnt_off + nbytes<long long>(nb) + 15) / 16) * 16;
    if (mom) {
        if ((rc = ensure(B.mom, mom_rows_off + nbytes<int4>(std::max(1L, n_strip_rows))))) return rc;
        ma.n_chan = n_chan;
        ma.n_ant = n_ant;
        ma.n_up = n_up;
        ma.vis = d_vis;
        ma.model = d_model;
        ma.wf = d_wf;
        ma.mrows = (const int4 *)((char *)B.mom.ptr + mom_rows_off);
        ma.strip_off = d_strip_off;
        ma.n_strips = n_strips;
        ma.n_chunks = (n_chan + 31) / 32;
        // an interval several times long: the rows inside each chunk keep a lane's key (units of
        // a whole strip x one chunk); else a row's chunks inside each row (units of whole rows x
        // a block of rows), so that an interval one time long flushes once per row.  Either way
        // about four units per resident warp
        ma.chunk_major = t.n_tint < n_time ? 1 : 0;
        const int max_strip = std::max(1, max_strip_rows);
        const long want_units = 4L * sm_count * 12;
        if (ma.chunk_major) {
            ma.group = 1;
            ma.rb = max_strip;
        } else {
            ma.group = ma.n_chunks;
            const long blocks = std::max(1L, (want_units + std::max(1, n_strips) - 1) / std::max(1, n_strips));
            ma.rb = (int)std::max(1L, (max_strip + blocks - 1) / blocks);
        }
        ma.n_rb = (max_strip + ma.rb - 1) / ma.rb;
        ma.tn = chain.t[n];
        ma.to = n_terms == 2 ? chain.t[1 - n] : chain.t[n];
        ma.mom = (float *)B.mom.ptr;
        mn.n_bins = nb;
        mn.n_ant = n_ant;
        mn.n_up = n_up;
        mn.type = t.type;
        mn.form = mom_form;
        mn.upair = d_upair;
        mn.mom = ma.mom;
        mn.params = (const double *)B.params.ptr;
        mn.tab = (const float4 *)B.tab.ptr;
        mn.n_fint = t.n_fint;
        mn.active = (const uint8_t *)B.active.ptr;
        mn.acc = (double *)B.acc.ptr;
        ua.bin_nbytes = (const long long *)((char *)B.mom.ptr + mom_cnt_off);
    }
    const long long mom_iter_bytes = 2LL * n_up * mom_n * 4 + 8LL * n_ant * (t.type == 1 ? KG_FULL : KG_DIAG);

    const int max_iter = t.max_iter;
    for (int k = 0; k < 2 * max_iter + 2; ++k) { cudaEvent_t ev; if ((rc = get_event(2 + k, ev))) return rc; }
    const int ev_pass = 2 + 2 * max_iter;     // the sums pass (its own bracket inside iteration 1's)
    // (no graph while a test stalls a stage: a captured graph would keep the stall)
    const bool use_graph = o->use_graph && !t.reduce && qc_wait_stall_stage() < 0;
    const unsigned rec_flags = use_graph ? cudaEventRecordExternal : cudaEventRecordDefault;

    auto enqueue = [&]() -> int {
        init_term_kernel<<<(std::max(nb, max_iter + 1) + 255) / 256, 256, 0, st>>>(nb, (uint8_t *)B.active.ptr, cnt,
                                                                                   max_iter + 1);
        CK(cudaGetLastError());
        if (ua.div) {
            CK(cudaMemsetAsync(B.div.ptr, 0, nbytes<double>((size_t)nb * nat * 2), st));
            CK(cudaMemcpyAsync(B.params0.ptr, B.params.ptr, pbytes, cudaMemcpyDeviceToDevice, st));
        }
        for (int k = 1; k <= max_iter; ++k) {
            aa.n_active = cnt + (k - 1);
            // inside a capture the record must be an external event node to be timed on replay
            {
                chunk_active_kernel<<<(ca_threads + 255) / 256, 256, 0, st>>>(aa.tn, n_chan, aa.n_chunks,
                                                                            (const uint8_t *)B.active.ptr, cnt + (k - 1),
                                                                            (uint8_t *)B.chunk_act.ptr);
                CK(cudaGetLastError());
            }
            CK(cudaEventRecordWithFlags(events[2 + 2 * (k - 1)], st, rec_flags));
            if (dds) {
                DDStreamArgs x;
                x.s = sa;
                x.s.n_active = cnt + (k - 1);
                x.n_dir = n_dir;
                x.nd_n = cur_nd[n];
                x.nd_o = n_terms == 2 ? cur_nd[1 - n] : 1;
                x.omega = delay[n] ? (const float *)B.domega.ptr : nullptr;
                const int gy = DS.dirs_per_cta > 0 ? (n_dir + DS.dirs_per_cta - 1) / DS.dirs_per_cta : 1;
                CK(DS.launch(dim3(grid, gy), block, stream_smem, st, x));
            } else if (ddp) {
                dda.n_active = cnt + (k - 1);
                CK(dd_launch_acc(dda, ts, grid, st));
            } else if (mom) {
                if (k == 1) {
                    CK(cudaMemsetAsync(B.mom.ptr, 0, nbytes<float>(mom_words_all), st));
                    CK(mom_launch_bytes(nb, (const long long *)B.nvis.ptr + 2 * (size_t)nb, mom_iter_bytes,
                                        (long long *)((char *)B.mom.ptr + mom_cnt_off), ua.acc_bytes, st));
                    CK(mom_launch_rows(n_strip_rows, d_strip_rows, d_rows, d_row_live, d_up_of_bl,
                                       const_cast<int4 *>(ma.mrows), st));
                    CK(cudaEventRecordWithFlags(events[ev_pass], st, rec_flags));
                    ma.n_active = cnt;
                    CK(mom_launch_pass(ma, mom_form, mom_ok, sm_count, st));
                    CK(cudaEventRecordWithFlags(events[ev_pass + 1], st, rec_flags));
                }
                mn.n_active = cnt + (k - 1);
                CK(mom_launch_normal(mn, st));
            } else if (ws) {
                wa.n_active = cnt + (k - 1);
                const uint8_t *ca = (const uint8_t *)B.chunk_act.ptr;
                if (order == 0) {
                    CK(cudaMemsetAsync(B.ws_n.ptr, 0, sizeof(int), st));
                    if (n_row)
                        ws_rows_kernel<<<(n_row + 255) / 256, 256, 0, st>>>(
                            n_row, wa.rt, wa.rt_scale, ca, wa.n_chunks, wa.nwr, wa.n_active, (int4 *)B.ws_rl.ptr,
                            m16 ? (float *)B.ws_rls.ptr : nullptr, (unsigned *)B.ws_rlb.ptr, (int *)B.ws_n.ptr);
                } else {
                    if (wa.nwk)
                        ws_strip_bits_kernel<<<(wa.nwk + 7) / 8, 256, 0, st>>>(
                            n_strip_rows, wa.rt, ca, wa.n_chunks, wa.nwk, wa.n_active, (unsigned *)B.ws_sb.ptr);
                    CK(cudaMemsetAsync(B.units.ptr, 0, sizeof(int), st));
                }
                CK(cudaGetLastError());
                if (self_feed) CK(L.wss_launch(ws_grid, ws_smem, st, wa));
                else CK(L.ws_launch(ws_grid, ws_smem, st, wa));
            } else if (streaming) {
                sa.n_active = cnt + (k - 1);
                if (sa.unit_counter) CK(cudaMemsetAsync(sa.unit_counter, 0, sizeof(int), st));
                if (ded) {
                    DelayStreamArgs dsa;
                    dsa.s = sa;
                    dsa.omega = (const float *)B.domega.ptr;
                    CK(DL.launch(grid, block, stream_smem, st, dsa));
                } else {
                    CK(L.stream_launch(grid, block, stream_smem, st, sa));
                }
            } else if (pipelined) {
                pa.a.n_active = cnt + (k - 1);
                CK(L.pipe_launch(grid, pipe_smem, st, pa));
            } else {
                CK(L.launch(grid, block, st, aa));
            }
            CK(cudaEventRecordWithFlags(events[2 + 2 * (k - 1) + 1], st, rec_flags));
            if (t.reduce) {
                const size_t KG = psums ? KG_SUMS : (t.type == 1 ? KG_FULL : KG_DIAG);
                if (o->allreduce((double *)B.acc.ptr, (int64_t)(psums ? nbu : nb) * nat * KG, st, o->allreduce_user))
                    return fail(QC_ECUDA, "allreduce callback failed");
            }
            ua.k = k;
            ua.alpha = (o->damping_mode == QC_DAMP_ALTERNATE) ? ((k % 2 == 0) ? 0.5 : 1.0)
                                                               : (o->damping > 0 ? o->damping : 1.0);
            ua.n_active_prev = cnt + (k - 1);
            ua.n_active_next = cnt + k;
            if (delay[n]) {
                dua.k = k;
                dua.alpha = ua.alpha;
                dua.n_active_prev = ua.n_active_prev;
                dua.n_active_next = ua.n_active_next;
                if (psums) delay_update_kernel<true><<<dua.d.n_tint * dua.d.n_fint, 128, 0, st>>>(dua);
                else delay_update_kernel<false><<<dua.d.n_tint * dua.d.n_fint, upd_block, 0, st>>>(dua);
            } else {
                update_kernel<<<nb, upd_block, 0, st>>>(ua);
            }
            CK(cudaGetLastError());
        }
        return QC_OK;
    };
    if (use_graph) {
        if (!B.graph_valid) {
            if (B.exec) { cudaGraphExecDestroy(B.exec); B.exec = nullptr; }
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            rc = enqueue();
            // always end the capture, so that a failure leaves the stream usable
            cudaError_t e = cudaStreamEndCapture(st, &g);
            if (rc || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                if (rc) return rc;
                return cuda_fail(e, "cudaStreamEndCapture");
            }
            e = cudaGraphInstantiate(&B.exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            B.graph_valid = true;
        }
        CK(cudaGraphLaunch(B.exec, st));
    } else {
        if ((rc = enqueue())) return rc;
    }
    launches += 1 + 3 * (long long)max_iter + (mom ? 3 : 0);
    // iteration bookkeeping: which accumulate launches did work, and their device time
    std::vector<int> hcnt(max_iter + 1);
    int herr = 0;
    CK(cudaMemcpyAsync(hcnt.data(), cnt, nbytes<int>(max_iter + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) {
        CK(cudaMemsetAsync(d_err, 0, sizeof(int), st));
        return fail(QC_ETIMEOUT, "a bounded wait in a bulk-copy accumulate kernel gave up");
    }
    double ms_sum = 0;
    long long worked = 0;
    int last = 0;
    for (int k = 1; k <= max_iter; ++k) {
        if (hcnt[k - 1] == 0) break;
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, events[2 + 2 * (k - 1)], events[2 + 2 * (k - 1) + 1]));
        ms_sum += ms;
        ++worked;
        last = k;
    }
    if (mom && hcnt[0] != 0) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, events[ev_pass], events[ev_pass + 1]));
        *pass_ms = ms;
    }
    *it_max = last;
    *acc_ms = ms_sum;
    *acc_launches = worked;
    return QC_OK;
}

// ---------------------------------------------------------------------------
// MAD residual flagging (Section 4, "Additional features"; global mode)
// ---------------------------------------------------------------------------
//
// The statistic of an unflagged cross-correlation sample is its whitened residual norm
// z = sqrt(sum_c w_c |r_c|^2), computed in float32 with every operation rounded (no fused
// multiply-add) in a fixed order.  Median and MAD are exact order statistics (the
// floor((n - 1) / 2)-th smallest value), found by a radix select over the float bit
// patterns, which order like the values for non-negative floats.  A sample is flagged when
// |z - median| > fl32(threshold * 1.4826) * MAD in float32.

namespace {

constexpr unsigned MAD_SENTINEL = 0x7f800000u;   // +inf: excluded samples sort after the rest

__device__ __forceinline__ bool mad_use(const int4 *rows, const uint8_t *flag, long i, int n_chan)
{
    const int4 r = rows[i / n_chan];
    return r.x != r.y && !(flag && flag[i]);
}

__global__ void mad_z_kernel(long n_vis, int n_chan, const float4 *resid, const float4 *weight, const uint8_t *flag,
                             const int4 *rows, unsigned *keys, unsigned long long *n_used)
{
    unsigned cnt = 0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_vis; i += (long)gridDim.x * blockDim.x) {
        unsigned key = MAD_SENTINEL;
        if (mad_use(rows, flag, i, n_chan)) {
            const float4 lo = resid[2 * i], hi = resid[2 * i + 1];
            const float4 w = weight[i];
            const float t0 = __fadd_rn(__fmul_rn(lo.x, lo.x), __fmul_rn(lo.y, lo.y));
            const float t1 = __fadd_rn(__fmul_rn(lo.z, lo.z), __fmul_rn(lo.w, lo.w));
            const float t2 = __fadd_rn(__fmul_rn(hi.x, hi.x), __fmul_rn(hi.y, hi.y));
            const float t3 = __fadd_rn(__fmul_rn(hi.z, hi.z), __fmul_rn(hi.w, hi.w));
            float acc = __fmul_rn(w.x, t0);
            acc = __fadd_rn(acc, __fmul_rn(w.y, t1));
            acc = __fadd_rn(acc, __fmul_rn(w.z, t2));
            acc = __fadd_rn(acc, __fmul_rn(w.w, t3));
            key = __float_as_uint(__fsqrt_rn(acc));
            ++cnt;
        }
        keys[i] = key;
    }
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_used, (unsigned long long)cnt);
}

// histogram of the 8 bits at `shift` of the keys whose bits above them equal `prefix`
__global__ void mad_hist_kernel(long n, const unsigned *keys, unsigned prefix, unsigned mask, int shift, unsigned *hist)
{
    __shared__ unsigned h[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const unsigned k = keys[i];
        if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[t], h[t]);
}

// keys of the used samples become the bits of |z - median|
__global__ void mad_dev_kernel(long n_vis, int n_chan, const uint8_t *flag, const int4 *rows, float med, unsigned *keys)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_vis; i += (long)gridDim.x * blockDim.x)
        if (mad_use(rows, flag, i, n_chan)) keys[i] = __float_as_uint(fabsf(__fsub_rn(__uint_as_float(keys[i]), med)));
}

__global__ void mad_flag_kernel(long n_vis, int n_chan, const uint8_t *flag, const int4 *rows, const unsigned *keys,
                                float thr, uint8_t *out, unsigned long long *n_flagged)
{
    unsigned cnt = 0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_vis; i += (long)gridDim.x * blockDim.x) {
        const bool f = mad_use(rows, flag, i, n_chan) && __uint_as_float(keys[i]) > thr;
        out[i] = f ? 1 : 0;
        cnt += f ? 1u : 0u;
    }
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_flagged, (unsigned long long)cnt);
}

// per-baseline mode: one block per group of rows (the rows of one baseline in either
// orientation); two exact order statistics of its used samples by four 8-bit radix passes
// with a shared-memory histogram, then its flags
__device__ __forceinline__ unsigned mad_block_select(const unsigned *keys, const int *grows, int n_grow, int n_chan,
                                                     const uint8_t *flag, unsigned long long k, unsigned *hist,
                                                     unsigned *s_res)
{
    unsigned prefix = 0, mask = 0;
    const long n = (long)n_grow * n_chan;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
        __syncthreads();
        for (long i = threadIdx.x; i < n; i += blockDim.x) {
            const long sidx = (long)grows[i / n_chan] * n_chan + (i % n_chan);
            if (flag && flag[sidx]) continue;
            const unsigned kk = keys[sidx];
            if ((kk & mask) == prefix) atomicAdd(&hist[(kk >> shift) & 0xffu], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long cum = 0;
            int b = 0;
            for (; b < 255; ++b) {
                if (cum + hist[b] > k) break;
                cum += hist[b];
            }
            s_res[0] = (unsigned)b;
            s_res[1] = (unsigned)(k - cum);
        }
        __syncthreads();
        prefix |= s_res[0] << shift;
        mask |= 0xffu << shift;
        k = s_res[1];
        __syncthreads();
    }
    return prefix;
}

__global__ void __launch_bounds__(256) mad_group_kernel(int n_chan, const int *goff, const int *grows,
                                                        const uint8_t *flag, unsigned *keys, float factor,
                                                        uint8_t *out, unsigned long long *n_flagged)
{
    __shared__ unsigned hist[256];
    __shared__ unsigned s_res[2];
    __shared__ unsigned long long s_cnt;
    const int g = blockIdx.x;
    const int *rows = grows + goff[g];
    const int n_grow = goff[g + 1] - goff[g];
    const long n = (long)n_grow * n_chan;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    unsigned long long used = 0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) {
        const long sidx = (long)rows[i / n_chan] * n_chan + (i % n_chan);
        if (!(flag && flag[sidx])) ++used;
    }
    atomicAdd(&s_cnt, used);
    __syncthreads();
    const unsigned long long n_used = s_cnt;
    float thr = INFINITY;
    if (n_used > 0) {
        const unsigned long long k = (n_used - 1) / 2;
        const unsigned med_bits = mad_block_select(keys, rows, n_grow, n_chan, flag, k, hist, s_res);
        const float med = __uint_as_float(med_bits);
        for (long i = threadIdx.x; i < n; i += blockDim.x) {
            const long sidx = (long)rows[i / n_chan] * n_chan + (i % n_chan);
            if (!(flag && flag[sidx])) keys[sidx] = __float_as_uint(fabsf(__fsub_rn(__uint_as_float(keys[sidx]), med)));
        }
        __syncthreads();
        const unsigned mad_bits = mad_block_select(keys, rows, n_grow, n_chan, flag, k, hist, s_res);
        thr = __fmul_rn(factor, __uint_as_float(mad_bits));
    }
    unsigned cnt = 0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) {
        const long sidx = (long)rows[i / n_chan] * n_chan + (i % n_chan);
        const bool f = !(flag && flag[sidx]) && __uint_as_float(keys[sidx]) > thr;
        out[sidx] = f ? 1 : 0;
        cnt += f ? 1u : 0u;
    }
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_flagged, (unsigned long long)cnt);
}

} // namespace

// the k-th smallest of n keys (0-based), k < n: four 8-bit radix passes from the top bits
static int mad_select(qc_ctx *c, const unsigned *keys, long n, unsigned long long k, unsigned *hist, cudaStream_t st,
                      unsigned &out)
{
    unsigned prefix = 0, mask = 0;
    unsigned h[256];
    for (int shift = 24; shift >= 0; shift -= 8) {
        CK(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned), st));
        mad_hist_kernel<<<grid_for(n, 256, c->sm_count), 256, 0, st>>>(n, keys, prefix, mask, shift, hist);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h, hist, sizeof h, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        unsigned long long cum = 0;
        int b = 0;
        for (; b < 256; ++b) {
            if (cum + h[b] > k) break;
            cum += h[b];
        }
        if (b == 256) return c->fail(QC_ECUDA, "radix select lost its element");
        k -= cum;
        prefix |= (unsigned)b << shift;
        mask |= 0xffu << shift;
    }
    out = prefix;
    return QC_OK;
}

extern "C" int qc_mad_flag(qc_ctx *c, const qc_term *terms, int32_t n_terms, double threshold, int32_t per_baseline,
                           uint8_t *flags_out, int32_t out_memory, int64_t *n_flagged)
{
    if (!c) return QC_EINVAL;
    c->err.clear();
    if (!flags_out) return c->fail(QC_EINVAL, "flags_out is NULL");
    if (c->n_dir > 1) return c->fail(QC_EUNSUPPORTED, "qc_mad_flag takes problems with one direction");
    if (!(threshold > 0) || !std::isfinite(threshold)) return c->fail(QC_EINVAL, "threshold must be positive and finite");
    if (out_memory != QC_MEM_HOST && out_memory != QC_MEM_DEVICE) return c->fail(QC_EINVAL, "out_memory invalid");
    int rc = c->validate_terms(terms, n_terms, false);
    if (rc) return rc;
    cudaStream_t st = c->own_stream;
    std::vector<qc_term> xt;
    if ((rc = c->expand_terms(terms, n_terms, xt, st))) return rc;
    Chain chain;
    if ((rc = c->stage_terms(xt.data(), n_terms, st, chain))) return rc;
    const long n_vis = (long)c->n_row * c->n_chan;
    if ((rc = c->ensure(c->scalars, 64))) return rc;
    if ((rc = c->ensure(c->resid_stage, nbytes<float4>(2 * (size_t)std::max(1L, n_vis))))) return rc;
    if ((rc = c->ensure(c->mad_keys, nbytes<unsigned>((size_t)std::max(1L, n_vis))))) return rc;
    if ((rc = c->ensure(c->mad_hist, 256 * sizeof(unsigned) + 2 * sizeof(unsigned long long)))) return rc;
    double *d_chi2 = (double *)c->scalars.ptr;
    float4 *dres = (float4 *)c->resid_stage.ptr;
    unsigned *keys = (unsigned *)c->mad_keys.ptr;
    unsigned *hist = (unsigned *)c->mad_hist.ptr;
    unsigned long long *cnt = (unsigned long long *)((char *)c->mad_hist.ptr + 256 * sizeof(unsigned));
    uint8_t *dout = (uint8_t *)flags_out;
    if (out_memory == QC_MEM_HOST) {
        if ((rc = c->ensure(c->mad_out, (size_t)std::max(1L, n_vis)))) return rc;
        dout = (uint8_t *)c->mad_out.ptr;
    }
    if (n_vis == 0) {
        if (n_flagged) *n_flagged = 0;
        return QC_OK;
    }
    if ((rc = c->run_residual(chain, dres, d_chi2, st))) return rc;
    CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
    const int grid = grid_for(n_vis, 256, c->sm_count);
    mad_z_kernel<<<grid, 256, 0, st>>>(n_vis, c->n_chan, dres, c->d_weight, c->d_flag, c->d_rows, keys, cnt);
    CK(cudaGetLastError());
    unsigned long long hc[2];
    CK(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (per_baseline) {
        // groups: the rows of each unordered antenna pair (cross-correlations only)
        std::vector<int4> hrows(c->n_row);
        CK(cudaMemcpyAsync(hrows.data(), c->d_rows, nbytes<int4>(c->n_row), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::vector<int> gid((size_t)c->n_ant * c->n_ant, -1), count;
        std::vector<int> row_g(c->n_row, -1);
        for (int r = 0; r < c->n_row; ++r) {
            const int a1 = hrows[r].x, a2 = hrows[r].y;
            if (a1 == a2) continue;
            int &slot = gid[(size_t)std::min(a1, a2) * c->n_ant + std::max(a1, a2)];
            if (slot < 0) { slot = (int)count.size(); count.push_back(0); }
            row_g[r] = slot;
            ++count[slot];
        }
        const int n_groups = (int)count.size();
        std::vector<int> goff(n_groups + 1, 0), grows;
        for (int gi = 0; gi < n_groups; ++gi) goff[gi + 1] = goff[gi] + count[gi];
        grows.resize(goff[n_groups]);
        std::vector<int> fill(goff.begin(), goff.end() - 1);
        for (int r = 0; r < c->n_row; ++r) if (row_g[r] >= 0) grows[fill[row_g[r]]++] = r;
        CK(cudaMemsetAsync(dout, 0, (size_t)n_vis, st));
        if (n_groups > 0) {
            if ((rc = c->ensure(c->mad_groups, nbytes<int>(goff.size() + grows.size())))) return rc;
            int *dgoff = (int *)c->mad_groups.ptr, *dgrows = dgoff + goff.size();
            CK(cudaMemcpyAsync(dgoff, goff.data(), nbytes<int>(goff.size()), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(dgrows, grows.data(), nbytes<int>(grows.size()), cudaMemcpyHostToDevice, st));
            mad_group_kernel<<<n_groups, 256, 0, st>>>(c->n_chan, dgoff, dgrows, c->d_flag, keys,
                                                      (float)(threshold * 1.4826), dout, cnt + 1);
            CK(cudaGetLastError());
        }
        if (out_memory == QC_MEM_HOST) CK(cudaMemcpyAsync(flags_out, dout, (size_t)n_vis, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hc + 1, cnt + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (n_flagged) *n_flagged = (int64_t)hc[1];
        return QC_OK;
    }
    float thr = 0.f;
    if (hc[0] > 0) {
        const unsigned long long k = (hc[0] - 1) / 2;
        unsigned med_bits = 0, mad_bits = 0;
        if ((rc = mad_select(c, keys, n_vis, k, hist, st, med_bits))) return rc;
        float med;
        memcpy(&med, &med_bits, sizeof med);
        mad_dev_kernel<<<grid, 256, 0, st>>>(n_vis, c->n_chan, c->d_flag, c->d_rows, med, keys);
        CK(cudaGetLastError());
        if ((rc = mad_select(c, keys, n_vis, k, hist, st, mad_bits))) return rc;
        float mad;
        memcpy(&mad, &mad_bits, sizeof mad);
        const float factor = (float)(threshold * 1.4826);
        thr = factor * mad;
    }
    mad_flag_kernel<<<grid, 256, 0, st>>>(n_vis, c->n_chan, hc[0] > 0 ? c->d_flag : nullptr, c->d_rows, keys,
                                         hc[0] > 0 ? thr : INFINITY, dout, cnt + 1);
    CK(cudaGetLastError());
    if (out_memory == QC_MEM_HOST) CK(cudaMemcpyAsync(flags_out, dout, (size_t)n_vis, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hc + 1, cnt + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (n_flagged) *n_flagged = (int64_t)hc[1];
    return QC_OK;
}
