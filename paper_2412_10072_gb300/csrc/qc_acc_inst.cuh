// qc_acc_inst.cuh -- instantiation helpers for the accumulate kernels of one
// solved-term family (included by qc_acc_diag.cu and qc_acc_full.cu).
#pragma once
#include "qc_internal.h"

namespace qc_inst {
using namespace qc;

constexpr int PIPE_NW = 15;   // consumer warps per CTA (16 warps with the producer)
constexpr int PIPE_NS = 5;    // shared-memory ring stages

template <int TS, int LK, int RK, bool SIMPLE, bool M16>
cudaError_t launch_acc(int grid, int block, cudaStream_t st, const AccArgs &a)
{
    acc_kernel<TS, LK, RK, SIMPLE, M16><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <int TS, int LK, int RK, bool SIMPLE, bool M16>
cudaError_t launch_pipe(int grid, cudaStream_t st, const PipeArgs &p)
{
    constexpr int bytes = PipeLayout<PIPE_NW, PIPE_NS, M16 ? 16 : 32>::BYTES;
    acc_pipe_kernel<TS, LK, RK, SIMPLE, M16, PIPE_NW, PIPE_NS><<<grid, (PIPE_NW + 1) * 32, bytes, st>>>(p);
    return cudaGetLastError();
}

template <int TS, int LK, int RK, bool SIMPLE, bool M16> AccLaunch make()
{
    AccLaunch l;
    l.fn = (const void *)acc_kernel<TS, LK, RK, SIMPLE, M16>;
    l.launch = launch_acc<TS, LK, RK, SIMPLE, M16>;
    l.pipe_fn = (const void *)acc_pipe_kernel<TS, LK, RK, SIMPLE, M16, PIPE_NW, PIPE_NS>;
    l.pipe_launch = launch_pipe<TS, LK, RK, SIMPLE, M16>;
    l.pipe_smem = PipeLayout<PIPE_NW, PIPE_NS, M16 ? 16 : 32>::BYTES;
    l.pipe_threads = (PIPE_NW + 1) * 32;
    return l;
}

// Chains of one or two terms get a kernel whose chain shape is fixed at compile
// time (the other term, if any, is the single left or right factor of its kind);
// longer chains use the general kernel, which multiplies every term out as a full
// 2x2 Jones matrix.
template <int TS, bool M16> AccLaunch pick(bool simple, int lk, int rk)
{
    if (!simple) return make<TS, KIND_FULL, KIND_FULL, false, M16>();
    if (lk == KIND_NONE && rk == KIND_NONE) return make<TS, KIND_NONE, KIND_NONE, true, M16>();
    if (lk == KIND_NONE && rk == KIND_DIAG) return make<TS, KIND_NONE, KIND_DIAG, true, M16>();
    if (lk == KIND_NONE && rk == KIND_FULL) return make<TS, KIND_NONE, KIND_FULL, true, M16>();
    if (lk == KIND_DIAG && rk == KIND_NONE) return make<TS, KIND_DIAG, KIND_NONE, true, M16>();
    if (lk == KIND_FULL && rk == KIND_NONE) return make<TS, KIND_FULL, KIND_NONE, true, M16>();
    return AccLaunch();
}
} // namespace qc_inst
