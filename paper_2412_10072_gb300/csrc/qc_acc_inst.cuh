// qc_acc_inst.cuh -- instantiation helpers for the accumulate kernels of one
// solved-term family (included by qc_acc_diag.cu and qc_acc_full.cu).
#pragma once
#include "qc_internal.h"

namespace qc_inst {
using namespace qc;

constexpr int PIPE_NW = 10;   // warps per CTA of the pipelined kernel
constexpr int PIPE_H = 2;     // row segments of 32 channels per warp step

constexpr int ACC_DEPTH = 4;  // cp.async ring depth (segments) of the prefetching kernel
constexpr int STREAM_DEPTH = 4;   // ring depth (steps) of the streaming kernel
constexpr int WS_NC = 7;          // consumer warps per CTA of the warp-specialised kernel (two CTAs per SM)
constexpr int WSS_NW = 8;         // warps per CTA of the self-feeding kernel (two CTAs per SM)

template <bool M16> constexpr int stream_smem_per_warp()
{
    return STREAM_DEPTH * ((M16 ? 4 : 5) * 32 * 16 + 2 * 16);
}


template <int TS, int LK, int RK, bool SIMPLE, bool M16>
cudaError_t launch_acc(int grid, int block, cudaStream_t st, const AccArgs &a)
{
    const int smem = (block / 32) * ACC_DEPTH * 32 * (M16 ? 4 : 5) * 16;
    acc_kernel<TS, LK, RK, SIMPLE, M16, ACC_DEPTH><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int TS, int LK, int RK, bool M16>
cudaError_t launch_pipe(int grid, int smem_bytes, cudaStream_t st, const PipeArgs &p)
{
    acc_pipe_kernel<TS, LK, RK, M16, PIPE_NW, PIPE_H><<<grid, PIPE_NW * 32, smem_bytes, st>>>(p);
    return cudaGetLastError();
}

template <int TS, int LK, int RK, bool M16>
cudaError_t launch_stream(int grid, int block, int smem_bytes, cudaStream_t st, const StreamArgs &a)
{
    acc_stream_kernel<TS, LK, RK, M16, STREAM_DEPTH><<<grid, block, smem_bytes, st>>>(a);
    return cudaGetLastError();
}

template <int TS, int LK, int RK, bool M16>
cudaError_t launch_ws(int grid, int smem_bytes, cudaStream_t st, const WsArgs &a)
{
    acc_ws_kernel<TS, LK, RK, M16, WS_NC><<<grid, (WS_NC + 1) * 32, smem_bytes, st>>>(a);
    return cudaGetLastError();
}

template <int TS, int LK, int RK, bool M16>
cudaError_t launch_wsself(int grid, int smem_bytes, cudaStream_t st, const WsArgs &a)
{
    if (a.order == 0) acc_run_kernel<TS, LK, RK, M16, 0, WSS_NW><<<grid, WSS_NW * 32, smem_bytes, st>>>(a);
    else acc_run_kernel<TS, LK, RK, M16, 1, WSS_NW><<<grid, WSS_NW * 32, smem_bytes, st>>>(a);
    return cudaGetLastError();
}

template <int TS, int LK, int RK, bool SIMPLE, bool M16> AccLaunch make()
{
    AccLaunch l;
    l.fn = (const void *)acc_kernel<TS, LK, RK, SIMPLE, M16, ACC_DEPTH>;
    l.acc_smem_per_warp = ACC_DEPTH * 32 * (M16 ? 4 : 5) * 16;
    l.launch = launch_acc<TS, LK, RK, SIMPLE, M16>;
    if constexpr (SIMPLE) {
        l.pipe_fn = (const void *)acc_pipe_kernel<TS, LK, RK, M16, PIPE_NW, PIPE_H>;
        l.pipe_launch = launch_pipe<TS, LK, RK, M16>;
        l.pipe_nw = PIPE_NW;
        l.pipe_h = PIPE_H;
        l.stream_fn = (const void *)acc_stream_kernel<TS, LK, RK, M16, STREAM_DEPTH>;
        l.stream_launch = launch_stream<TS, LK, RK, M16>;
        l.stream_smem_per_warp = stream_smem_per_warp<M16>();
        l.ws_fn = (const void *)acc_ws_kernel<TS, LK, RK, M16, WS_NC>;
        l.ws_launch = launch_ws<TS, LK, RK, M16>;
        l.ws_nc = WS_NC;
        l.wss_fn = (const void *)acc_run_kernel<TS, LK, RK, M16, 0, WSS_NW>;
        l.wss_fn1 = (const void *)acc_run_kernel<TS, LK, RK, M16, 1, WSS_NW>;
        l.wss_launch = launch_wsself<TS, LK, RK, M16>;
        l.wss_nw = WSS_NW;
    }
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
