// qc_acc_delay.cu -- instantiations of the streaming accumulate kernel of a solved delay
// term, for each kind of the other term of a chain of one or two terms.
#include "qc_internal.h"

using namespace qc;

namespace {

constexpr int DELAY_DEPTH = 4;   // ring depth (steps), as the other streaming kernels

template <bool M16> constexpr int smem_per_warp()
{
    return DELAY_DEPTH * ((M16 ? 4 : 5) * 32 * 16 + 2 * 16);
}

template <int LK, int RK, bool M16>
cudaError_t launch_delay(int grid, int block, int smem_bytes, cudaStream_t st, const DelayStreamArgs &a)
{
    acc_delay_kernel<LK, RK, M16, DELAY_DEPTH><<<grid, block, smem_bytes, st>>>(a);
    return cudaGetLastError();
}

template <int LK, int RK, bool M16> DelayLaunch make()
{
    DelayLaunch l;
    l.fn = (const void *)acc_delay_kernel<LK, RK, M16, DELAY_DEPTH>;
    l.launch = launch_delay<LK, RK, M16>;
    l.smem_per_warp = smem_per_warp<M16>();
    return l;
}

template <bool M16> DelayLaunch pick(int lk, int rk)
{
    if (lk == KIND_NONE && rk == KIND_NONE) return make<KIND_NONE, KIND_NONE, M16>();
    if (rk == KIND_NONE) return lk == KIND_FULL ? make<KIND_FULL, KIND_NONE, M16>() : make<KIND_DIAG, KIND_NONE, M16>();
    if (lk == KIND_NONE) return rk == KIND_FULL ? make<KIND_NONE, KIND_FULL, M16>() : make<KIND_NONE, KIND_DIAG, M16>();
    return DelayLaunch();
}

} // namespace

DelayLaunch delay_launcher(int lk, int rk, bool m16) { return m16 ? pick<true>(lk, rk) : pick<false>(lk, rk); }
