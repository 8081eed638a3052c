// qc_acc.cu -- instantiations of the accumulate kernel for every
// (solved-term family, left-chain kind, right-chain kind, model precision).
#include "qc_internal.h"

using namespace qc;

namespace {

template <int TS, int LK, int RK, bool M16>
cudaError_t launch_acc(int grid, int block, cudaStream_t st, const AccArgs &a)
{
    acc_kernel<TS, LK, RK, M16><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <int TS, int LK, int RK, bool M16> AccLaunch make()
{
    AccLaunch l;
    l.fn = (const void *)acc_kernel<TS, LK, RK, M16>;
    l.launch = launch_acc<TS, LK, RK, M16>;
    return l;
}

template <int TS, int LK, bool M16> AccLaunch by_rk(int rk)
{
    switch (rk) {
    case KIND_NONE: return make<TS, LK, KIND_NONE, M16>();
    case KIND_DIAG: return make<TS, LK, KIND_DIAG, M16>();
    default: return make<TS, LK, KIND_FULL, M16>();
    }
}

template <int TS, bool M16> AccLaunch by_lk(int lk, int rk)
{
    switch (lk) {
    case KIND_NONE: return by_rk<TS, KIND_NONE, M16>(rk);
    case KIND_DIAG: return by_rk<TS, KIND_DIAG, M16>(rk);
    default: return by_rk<TS, KIND_FULL, M16>(rk);
    }
}

} // namespace

AccLaunch acc_launcher(int ts, int lk, int rk, bool m16)
{
    if (ts == TS_FULL) return m16 ? by_lk<TS_FULL, true>(lk, rk) : by_lk<TS_FULL, false>(lk, rk);
    return m16 ? by_lk<TS_DIAG, true>(lk, rk) : by_lk<TS_DIAG, false>(lk, rk);
}
