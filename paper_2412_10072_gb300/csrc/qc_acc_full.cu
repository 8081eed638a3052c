// qc_acc_full.cu -- accumulate kernels for full 2x2 solved terms.
#include "qc_acc_inst.cuh"

AccLaunch acc_launcher_full(bool simple, int lk, int rk, bool m16)
{
    return m16 ? qc_inst::pick<qc::TS_FULL, true>(simple, lk, rk) : qc_inst::pick<qc::TS_FULL, false>(simple, lk, rk);
}
