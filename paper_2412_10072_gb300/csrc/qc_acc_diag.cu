// qc_acc_diag.cu -- accumulate kernels for diagonal and phase-only solved terms.
#include "qc_acc_inst.cuh"

AccLaunch acc_launcher_diag(bool simple, int lk, int rk, bool m16)
{
    return m16 ? qc_inst::pick<qc::TS_DIAG, true>(simple, lk, rk) : qc_inst::pick<qc::TS_DIAG, false>(simple, lk, rk);
}
