// qc_moments.cuh -- argument blocks of the sums pass and the per-iteration normal equations of
// a single-term chain (kernels in qc_moments.cu).
#pragma once

#include "qc_kernels.cuh"

namespace qc {

constexpr int MOM_N = 100;          // FP64 words per (interval, baseline): S 64, T 32, U 4
constexpr int MOM_T = 64, MOM_U = 96;

// Hermitian pairs (u, v), u < v, of the 4x4 S blocks: packed as 4 diagonal reals then 6 (re, im)
__host__ __device__ constexpr int mom_pair(int u, int v)
{
    return u == 0 ? (v == 1 ? 0 : v == 2 ? 1 : 2) : u == 1 ? (v == 2 ? 3 : 4) : 5;
}

struct MomArgs {
    int n_chan, n_up;                    // n_up: unordered antenna pairs with data
    const float4 *vis, *model, *wf;      // wf: weights with flags and autocorrelations folded in (w = 0)
    const int4 *mrows;                   // [strip rows] {row or -1, first bin of its time, pair, ant1 > ant2}
    const int *strip_off;                // rows of each ordered baseline (offsets into mrows)
    int n_strips, n_chunks;              // n_chunks: 16-channel chunks of a row
    int group;                           // 16-channel chunks per unit of work
    DevTerm tn;                          // the solved term (maps)
    double *mom;                         // [bins][n_up][MOM_N]
    const int *n_active;
};

struct MomNormArgs {
    int n_bins, n_ant, n_up, type;       // type: QC_TERM_* (diag, full, phase)
    const int *upair;                    // [n_ant][n_ant] unordered pair index or -1
    const double *mom;                   // [bins][n_up][MOM_N]
    const double *params;                // FP64 gains of the solved term
    const uint8_t *active;               // [bins]
    const int *n_active;
    double *acc;                         // [bins][n_ant][KG] (written)
};

} // namespace qc
