// qc_moments.cuh -- argument blocks of the sums pass and the per-iteration normal equations of
// a single-term chain (kernels in qc_moments.cu).
#pragma once

#include "qc_kernels.cuh"

namespace qc {

constexpr int MOM_N = 100;          // FP32 words per (interval, pair), full form: S 64, T 32, U 4
constexpr int MOM_T = 64, MOM_U = 96;
// diagonal form (a diagonal or phase-only solved term with a term to its left): S' 16 (4x4
// Hermitian packed as S), T' 8, U 1, three words of padding (slots of whole 16-byte vectors)
constexpr int MOM_E = 28;
constexpr int MOM_ET = 16, MOM_EU = 24;
constexpr int FORM_FULL = 0, FORM_E = 1;

// Hermitian pairs (u, v), u < v, of the 4x4 S blocks: packed as 4 diagonal reals then 6 (re, im)
__host__ __device__ constexpr int mom_pair(int u, int v)
{
    return u == 0 ? (v == 1 ? 0 : v == 2 ? 1 : 2) : u == 1 ? (v == 2 ? 3 : 4) : 5;
}

struct MomArgs {
    int n_chan, n_ant, n_up;             // n_up: unordered antenna pairs with data
    const float4 *vis, *model, *wf;      // wf: weights with flags and autocorrelations folded in (w = 0)
    // [strip rows] {row or -1 (nothing usable), time, pair | conj << 31, p | q << 16}: p, q the
    // antennas of the baseline as oriented in the sums (p < q); conj: the row is (q, p)
    const int4 *mrows;
    const int *strip_off;                // rows of each ordered baseline (offsets into mrows)
    int n_strips, n_chunks;              // n_chunks: 32-channel chunks of a row
    int group;                           // chunks per unit of work
    int rb, n_rb;                        // rows of a strip per unit of work, blocks per strip
    int chunk_major;                     // 1: a unit's rows inside each chunk; 0: a row's chunks inside it
    DevTerm tn;                          // the solved term (maps)
    DevTerm to;                          // the fixed other term of a two-term chain (tables)
    float *mom;                          // [bins][n_up][MOM_N or MOM_E]
    const int *n_active;
};

struct MomNormArgs {
    int n_bins, n_ant, n_up, type;       // type: QC_TERM_* (diag, full, phase)
    int form;                            // FORM_FULL or FORM_E
    const int *upair;                    // [n_ant][n_ant] unordered pair index or -1
    const float *mom;                    // [bins][n_up][MOM_N or MOM_E]
    const double *params;                // FP64 gains of the solved term
    const float4 *tab;                   // their FP32 table [n_tint][n_ant][n_fint] x (1 | 2)
    int n_fint;
    const uint8_t *active;               // [bins]
    const int *n_active;
    double *acc;                         // [bins][n_ant][KG] (written)
};

} // namespace qc
