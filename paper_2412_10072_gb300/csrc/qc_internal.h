// qc_internal.h -- the context behind the opaque qc_ctx handle of qc.h.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/qc.h"
#include "qc_stream.cuh"
#include "qc_delay.cuh"
#include "qc_stream_delay.cuh"
#include "qc_dd_stream.cuh"
#include "qc_ws.cuh"
#include "qc_robust.cuh"
#include "qc_moments.cuh"

// Every device allocation of the library goes through these two calls.  They count the
// live allocations and honour the test hook of qc_test_fail_alloc (qc.h), so that tests can
// make an allocation fail on the host and check that nothing leaks.
cudaError_t qc_dev_malloc(void **p, size_t bytes);
void qc_dev_free(void *p);
// Bounded-wait settings of the pipelined kernels (qc_test_wait_limit in qc.h): the wall-time
// limit of each wait and, for tests, a ring stage whose copies are never issued.
uint64_t qc_wait_limit_ns();
int qc_wait_stall_stage();

namespace qc {
// Chains with direction-dependent terms (qc_dd.cu).
struct DDArgs {
    Data D;                  // model is [n_row][n_chan][n_dir] x 2 float4
    const float4 *wf;        // [n_row][n_chan] weights with flags folded in
    const uint8_t *row_live; // [n_row]
    int n_dir;
    Chain C;                 // C.n: the solved term (-1 for the residual)
    int nd[MAXT];            // directions in term j's table (1: direction-independent)
    int dd_solved;           // the solved term is direction-dependent (grid dimension y: direction)
    double *acc;             // [bins][n_ant * nd[n]][KG]
    const uint8_t *active;   // [bins]
    const int *n_active;     // nonzero: some interval still iterating
    float4 *resid;           // residual: [n_row][n_chan] x 2, or null
    double *chi2;            // residual: one double (accumulated)
};
} // namespace qc
cudaError_t dd_launch_acc(const qc::DDArgs &a, int ts, int grid_x, cudaStream_t st);
// Single-term chains from per-(interval, baseline) sums (qc_moments.cu).
cudaError_t mom_launch_pass(const qc::MomArgs &a, int form, int ok, int sm_count, cudaStream_t st);
cudaError_t mom_launch_normal(const qc::MomNormArgs &a, cudaStream_t st);
cudaError_t mom_launch_bytes(int n_bins, const long long *bin_nbytes, long long per_iter, long long *iter_nbytes,
                             unsigned long long *acc_bytes, cudaStream_t st);
cudaError_t mom_launch_rows(long n, const int *strip_rows, const int4 *rows, const uint8_t *row_live,
                            const int *up_of_bl, int4 *out, cudaStream_t st);
size_t mom_words(int form);
cudaError_t dd_launch_residual(const qc::DDArgs &a, int grid, cudaStream_t st);

struct Buf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Device buffers of one chain position, reused across calls while large enough.
struct TermBufs {
    // per-bin sample counts (Buf nvis) are a function of the term's maps and of the context's
    // flags, which are fixed for its lifetime: kept while the maps are unchanged
    uint64_t count_sig = 0;
    const void *count_buf = nullptr;
    Buf maps;      // t_map then f_map (int32)
    std::vector<int> hmaps;   // host copy of the maps (staging for the upload)
    Buf tab;       // FP32 kernel table of the term's Jones matrices
    Buf params;    // FP64 master copy of the term's parameters
    Buf stage;     // gains in the public layout (host staging / conversion)
    Buf acc;       // FP64 normal-equation accumulators [bins][ant][KG]
    Buf active;    // uint8 [bins]
    Buf cnt;       // int [max_iter + 1]: intervals active entering iteration k
    Buf nvis;      // int64 [3][bins]: samples, unflagged samples, algorithmic bytes
    Buf iters;     // int [bins]
    Buf flags;     // int8 [bins][ant]
    Buf chunk_act; // uint8 [n_tint][n_chunks] for the pipelined kernel
    Buf row_info;  // int4 [n_row] {p, q, tn, to} for the pipelined kernel
    Buf chunk_info;// int4 [n_chunks] Jones slice ranges of the 32-channel chunks
    Buf rt;        // int4 [n_row] step-major row table of the streaming kernel
    Buf rt_scale;  // float [n_row] its FP16 model scales
    Buf fmap2;     // int2 [n_chan] {f_map of this term, f_map of the other term}
    Buf units;     // int: unit counter of the streaming kernel's strip tiles
    Buf ws_rl;     // warp-specialised kernel, row tiles: int4 [n_row] rows with an active chunk
    Buf ws_rls;    //   float [n_row] their FP16 model scales
    Buf ws_rlb;    //   uint32 [n_row][words] their active-chunk bits
    Buf ws_n;      //   int: number of listed rows
    Buf ws_sb;     // warp-specialised kernel, strip tiles: uint32 [n_chunks][words] active-entry bits
    Buf div;       // divergence flagging: double [bins][ant][2] first / last relative updates
    Buf params0;   // divergence flagging: the FP64 parameters before the solve
    Buf mom;       // single-term chains: FP64 sums per (interval, unordered baseline)
    Buf dfmap;     // delay terms: int [n_chan] parameter interval of each channel
    Buf dfr;       // delay terms: int2 [n_fint] first and last channel of each interval
    Buf dnu;       // delay terms: double [n_chan] channel frequencies
    Buf domega;    // delay terms: float [n_chan] 2 pi nu - omega_ref
    double omega_ref = 0;     // delay terms: 2 pi times the mean channel frequency
    std::vector<int2> hfr;    // host copy of dfr (its size is the term's n_fint)
    std::vector<int> hufmap;  // delay terms: host copy of the term's own f_map
    cudaGraphExec_t exec = nullptr;
    bool graph_valid = false;
};

// One instantiation of the accumulate kernel: its address (for occupancy
// queries) and a launcher.
struct AccLaunch {
    const void *fn = nullptr;        // prefetching accumulate kernel
    cudaError_t (*launch)(int grid, int block, cudaStream_t st, const qc::AccArgs &a) = nullptr;
    int acc_smem_per_warp = 0;       // its dynamic shared memory per warp
    const void *pipe_fn = nullptr;   // pipelined kernel (chains of one or two terms only)
    cudaError_t (*pipe_launch)(int grid, int smem_bytes, cudaStream_t st, const qc::PipeArgs &p) = nullptr;
    int pipe_nw = 0;                 // its warps per CTA
    int pipe_h = 1;                  // row segments per warp step
    const void *stream_fn = nullptr; // streaming kernel (chains of one or two terms only)
    cudaError_t (*stream_launch)(int grid, int block, int smem_bytes, cudaStream_t st, const qc::StreamArgs &a) = nullptr;
    int stream_smem_per_warp = 0;
    const void *ws_fn = nullptr;     // warp-specialised kernel (chains of one or two terms only)
    cudaError_t (*ws_launch)(int grid, int smem_bytes, cudaStream_t st, const qc::WsArgs &a) = nullptr;
    int ws_nc = 0;                   // its consumer warps per CTA
    const void *wss_fn = nullptr;    // self-feeding kernel, row tiles (chains of one or two terms only)
    const void *wss_fn1 = nullptr;   //   ... strip tiles
    cudaError_t (*wss_launch)(int grid, int smem_bytes, cudaStream_t st, const qc::WsArgs &a) = nullptr;
    int wss_nw = 0;                  // its warps per CTA
};
// The streaming kernel of a solved delay term (chains of one or two terms).
struct DelayLaunch {
    const void *fn = nullptr;
    cudaError_t (*launch)(int grid, int block, int smem_bytes, cudaStream_t st, const qc::DelayStreamArgs &a) = nullptr;
    int smem_per_warp = 0;
};
DelayLaunch delay_launcher(int lk, int rk, bool m16);
// The streaming kernel of chains of one or two terms with directions (qc_dd_stream_*.cu):
// gk the solved term's kind, ok the other term's (KIND_NONE: none), oleft the other term is
// to the left of the solved one, dsums a solved delay term with parameter sums, dd the solved
// term is direction-dependent.  dirs_per_cta: directions of a direction-dependent solved term
// whose blocks one CTA forms (grid dimension y covers the rest), 0 otherwise.
struct DDSLaunch {
    const void *fn = nullptr;
    cudaError_t (*launch)(dim3 grid, int block, int smem_bytes, cudaStream_t st, const qc::DDStreamArgs &a) = nullptr;
    int dirs_per_cta = 0;
};
DDSLaunch dds_launcher_diag(int ok, bool oleft);
DDSLaunch dds_launcher_diag_dd(int ok, bool oleft);
DDSLaunch dds_launcher_full(int ok, bool oleft);
DDSLaunch dds_launcher_full_dd(int ok, bool oleft);
DDSLaunch dds_launcher_delay(int ok, bool oleft);
inline DDSLaunch dds_launcher(int gk, int ok, bool oleft, bool dsums, bool dd)
{
    if (dsums) return (gk == qc::KIND_DIAG && !dd) ? dds_launcher_delay(ok, oleft) : DDSLaunch();
    if (gk == qc::KIND_FULL) return dd ? dds_launcher_full_dd(ok, oleft) : dds_launcher_full(ok, oleft);
    return dd ? dds_launcher_diag_dd(ok, oleft) : dds_launcher_diag(ok, oleft);
}
AccLaunch acc_launcher_diag(bool simple, int lk, int rk, bool m16);
AccLaunch acc_launcher_full(bool simple, int lk, int rk, bool m16);
inline AccLaunch acc_launcher(int ts, bool simple, int lk, int rk, bool m16)
{
    return ts == qc::TS_FULL ? acc_launcher_full(simple, lk, rk, m16) : acc_launcher_diag(simple, lk, rk, m16);
}

struct qc_ctx {
    int dev = 0, sm_count = 1, smem_optin = 0, smem_per_sm = 0;
    cudaStream_t own_stream = nullptr;
    int n_row = 0, n_chan = 0, n_ant = 0, n_time = 0, n_bl = 0, n_strips = 0;
    int n_dir = 1;                    // directions of the model (Eq. baselinemodel)
    long n_strip_rows = 0;            // rows in the baseline strips (cross-correlations)
    int max_strip_rows = 0;           // rows of the longest strip
    bool m16 = false, has_flag = false;
    const float4 *d_vis = nullptr, *d_model = nullptr, *d_weight = nullptr;
    const uint8_t *d_flag = nullptr;
    const uint4 *d_model16 = nullptr;
    const float *d_bl_scale = nullptr;
    int4 *d_rows = nullptr;
    int *d_strip_rows = nullptr, *d_strip_off = nullptr;
    int n_up = 0;                     // unordered antenna pairs with cross-correlation rows
    int *d_up_of_bl = nullptr;        // [ordered baseline] -> unordered pair
    int *d_upair = nullptr;           // [n_ant][n_ant] -> unordered pair or -1
    uint8_t *d_row_live = nullptr;    // [n_row]
    const float4 *d_wf = nullptr;     // [n_row][n_chan] weights with flags folded in (streaming kernel)
    const float4 *d_weight_use = nullptr;   // robust reweighting: the weights every kernel reads (d_wf)
    Buf rob_w0;                       // robust reweighting: the folded weights before reweighting
    Buf rob_lam;                      //   float [n_row][n_chan] factors of the last reweighting
    Buf rob_res;                      //   residual of the current chain
    Buf rob_sums;                     //   double [4]: M-step sums, chi^2 scratch
    int *d_err = nullptr;             // device error flag of bounded waits
    std::vector<void *> owned;
    std::vector<cudaEvent_t> events;
    TermBufs tb[QC_MAX_TERMS];
    Buf scalars;                      // counters and chi^2 scratch
    Buf mad_keys;                     // MAD flagging: uint32 [n_vis] statistic keys
    Buf mad_hist;                     // MAD flagging: uint32 [256] histogram + counters
    Buf mad_out;                      // MAD flagging: uint8 [n_vis] flags (host output staging)
    Buf mad_groups;                   // MAD flagging, per-baseline mode: group offsets, then rows
    Buf resid_stage;
    long long launches = 0;
    std::vector<const void *> configured_fns;   // kernels whose dynamic smem limit was raised
    std::string err;

    ~qc_ctx();
    int fail(int code, const std::string &msg);
    int cuda_fail(cudaError_t e, const char *what);
    void *alloc(size_t bytes, cudaError_t *e);
    void release(void *p);
    int ensure(Buf &b, size_t bytes);
    int get_event(int i, cudaEvent_t &ev);
    bool configured(const void *fn) const;
    int validate_terms(const qc_term *terms, int n_terms, bool need_solve_fields);
    // delay terms of the current call (by chain position) and the view the kernels work on:
    // a diagonal term with one bin per (time interval, channel) and the identity channel map
    bool delay[QC_MAX_TERMS] = {};
    // directions in a term's tables: N_D for a direction-dependent term, else 1; such a term
    // is stored over n_ant * N_D (antenna, direction) pairs
    int term_nd(const qc_term &t) const { return (t.dd && n_dir > 1) ? n_dir : 1; }
    int term_nat(const qc_term &t) const { return n_ant * term_nd(t); }
    int cur_nd[QC_MAX_TERMS] = {1, 1, 1, 1};   // term_nd of the chain staged by the current call
    std::vector<int> fid;             // identity channel map [n_chan]
    int expand_terms(const qc_term *terms, int n_terms, std::vector<qc_term> &xt, cudaStream_t st);
    qc::DelayArgs delay_args(int j, const qc_term &xt_j);
    int stage_terms(const qc_term *terms, int n_terms, cudaStream_t st, qc::Chain &chain);
    qc::Data data_desc() const;
    int run_residual(const qc::Chain &chain, float4 *dres, double *d_chi2, cudaStream_t st);
    int pick_order(const qc_term &t, const qc_opts *o) const;
    int solve_term(const qc_term *terms, int n_terms, int n, qc::Chain chain, const qc_opts *o, cudaStream_t st,
                   int *it_max, double *acc_ms, long long *acc_launches, double *pass_ms);
};
