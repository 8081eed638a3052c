/*
 * qc.h -- C ABI of the GB300 gain-calibration solver (libqc.so).
 *
 * The library solves, per solution interval, for per-antenna Jones gains of
 * a chain of gain terms with the approximate ("AllJones") Gauss-Newton
 * method of arxiv 2412.10072 (QuartiCal), Sections 2.2-2.4 and Algorithm 1
 * (Section 4.3).  Every step of an iteration runs in hand-written sm_103a
 * CUDA kernels; nothing is computed on the host.
 *
 * Conventions shared by all entry points
 * ---------------------------------------
 *  - Visibilities, model visibilities and weights are laid out
 *    [n_row][n_chan][4]: rows are the Measurement-Set rows (one time and one
 *    baseline each, Section 4.1), the four correlations of a 2x2 matrix are
 *    in row-major order XX XY YX YY (Eq. gvec, Eq. jones).  Complex values
 *    are complex64: interleaved (re, im) float32 pairs.
 *  - Gains of one term are [n_tint][n_fint][n_ant][4] complex64 (the
 *    paper's (gain_time, gain_freq, antenna, correlation) layout of
 *    Fig. xarray_dataset, one direction); a diagonal term ignores XY/YX and
 *    writes them as 0.  Phase-only terms use float32 [n_tint][n_fint][n_ant][2]
 *    holding (phi_X, phi_Y) in radians (Scenario 1 of Section 2.4).  Delay
 *    terms use float32 [n_tint][n_fint][n_ant][4] holding (phi_X, tau_X,
 *    phi_Y, tau_Y): the diagonal gain of correlation c at the frequency nu of
 *    a channel is exp(i (phi_c + 2 pi tau_c nu)), so the gain changes from
 *    channel to channel while its parameters are shared by every sample of a
 *    solution interval (Scenario 2 of Section 2.4; the residual delay and
 *    phase term K of Section 5.1).
 *  - t_map [n_time] and f_map [n_chan] map each data time / channel to the
 *    term's solution interval (Section 4.3: "interval mappings").  Values
 *    must lie in [0, n_tint) / [0, n_fint) and f_map must be non-decreasing
 *    (intervals are contiguous sample ranges, Section 2.2).
 *  - Ownership: the caller owns every array it passes.  Host inputs are
 *    copied at qc_create; device inputs (memory = QC_MEM_DEVICE) are
 *    borrowed and must stay valid and unchanged until qc_destroy.
 *  - Errors: every call returns QC_OK (0) or a negative status; nothing
 *    aborts.  The message of the last failure of a context is available
 *    from qc_last_error.  A context is not thread-safe: one per thread.
 *  - Only device 0 of the calling thread's current device is used; kernels
 *    run on the stream given in the options (NULL: the context's own
 *    stream).
 */
#ifndef QC_H
#define QC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QC_OK             0
#define QC_EINVAL        -1   /* invalid argument (sizes, indices, maps, NULL pointers)      */
#define QC_ENOMEM        -2   /* device or host allocation failed                            */
#define QC_ECUDA         -3   /* a CUDA runtime call or kernel launch failed                 */
#define QC_ETIMEOUT      -4   /* a bounded device wait gave up (2 s); the context stays usable */
#define QC_EUNSUPPORTED  -5   /* valid request outside what this library implements         */

#define QC_TERM_DIAG   0      /* diagonal complex gain, free parameters g_XX, g_YY           */
#define QC_TERM_FULL   1      /* full 2x2 complex gain, free parameters all four entries     */
#define QC_TERM_PHASE  2      /* phase-only diagonal gain exp(i phi_X), exp(i phi_Y)         */
#define QC_TERM_DELAY  3      /* delay and phase: exp(i (phi_c + 2 pi tau_c nu)) per channel */

#define QC_MEM_HOST    0
#define QC_MEM_DEVICE  1

#define QC_MAX_TERMS   4      /* longest Jones chain accepted                                 */

#define QC_DAMP_CONST      0  /* step length alpha_k = damping for every iteration           */
#define QC_DAMP_ALTERNATE  1  /* alpha_k = 1 on odd, 1/2 on even iterations (k from 1)       */

typedef struct qc_ctx qc_ctx;

/*
 * One calibration problem: the inputs d, m, w of Algorithm 1 plus flags and
 * the row metadata of Section 4.1.
 *   n_row, n_chan, n_time : data sizes; n_corr must be 4.
 *   n_dir                 : directions N_D of the model (Eq. baselinemodel),
 *                           1..QC_MAX_DIRS; with N_D > 1 the model holds one
 *                           set of visibilities per direction (see below).
 *   n_ant                 : antennas; ant1/ant2 in [0, n_ant).
 *   data                  : complex64 [n_row][n_chan][4].
 *   model                 : complex64 [n_row][n_chan][n_dir][4] (the usual
 *                           [n_row][n_chan][4] when n_dir = 1).
 *   weight                : float32 [n_row][n_chan][4], >= 0, per correlation.
 *   flag                  : uint8 [n_row][n_chan], nonzero = flagged, or NULL.
 *   ant1, ant2, time_idx  : int32 [n_row], HOST pointers always; rows with
 *                           ant1 == ant2 (autocorrelations) are ignored.
 *   memory                : where data/model/weight/flag live.
 *   model_fp16            : 1 = store the model on the device as float16
 *                           (re, im) pairs scaled by a per-baseline float32
 *                           factor (max |component| of that baseline) and
 *                           accumulate with compensated float32 sums
 *                           (n_dir = 1 only).
 * Directions (n_dir > 1): the model visibility of a sample is
 * V_pq = sum_d C_{p,d} M_{pq,d} C_{q,d}^H (Eq. baselinemodel), where each
 * chain term is direction-dependent (qc_term.dd = 1: its own gains per
 * direction, Eq. g_derivative_dd) or direction-independent (the same gains in
 * every direction, Eq. g_derivative_di).  Chains with directions take
 * diagonal and full terms, either kind, and direction-independent delay
 * terms (QC_EUNSUPPORTED for phase-only terms, direction-dependent delay
 * terms, qc_mad_flag and qc_delay_init), and a solved direction-independent
 * term must not have a direction-dependent term to its left
 * (QC_EUNSUPPORTED otherwise; its Jacobian is then L_p (x) (sum_d X_d)^T).
 */
#define QC_MAX_DIRS    64
typedef struct {
    int32_t n_row, n_chan, n_corr, n_ant, n_dir, n_time;
    const void *data;
    const void *model;
    const float *weight;
    const uint8_t *flag;
    const int32_t *ant1, *ant2, *time_idx;
    int32_t memory;
    int32_t model_fp16;
} qc_problem;

/*
 * One term of the Jones chain C_a = prod_j G_{j,a} (Eq. joneschain), listed
 * leftmost first.
 *   gains       : in/out, layout above; read as the initial estimate g_0 of
 *                 Algorithm 1 and, for a solved term, overwritten on QC_OK.
 *   gain_flags  : out int8 [n_tint][n_fint][n_ant] or NULL: 1 where the
 *                 block had no data or was singular (the gain is then left
 *                 unchanged), else 0.
 *   iters       : out int32 [n_tint][n_fint] or NULL: iterations of the
 *                 last solve of this term (last epoch).
 *   solve       : 0 = hold fixed, 1 = solve.
 *   max_iter    : N_max of Algorithm 1 (>= 1 when solved).
 *   tol         : epsilon of Algorithm 1: an interval stops once
 *                 ||g_k - g_{k-1}||_F / ||g_k||_F < tol (FP64 norms).
 *   memory      : where gains, gain_flags and iters live.
 *   reduce      : 1 = the term's intervals span several processes; the
 *                 partial normal equations are summed with the options'
 *                 allreduce callback before every update.  The buffer holds
 *                 sums over samples per (interval, antenna): the JHJ block
 *                 and the right-hand side, as J^H W r, or as J^H W d when the
 *                 streaming kernel formed it (the update then takes
 *                 J^H W r = J^H W d - JHJ g); the callback sums every word.
 *   chan_freq   : QC_TERM_DELAY only (NULL otherwise): HOST float64 [n_chan],
 *                 the frequency of every channel, finite, in a unit of the
 *                 caller's choice; tau is in the inverse unit (GHz and ns keep
 *                 the 4x4 normal-equation blocks well conditioned; with Hz the
 *                 tau columns are ~1e9 times the phi columns and every block
 *                 fails the conditioning test).  A delay term's 4x4 real block
 *                 over (phi_X, tau_X, phi_Y, tau_Y) sums 2 Re(E^H W E) over
 *                 every sample of the interval (Eq. jhj_case2, Eq. jhwr_case2);
 *                 convergence uses the gains over the interval's channels.
 *                 Delay terms are accepted by qc_solve and qc_residual.  A
 *                 solved delay term in a chain of one or two terms (kernel 0
 *                 or 3) has its own streaming kernel, which applies the chain
 *                 rule per sample; otherwise the accumulate kernels form
 *                 diagonal blocks per (time interval, channel) bin and the
 *                 update reduces them over the interval's channels.
 *   dd          : 1 = direction-dependent: with n_dir > 1 the gains (and
 *                 gain_flags) carry a direction axis after the antenna axis,
 *                 [n_tint][n_fint][n_ant][n_dir][4] ([..][n_ant][n_dir] for the
 *                 flags), and the AllJones blocks are per (interval, antenna,
 *                 direction) (Eq. g_derivative_dd).  0 = direction-independent.
 *                 Ignored when n_dir = 1.
 */
typedef struct {
    int32_t type, n_tint, n_fint;
    const int32_t *t_map;
    const int32_t *f_map;
    void *gains;
    int8_t *gain_flags;
    int32_t *iters;
    int32_t solve, max_iter;
    double tol;
    int32_t memory;
    int32_t reduce;
    const double *chan_freq;
    int32_t dd;
} qc_term;

/*
 * Sum `n` doubles of a device buffer across processes in place, ordered on
 * `stream` (for example an NCCL all-reduce).  Return 0 on success.
 */
typedef int (*qc_allreduce_fn)(double *device_buffer, int64_t n, void *stream, void *user);

typedef struct {
    int32_t n_epochs;          /* passes over the chain (Section 4.3); >= 1        */
    int32_t damping_mode;      /* QC_DAMP_CONST or QC_DAMP_ALTERNATE               */
    double damping;            /* alpha for QC_DAMP_CONST (0 -> 1.0)               */
    void *stream;              /* cudaStream_t, or NULL for the context stream     */
    int32_t use_graph;         /* 1 = replay each term's iterations as a CUDA graph */
    int32_t want_chi2;         /* 1 = fill chi2_before / chi2_after                 */
    int32_t order;             /* -1 auto, 0 row-major tiles, 1 baseline-strip tiles */
    int32_t block_threads;     /* threads per CTA of the accumulate kernel (0: auto) */
    int32_t ctas_per_sm;       /* resident CTAs per SM for its grid (0: auto)        */
    int32_t kernel;            /* accumulate kernel: 0 auto (3 for chains of <= 2 terms,
                                  2 otherwise), 1 bulk-copy pipeline with per-warp rings
                                  (chains of <= 2 terms), 2 per-lane cp.async prefetching
                                  kernel, 3 streaming kernel (step-major row table, flags
                                  folded into weights; chains of <= 2 terms), 4 warp-
                                  specialised kernel (a producer warp per CTA issues
                                  cp.async.bulk copies into its consumer warps' rings),
                                  5 self-feeding bulk-copy kernel (each warp refills its
                                  own ring with cp.async.bulk; bookkeeping once per run of
                                  steps with unchanged bins).  Kernels 4 and 5 take chains
                                  of <= 2 terms; a solved delay term uses its streaming
                                  kernel under them. */
    qc_allreduce_fn allreduce; /* required when a solved term has reduce = 1       */
    void *allreduce_user;
    int32_t div_flag;          /* 1 = flag diverging gains (see below)              */
    int32_t robust;            /* 1 = robust reweighting between epochs (below)     */
    double robust_nu;          /* its degrees of freedom nu (> 0; 0 -> 5)           */
    int32_t moments;           /* 1 = single-term chains from per-baseline sums (below) */
} qc_opts;

/*
 * Sufficient statistics (not in the paper), opt-in with qc_opts.moments.  While one
 * term is solved the other terms are fixed, so every sample of a baseline (p, q) in a
 * solution interval enters Eq. jhj_entry_simplified and Eq. jhr_entry_simplified
 * through sums that do not depend on the solved gains.  One pass over the data per
 * term solve forms them per (interval, antenna pair); every iteration forms the blocks
 * from the sums and the current gains.  Two forms (chains of one or two terms, one
 * direction, complex64 model, the solved term not a delay term):
 *  - full form, the solved term (any kind) has no term to its left: with
 *    X = R_p M R_q^H (R the term to its right, X = M without one), per correlation kj
 *    S[kj][u][v] = sum w_kj conj(X_u) X_v, T[kj][u] = sum w_kj conj(X_u) D_kj,
 *    U[kj] = sum w_kj |D_kj|^2 (100 FP32 words per interval and pair);
 *  - diagonal form, a diagonal or phase-only solved term with a term L to its left:
 *    with E_kj,ab = L_p,ka M_ab conj(L_q,jb), S'[u][v] = sum sum_kj w_kj conj(E_kj,u)
 *    E_kj,v, T'[u] = sum sum_kj w_kj conj(E_kj,u) D_kj (28 FP32 words per interval and pair).
 * Other solves (a full-Jones term with a term to its left, longer chains, sums of 2^31
 * or more slots) ignore the option.  qc_stats.vis_iters counts the samples of the
 * active intervals per iteration as without it; qc_stats.acc_bytes counts the pass (the
 * samples' bytes, once) and, per iteration and active interval, the sums read on both
 * sides and the accumulators written; qc_stats.pass_ms the passes' device time.
 */

/*
 * Gain flagging on divergence (Section 4.3, "Gain flagging": gains whose updates
 * do not tend to zero), opt-in with qc_opts.div_flag, for diagonal, full and
 * phase-only terms solved with max_iter = K >= 4: the relative update of antenna
 * a in an interval at iteration k is d_a(k) = ||g_a(k) - g_a(k-1)||_F / ||g_a(k)||_F
 * (FP64).  An interval that ends at K without converging flags every antenna with
 * max(d_a(K-1), d_a(K)) >= 0.9 max(d_a(1), d_a(2)) > 0 (its updates have not shrunk
 * by more than a tenth): its gain flag becomes 2 and its gain is restored to its
 * value before that term's solve in this epoch.
 *
 * Robust reweighting (Section 4.3, "Robust reweighting", after Sob et al. 2020),
 * opt-in with qc_opts.robust and n_epochs >= 2: the noise is read as complex
 * Student's t with nu degrees of freedom, a scale mixture of complex Gaussians,
 * and between epochs one expectation-maximisation step reweights every sample s
 * from the residual r of the current chain: z_s = sum_c w_c |r_c|^2 over its k_s
 * correlations with w_c > 0 (w the caller's weights, flags applied),
 * sigma^2 = sum_s lambda_s z_s / sum_s k_s (previous factors; 1 at first),
 * lambda_s = (nu + 2 k_s) / (nu + 2 z_s / sigma^2), and the next epoch solves with
 * weights w_c lambda_s.  The caller's weights are unchanged on return;
 * chi2_before / chi2_after use them.
 */

typedef struct {
    double chi2_before, chi2_after;   /* Eq. min, FP64 sums (when want_chi2)           */
    double ms;                        /* device time of the whole solve (CUDA events)  */
    double acc_ms;                    /* device time inside the accumulate kernels     */
    int64_t vis_iters;                /* sum over iterations of samples in active intervals */
    int64_t acc_bytes;                /* algorithmic bytes read by the accumulate kernels */
    int64_t acc_launches;             /* accumulate kernels that did work              */
    int64_t launches;                 /* kernels launched by this call                 */
    int32_t n_iter_max;               /* largest iteration count of any interval       */
    double pass_ms;                   /* device time of the sums passes (qc_opts.moments;
                                         included in acc_ms), else 0                    */
} qc_stats;

/*
 * Validate a problem and stage it on the device.  On QC_OK *out holds a new
 * context (release with qc_destroy); on failure *out is NULL and the status
 * says why (QC_EINVAL for bad sizes/indices, QC_ENOMEM, QC_ECUDA).
 */
int qc_create(const qc_problem *p, qc_ctx **out);

/*
 * Run the chain schedule: for each epoch, each solved term in chain order
 * is iterated with Algorithm 1 until every one of its solution intervals
 * has converged or reached max_iter (Section 4.3).  One iteration forms the
 * corrected-model residual over every baseline and accumulates the
 * per-antenna blocks of J^H W J and J^H W r of the term (Eq.
 * jhj_entry_simplified, Eq. jhr_entry_simplified, or the 2 Re(.) forms of
 * Scenario 1 for phase terms) in one data pass, then solves each block in
 * FP64 and updates g <- g + alpha_k JHJ^{-1} JHr (Eq. update, Algorithm 1).
 * `stats` may be NULL.  Gains, flags and iteration counts are written back
 * only on QC_OK.
 */
int qc_solve(qc_ctx *c, qc_term *terms, int32_t n_terms, const qc_opts *o, qc_stats *stats);

/*
 * chi^2 = sum of w |d - C_p M C_q^H|^2 over unflagged cross-correlation
 * samples and correlations (Eq. min, Eq. baselineresidual), accumulated in
 * FP64.  If `resid` is not NULL the residual r is written as complex64
 * [n_row][n_chan][4] (zero for flagged samples and autocorrelations) in
 * `resid_memory`.
 */
int qc_residual(qc_ctx *c, const qc_term *terms, int32_t n_terms, void *resid, int32_t resid_memory,
                double *chi2);

/*
 * Initial estimate of a delay term's parameters (Section 4.3, "Initial
 * estimates": the peak of the Fourier transform along frequency of the
 * baselines that include the reference antenna).  For every time interval,
 * frequency interval, antenna a and correlation c in {XX, YY}:
 *   x(nu) = sum of w d conj(m) of correlation c over the interval's unflagged
 *           samples on baselines (a, ref) or (ref, a), conjugated for (ref, a);
 *   X_k   = FFT of x over the interval's channels zero-padded to N, the next
 *           power of two >= oversample x channels, at the delays
 *           tau_k = k / (N dnu), k = -N/2 .. N/2 - 1;
 *   tau_c = tau_k and phi_c = arg X_k - 2 pi tau_k nu_0 at the largest |X_k|
 *           (the lowest k among equal values), nu_0 the interval's first channel.
 * The reference antenna, antennas without data and one-channel intervals get
 * tau = 0 (one channel: phi = arg x).  term->gains (float32 [n_tint][n_fint]
 * [n_ant][4], in term->memory) is overwritten; term->solve is ignored.
 *   ref_ant    : reference antenna, in [0, n_ant).
 *   oversample : >= 1 (0: 4); N must not exceed 16384.
 * Errors: QC_EINVAL for a term that is not QC_TERM_DELAY or fails the checks
 * of qc_solve, a reference antenna out of range or oversample < 0;
 * QC_EUNSUPPORTED when an interval's channels are not uniformly spaced
 * (|nu_c - nu_0 - c dnu| > 1e-6 |dnu|) or N would exceed 16384.
 */
int qc_delay_init(qc_ctx *c, qc_term *term, int32_t ref_ant, int32_t oversample);

/*
 * MAD residual flagging after calibration (Section 4, "Additional features":
 * outliers of the residual visibilities by the Median Absolute Deviation,
 * over all baselines at once or per baseline).  With the chain `terms` (as in qc_residual):
 *   z_s   = sqrt(sum over the 4 correlations of w |r|^2) of every unflagged
 *           cross-correlation sample s, in float32, every operation rounded
 *           (no fused multiply-add), in the order ((w0 t0 + w1 t1) + w2 t2)
 *           + w3 t3 with t_c = re^2 + im^2;
 *   med   = the floor((n - 1) / 2)-th smallest z (exact order statistic);
 *   MAD   = the same order statistic of |z - med|;
 *   flag s when |z_s - med| > fl32(threshold * 1.4826) * MAD (float32).
 *   per_baseline : 0 = med and MAD over all baselines (global mode); 1 = over
 *               the samples of each baseline (its rows in either orientation
 *               and all channels) separately (the paper's per-baseline mode).
 *   flags_out : out uint8 [n_row][n_chan] in out_memory: 1 = outlier, 0 else
 *               (samples already flagged and autocorrelations are 0; the
 *               caller merges them with its own flags).
 *   n_flagged : out (nullable), number of samples set to 1.
 * Errors: QC_EINVAL for NULL flags_out, threshold not positive and finite, or
 * terms failing the checks of qc_residual.
 */
int qc_mad_flag(qc_ctx *c, const qc_term *terms, int32_t n_terms, double threshold, int32_t per_baseline,
                uint8_t *flags_out, int32_t out_memory, int64_t *n_flagged);

/* Release a context and every device buffer it owns.  NULL-safe. */
void qc_destroy(qc_ctx *c);

/*
 * chi^2 of a one-term problem without allocating anything (the paper has no
 * counterpart: this serves callers that must not allocate device memory, such
 * as real-time pipelines whose device memory is reserved up front, or host
 * frameworks that own every device buffer through their own pool).
 *
 * Computes the same chi^2 as qc_residual for a chain of a single term (type,
 * n_tint, n_fint, t_map, f_map, gains as in qc_term), with every argument in
 * DEVICE memory: data/model complex64 [n_row][n_chan][4] and weight float32
 * [n_row][n_chan][4] (16-byte aligned), flag uint8 [n_row][n_chan] or NULL,
 * ant1/ant2/time_idx int32 [n_row], t_map [n_time], f_map [n_chan], gains in the
 * qc_term layout, and the result written to *chi2 (one device double, FP64
 * sum in a fixed order).  Kernels are enqueued on `stream` (NULL: the legacy
 * default stream); the call returns without synchronising.
 *
 * Index checks: the index arrays are in device memory, so the host cannot read
 * them.  The kernel checks every index before it uses it: ant1/ant2 in
 * [0, n_ant), time_idx in [0, n_time), t_map values in [0, n_tint) and f_map
 * values in [0, n_fint).  A sample with an index out of range is skipped
 * (nothing is read through that index) and the call's result is NaN; the
 * return code is still QC_OK, since the check runs on the GPU after the call
 * returns.  Sizes are checked on the host (QC_EINVAL).
 *
 * Scratch: the kernel-layout gain table, the per-CTA partial sums and the
 * index-check word live in a static device array of
 * (QC_NOALLOC_MAX_GAINS * 32 + QC_NOALLOC_MAX_BLOCKS * 8 + 256) bytes
 * (about 2 MiB + 8 KiB) that every device which loads the library keeps until
 * the process exits.  Problems with n_tint * n_fint * n_ant > QC_NOALLOC_MAX_GAINS
 * are rejected with QC_EINVAL (message in qc_last_error(NULL)).  The first call
 * on a device looks up the device address of that array (cudaGetSymbolAddress,
 * no allocation); make that first call before capturing a stream into a CUDA
 * graph.  Every call reuses the same array and leaves its contents behind
 * (the index-check word is cleared at the start of each call):
 * calls on one device whose kernels may overlap (for example on two streams)
 * race on it, so order them (one stream, or events).  Each device has its own
 * copy, so calls on different devices do not interfere.
 */
#define QC_NOALLOC_MAX_GAINS   65536
#define QC_NOALLOC_MAX_BLOCKS  1024
int qc_residual_noalloc(int32_t n_row, int32_t n_chan, int32_t n_ant, int32_t n_time, const void *data,
                        const void *model, const float *weight, const uint8_t *flag, const int32_t *ant1,
                        const int32_t *ant2, const int32_t *time_idx, int32_t type, int32_t n_tint, int32_t n_fint,
                        const int32_t *t_map, const int32_t *f_map, const void *gains, double *chi2, void *stream);

/*
 * Test hooks (the paper has no counterpart).  Failure paths are exercised
 * without faulting the GPU: the failure is made on the host, or a bounded
 * wait is made to run out.  Process-wide; not for production use.
 *   qc_test_fail_alloc(n): the n-th device allocation of the library from now
 *       on (1-based) fails as if cudaMalloc had returned
 *       cudaErrorMemoryAllocation, without calling it; the call that made it
 *       returns QC_ENOMEM and releases what it had allocated.  n <= 0 disarms.
 *   qc_test_live_allocs(): device allocations of the library not yet freed
 *       (contexts, batches and their temporary buffers).
 *   qc_test_wait_limit(limit_ns, stall): wall-time limit of each bounded wait
 *       on a ring-stage barrier of the bulk-copy accumulate kernels (default
 *       2 s; limit_ns <= 0 restores it).  With stall >= 0, every warp's
 *       stall-th stage is never filled and its barrier never completes, so the
 *       kernel's wait on it gives up after limit_ns: the kernel records the
 *       error, waits (bounded) for its copies in flight and returns; qc_solve
 *       returns QC_ETIMEOUT and the context stays usable.  stall < 0 disarms.
 *       While a stall is armed, qc_solve does not use CUDA graphs.
 */
void qc_test_fail_alloc(int64_t n);
int64_t qc_test_live_allocs(void);
void qc_test_wait_limit(int64_t limit_ns, int32_t stall);

/* Message of the last failed call on `c` ("" if none); with c == NULL, of the last failed qc_create. */
const char *qc_last_error(const qc_ctx *c);

/* Library version string. */
const char *qc_version(void);


/* ------------------------------------------------------------------------ */
/* Batched solves of many independent solution intervals                     */
/* ------------------------------------------------------------------------ */

/*
 * A batch of independent calibration problems, each one solution interval
 * of one diagonal complex gain term (Section 2.3, last paragraph: solution
 * intervals are solved independently of each other).  Problem i owns rows
 * [row_offset[i], row_offset[i+1]) and samples [vis_offset[i], vis_offset[i+1])
 * of the concatenated arrays, laid out [row][chan][4] with its own channel
 * count n_chan[i] (so vis_offset[i+1] - vis_offset[i] = rows_i * n_chan[i]),
 * and n_ant[i] antennas; ant1/ant2 are antenna indices local to the problem.
 *   data, model : complex64; weight: float32 (per correlation); flag: uint8
 *                 per sample or NULL; all in `memory`.
 *   row_offset, vis_offset, n_chan, n_ant, ant1, ant2 : HOST arrays.
 *   model_fp16  : as in qc_problem (per-baseline scales, compensated sums).
 * Gains of problem i occupy entries [gain_offset_i, gain_offset_i + n_ant[i])
 * of a [sum n_ant][2] complex64 array (g_XX, g_YY), gain_offset_i being the
 * running sum of n_ant.
 */
typedef struct qc_batch qc_batch;

typedef struct {
    int32_t n_prob;
    const int64_t *row_offset;   /* [n_prob + 1] */
    const int64_t *vis_offset;   /* [n_prob + 1] */
    const int32_t *n_chan;       /* [n_prob] */
    const int32_t *n_ant;        /* [n_prob], 2 .. QC_BATCH_MAX_ANT */
    const void *data, *model;
    const float *weight;
    const uint8_t *flag;
    const int32_t *ant1, *ant2;  /* [total rows] */
    int32_t memory;
    int32_t model_fp16;
} qc_batch_problem;

#define QC_BATCH_MAX_ANT 256

#define QC_SCHED_AUTO     0      /* autotuned (or LPT when not tuned)                   */
#define QC_SCHED_LPT      1      /* longest problem first from a shared work counter    */
#define QC_SCHED_STATIC   2      /* problem i -> CTA i mod grid, in index order         */

typedef struct {
    int32_t max_iter;            /* N_max of Algorithm 1                                 */
    double tol;                  /* per-problem relative gain change to stop             */
    int32_t damping_mode;        /* QC_DAMP_CONST or QC_DAMP_ALTERNATE                   */
    double damping;
    void *stream;                /* cudaStream_t or NULL                                 */
    int32_t threads;             /* threads per CTA (0: tuned or 256)                    */
    int32_t ctas_per_sm;         /* resident CTAs per SM (0: tuned or occupancy)          */
    int32_t schedule;            /* QC_SCHED_*                                           */
    int32_t use_graph;           /* 1: replay the persistent launch as a CUDA graph       */
    int32_t depth;               /* copy stages in flight per warp, 3/4/6 (0: tuned or 4)  */
    /* Optional fallback start (device pointers, both or neither): the first pass also
     * sums chi^2 at the given gains, and a problem whose chi^2 there exceeds
     * fallback_chi2[problem] by more than a relative 1e-5 (the rounding of the two
     * sums), or is not finite, restarts from fallback_gains.                       */
    const void *fallback_gains;  /* [sum n_ant][2] complex64                           */
    const double *fallback_chi2; /* [n_prob] chi^2 at fallback_gains                  */
    /* Size classes: with split > 0 the problems with fewer than `split` samples
     * (rows x channels) form a second class, launched concurrently with its own CTA
     * size (the tile: small_threads consecutive samples per CTA step) and residency
     * (LPT schedule for both).  split = 0: tuned, else one class; split < 0: one class. */
    int64_t split;
    int32_t small_threads;       /* threads per CTA of the small class (0: tuned or 64)   */
    int32_t small_ctas_per_sm;   /* its resident CTAs per SM (0: tuned or occupancy)      */
} qc_batch_opts;

typedef struct {
    double ms;                   /* device time of the solve (CUDA events)               */
    int64_t vis_iters;           /* sum over problems of samples x iterations            */
    int64_t bytes;               /* algorithmic bytes read (data passes)                 */
    int32_t n_iter_max;
    double mean_iters;
    int32_t threads, ctas_per_sm, schedule, grid;   /* launch configuration used          */
    int32_t depth;
    int32_t n_fallback;          /* problems restarted from the fallback gains           */
    int64_t split;               /* size threshold used (<= 0: one class)                 */
    int32_t small_threads, small_ctas_per_sm, small_grid, n_small;   /* the small class   */
} qc_batch_stats;

/* Validate and stage a batch (host arrays copied, device arrays borrowed). */
int qc_batch_create(const qc_batch_problem *p, qc_batch **out);

/*
 * Solve every problem of the batch with Algorithm 1 in one persistent
 * kernel launch: each CTA takes whole problems (longest first, or as the
 * schedule says) and iterates them to convergence or max_iter on chip;
 * per iteration it forms the residual of every sample, accumulates the
 * per-antenna diagonal JHJ / JHr blocks (Eq. jhj_entry_simplified,
 * Eq. jhr_entry_simplified) in shared memory and updates the gains with an
 * FP64 block solve (Eq. update).  The CTA's warps stream contiguous runs of
 * 32-sample steps through per-warp rings of `depth` asynchronous-copy stages
 * in shared memory; flagged samples and autocorrelations are not read.
 * A problem never spans CTAs: its time is bounded below by what one SM streams
 * (about 1/152 of the device's bandwidth), so one problem of millions of
 * samples among many small ones sets the launch's duration.  Such problems
 * belong in qc_solve, which spreads an interval's samples over every SM.
 *   gains      : in/out [sum n_ant][2] complex64; read as g_0.
 *   gain_flags : out [sum n_ant] int8 or NULL (1: no data for the antenna).
 *   iters      : out [n_prob] int32 or NULL.
 *   mem        : where gains/gain_flags/iters live (QC_MEM_HOST or DEVICE).
 */
int qc_batch_solve(qc_batch *b, void *gains, int8_t *gain_flags, int32_t *iters, int32_t mem,
                   const qc_batch_opts *o, qc_batch_stats *stats);

/*
 * The same solve from per-baseline sufficient statistics (not in the paper).  A
 * problem is one solution interval of one diagonal term, so the samples of a
 * baseline enter JHJ and JHr (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified)
 * only through S_c = sum w_c |m_c|^2 and T_c = sum w_c conj(m_c) d_c per
 * correlation, and chi^2 (Eq. min) through them and U = sum_c w_c |d_c|^2.  One
 * pass over the samples forms them (float32 sums in shared memory); the
 * iterations then form the normal equations from them, with the update and
 * convergence test of qc_batch_solve.  With a fallback start, chi^2 at the
 * starting and at the fallback gains both come from the sums (fallback_chi2 must
 * be given but is not read) and the rule of qc_batch_opts applies.  Arguments and
 * outputs as qc_batch_solve; stats.bytes counts the one data pass.
 * QC_EUNSUPPORTED for batches with more than 64 antennas in a problem.
 */
int qc_batch_solve_moments(qc_batch *b, void *gains, int8_t *gain_flags, int32_t *iters, int32_t mem,
                           const qc_batch_opts *o, qc_batch_stats *stats);

/*
 * Autotuner: time the batch solve (from unit gains, `base` options, results
 * discarded) for candidate launch shapes and keep the fastest for later solves
 * that leave the shape to it (threads / ctas_per_sm / depth / split /
 * small_* = 0, schedule QC_SCHED_AUTO).  Stage 1, one class: threads per CTA
 * in {128, 256, 512} (the tile: that many consecutive samples per CTA step,
 * threads / n_chan baselines x n_chan channels), copy stages per warp in
 * {3, 4, 6}, resident CTAs per SM in {1, 2, 4} (as shared memory allows),
 * schedule in {LPT, static}.  Stage 2, with the best stage-1 shape for the
 * large problems: a size threshold in {2^10, 2^12, 2^14, 2^16} samples below
 * which problems go to a concurrent class of small CTAs, threads in {64, 128}
 * and {4, 8} per SM.  Results are cached for the process per device and shape
 * class of the batch (problem count, FP16 model, log2 size histogram): another
 * batch of the same class uses them without tuning.  best (nullable) receives
 * the chosen shape and its time; `n_tried` (nullable) the candidates timed.
 */
int qc_batch_autotune(qc_batch *b, const qc_batch_opts *base, qc_batch_stats *best, int32_t *n_tried);

/*
 * Per-problem chi^2 (Eq. min) at the given gains: chi2 [n_prob] FP64, host
 * or device per `mem`.
 */
int qc_batch_residual(qc_batch *b, const void *gains, int32_t mem, double *chi2);

/* Release a batch.  NULL-safe. */
void qc_batch_destroy(qc_batch *b);

/* Message of the last failed call on `b` ("" if none); NULL: last failed qc_batch_create. */
const char *qc_batch_last_error(const qc_batch *b);

/* ------------------------------------------------------------------------ */
/* Learned warm start of the batched solver                                  */
/* ------------------------------------------------------------------------ */

/*
 * Initial estimates (Section 4.3, "Initial estimates"): a multilayer
 * perceptron predicts each interval's diagonal gains from per-antenna
 * features; Algorithm 1 then iterates from them as usual.
 *
 * Network: Linear(10 -> 128) GELU, Linear(128 -> 128) GELU,
 * Linear(128 -> 128) GELU, Linear(128 -> 4), plus a skip connection that adds
 * input features 6..9 (the previous-interval gains) to the 4 outputs, so the
 * layers learn the correction to them; GELU(z) = z (1 + erf(z/sqrt 2))/2.
 * Parameters are one float32 buffer of QC_MLP_NPARAM values: W1 [128][10],
 * b1 [128], W2 [128][128], b2, W3 [128][128], b3, W4 [4][128], b4 (weights
 * row-major [out][in]).  Outputs per antenna: (Re g_XX, Im g_XX, Re g_YY,
 * Im g_YY) in the gauge where the sum of the interval's gains is real and
 * positive per correlation.
 */
#define QC_MLP_IN      10
#define QC_MLP_HIDDEN  128
#define QC_MLP_OUT     4
#define QC_MLP_NPARAM  34948

/*
 * Per-antenna features of every problem of a batch, float32 [sum n_ant][10]
 * (device or host per `mem`), from one data pass at unit gains:
 *   0,1  |z_XX|, |z_YY| with z_k = JHr_k / JHJ_kk, the normalised first
 *        Gauss-Newton step at unit gains (Eq. jhr_entry_simplified)
 *   2,3  arg of the one-step gain 1 + z_k (the first Gauss-Newton iterate from
 *        unit gains), referenced so that the sum of the interval's one-step
 *        gains is real-positive: the phase of the gain in the targets' gauge,
 *        since 1 + z_p ~ g_p conj(weighted mean of g_q)
 *   4,5  mean |d_kk| / |m_kk| over the antenna's unflagged samples
 *   6..9 previous-interval gains (Re, Im of g_XX, g_YY), referenced so that
 *        their sum over the interval's antennas is real-positive; unit gains
 *        when prev_gains is NULL.
 * Antennas without data get zeros for 0..5.  prev_chi2 (nullable, needs
 * prev_gains; same memory as `features`) receives each problem's chi^2 at the
 * previous-interval gains from the same pass: the bound of the fallback check
 * (qc_batch_opts.fallback_chi2).
 */
int qc_batch_features(qc_batch *b, const void *prev_gains, float *features, double *prev_chi2, int32_t mem,
                      void *stream);

/*
 * Initial gains from network outputs y [sum n_ant][4] (device): g = (y0 + i y1,
 * y2 + i y3).  A problem whose outputs are not all finite, or (check_chi2 = 1)
 * whose chi^2 at the predicted gains exceeds its chi^2 at `fallback` (device
 * [sum n_ant][2] complex64: previous-interval or unit gains), starts from
 * `fallback` instead.  gains_out: device [sum n_ant][2] complex64.  n_fallback
 * (nullable, host) receives the number of problems that fell back.
 */
int qc_batch_warmstart(qc_batch *b, const float *y, const void *fallback, int32_t check_chi2, void *gains_out,
                       int32_t *n_fallback, void *stream);

/*
 * Rotate each problem's gains (device [sum n_ant][2] complex64; in place allowed)
 * by the conjugate unit phase of their sum over the problem's antennas, per
 * correlation: the gauge of the network's targets and previous-gain features.
 */
int qc_batch_reference_gains(qc_batch *b, const void *gains_in, void *gains_out, void *stream);

/*
 * Network kernels (device pointers, `stream` may be NULL):
 *   forward  : y [n][4] = net(x [n][10]); z (nullable) [n][3][128] receives the
 *              three hidden pre-activations for the backward pass.
 *   backward : grad [QC_MLP_NPARAM] = d loss / d params and *loss (device
 *              double) = mean over n x 4 of (y - target)^2.
 *   adam     : one Adam step (bias-corrected, step counted from 1).
 */
int qc_mlp_forward(const float *params, const float *x, int64_t n, float *y, float *z, void *stream);
int qc_mlp_backward(const float *params, const float *x, const float *z, const float *y, const float *target,
                    int64_t n, float *grad, double *loss, void *stream);
int qc_mlp_adam(float *params, const float *grad, float *m, float *v, float lr, float beta1, float beta2, float eps,
                int32_t step, void *stream);
const char *qc_mlp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QC_H */
