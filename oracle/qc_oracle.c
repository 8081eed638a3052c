/*
 * qc_oracle.c -- FP64 CPU oracle of the approximate Gauss-Newton ("AllJones")
 * gain solver of arxiv 2412.10072 (QuartiCal), Sections 2.2-2.4 and Algorithm 1 (Section 4.3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the solver computes.  It is used by the tests, by the
 * smoke check and by the CPU-baseline leg of the benchmark, never by the
 * product path, and it shares no code with the CUDA library.
 *
 * Everything is double precision and written as plain loops in the order the
 * paper states the mathematics:
 *   - Jones chain and its factorisation around term n       (Eq. joneschain, Eq. jonesfactor)
 *   - model visibility  V = C_p M C_q^H                     (Eq. baselinemodel)
 *   - residual          r = vec(D) - vec(V)                  (Eq. baselineresidual)
 *   - vec trick         vec(A X B) = (A (x) B^T) vec(X)      (Eq. vectrick)
 *   - derivative        dv/dg_{n,p} = L_p (x) (R_p M C_q^H)^T (Eq. g_derivative_dd)
 *   - per-antenna blocks of J^H W J and J^H W r, summed over all baselines
 *     containing the antenna including conjugate baselines
 *     (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified)
 *   - block update      g <- g + JHJ^{-1} JHr      (Eq. update, Algorithm 1)
 *   - phase-only terms  E = dv/dg dg/dphi, JHJ = 2 Re(E^H W E),
 *                       JHr = 2 Re(E^H W r)   (Scenario 1: Eq. jhj_case1, Eq. jhwr_case1)
 *   - delay terms       gains evaluated per channel from per-interval parameters
 *                       (phi_c, tau_c): g_c(nu) = exp(i (phi_c + 2 pi tau_c nu)); the
 *                       sums run over every sample of the parameter interval
 *                       (Scenario 2: Eq. jhj_case2, Eq. jhwr_case2)
 *   - chi^2 = r^H W r                                        (Eq. min)
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - JHr is the minus-free form of Eq. jhr_entry_simplified and the update
 *     adds the step, as Algorithm 1 writes it (Eq. update_set / Eq. update
 *     subtract because Eq. jacobian_A has J = -dv/dg).
 *   - A diagonal term keeps the complete 2x2 block over its two free
 *     parameters (XX, YY); a full term the 4x4 block; a phase term the 2x2
 *     real block over (phi_X, phi_Y).
 *   - Convergence per solution interval: relative Frobenius change
 *     ||g_k - g_{k-1}|| / ||g_k|| < tol, at most max_iter iterations.
 *   - Damping: step length alpha_k = damping (default 1, the literal
 *     Algorithm 1), or with damping_mode 1 the alternating 1, 1/2, 1, 1/2 ...
 *     averaging of the StefCal iteration.
 *   - A block with zero trace or reciprocal condition number below 1e-12 is
 *     not updated and its gain flag is set.
 *   - Delay terms (the residual delay and phase term K of Section 5.1): two real
 *     parameters per correlation, phi_c and tau_c, ordered (phi_X, tau_X,
 *     phi_Y, tau_Y), a diagonal gain, and a frequency axis nu per channel in
 *     units chosen by the caller (tau in the inverse unit).  Convergence uses
 *     the gains: the relative Frobenius change over the antennas and the
 *     channels of the interval.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { OC_DIAG = 0, OC_FULL = 1, OC_PHASE = 2, OC_DELAY = 3 };
enum { OC_OK = 0, OC_EINVAL = -1, OC_ENOMEM = -2 };

typedef struct {
    int n_row, n_chan, n_ant, n_time;
    const cplx *data;            /* [row][chan][4] */
    const cplx *model;           /* [row][chan][4] */
    const double *weight;        /* [row][chan][4] */
    const unsigned char *flag;   /* [row][chan], nonzero = flagged; may be NULL */
    const int *ant1, *ant2, *time_idx;   /* [row] */
} oc_problem;

typedef struct {
    int type, n_tint, n_fint;
    const int *t_map;            /* [n_time] -> time interval */
    const int *f_map;            /* [n_chan] -> freq interval */
    double *params;              /* DIAG/FULL: complex [tint][fint][ant][4] as (re,im) pairs;
                                    PHASE: real [tint][fint][ant][2];
                                    DELAY: real [tint][fint][ant][4] = (phi_X, tau_X, phi_Y, tau_Y) */
    signed char *gain_flags;     /* [tint][fint][ant], may be NULL */
    int solve, max_iter;
    double tol;
    const double *chan_freq;     /* DELAY: [n_chan] frequency of each channel; else unused */
} oc_term;

typedef struct {
    int n_epochs;
    int damping_mode;            /* 0: constant alpha; 1: alternate 1, 1/2 */
    double damping;              /* alpha for mode 0 */
    int div_flag;                /* 1: flag diverging gains (Section 4.3, "Gain flagging"; see oc_solve_term) */
} oc_opts;

/* ------------------------------------------------------------------------ */
/* 2x2 complex matrices, row-major: A = [[A0, A1], [A2, A3]] (Eq. jones)      */
/* ------------------------------------------------------------------------ */

static void mat_eye(cplx A[4]) { A[0] = 1; A[1] = 0; A[2] = 0; A[3] = 1; }

static void mat_mul(const cplx A[4], const cplx B[4], cplx out[4])
{
    cplx t[4];
    t[0] = A[0] * B[0] + A[1] * B[2];
    t[1] = A[0] * B[1] + A[1] * B[3];
    t[2] = A[2] * B[0] + A[3] * B[2];
    t[3] = A[2] * B[1] + A[3] * B[3];
    memcpy(out, t, sizeof t);
}

static void mat_herm(const cplx A[4], cplx out[4])
{
    cplx t[4] = { conj(A[0]), conj(A[2]), conj(A[1]), conj(A[3]) };
    memcpy(out, t, sizeof t);
}

/* Number of free parameters of a term: 2 (diag, phase) or 4 (full, delay). */
static int n_param(int type) { return (type == OC_FULL || type == OC_DELAY) ? 4 : 2; }

static const double TWO_PI = 6.283185307179586476925286766559;

/* Diagonal gains of a delay term's parameters u at frequency nu. */
static void delay_gains(const double *u, double nu, cplx *gx, cplx *gy)
{
    *gx = cexp(I * (u[0] + TWO_PI * u[1] * nu));
    *gy = cexp(I * (u[2] + TWO_PI * u[3] * nu));
}

static size_t bin_index(const oc_term *T, int it, int jf) { return (size_t)it * T->n_fint + jf; }

/* Jones matrix of term T for antenna a at data time t and channel c (Eq. jones). */
static void term_jones(const oc_term *T, int n_ant, int t, int c, int a, cplx J[4])
{
    size_t b = bin_index(T, T->t_map[t], T->f_map[c]) * n_ant + a;
    if (T->type == OC_PHASE) {
        const double *phi = T->params + 2 * b;
        J[0] = cexp(I * phi[0]); J[1] = 0; J[2] = 0; J[3] = cexp(I * phi[1]);
        return;
    }
    if (T->type == OC_DELAY) {
        delay_gains(T->params + 4 * b, T->chan_freq[c], &J[0], &J[3]);
        J[1] = 0; J[2] = 0;
        return;
    }
    const double *g = T->params + 8 * b;
    J[0] = g[0] + I * g[1];
    J[3] = g[6] + I * g[7];
    if (T->type == OC_FULL) { J[1] = g[2] + I * g[3]; J[2] = g[4] + I * g[5]; }
    else { J[1] = 0; J[2] = 0; }
}

/* Factorisation of the chain of antenna a around term n:  C = L G_n R  (Eq. jonesfactor). */
static void chain_factors(const oc_term *terms, int n_terms, int n, int n_ant,
                          int t, int c, int a, cplx L[4], cplx G[4], cplx R[4])
{
    cplx J[4];
    mat_eye(L); mat_eye(R); mat_eye(G);
    for (int j = 0; j < n_terms; ++j) {
        term_jones(&terms[j], n_ant, t, c, a, J);
        if (j < n) mat_mul(L, J, L);
        else if (j == n) memcpy(G, J, sizeof(cplx) * 4);
        else mat_mul(R, J, R);
    }
}

/* Full chain C_a = prod_j G_{j,a} (Eq. joneschain). */
static void chain_product(const oc_term *terms, int n_terms, int n_ant, int t, int c, int a, cplx C[4])
{
    cplx J[4];
    mat_eye(C);
    for (int j = 0; j < n_terms; ++j) {
        term_jones(&terms[j], n_ant, t, c, a, J);
        mat_mul(C, J, C);
    }
}

/* ------------------------------------------------------------------------ */
/* Normal equations of term n (Eq. jhj_entry_simplified, Eq. jhr_entry_simplified;
 * Scenario 1 for phase terms)                                                 */
/* ------------------------------------------------------------------------ */

/*
 * jhj: complex [n_tint*n_fint][n_ant][np][np], jhr: complex [n_tint*n_fint][n_ant][np],
 * np = n_param(type).  Both are overwritten.  Bins whose `active` entry is 0
 * are skipped (active may be NULL: all bins).
 *
 * Each unflagged sample of a cross-correlation row contributes twice: once
 * for antenna p through baseline pq and once for antenna q through the
 * conjugate baseline qp, for which D, M -> D^H, M^H and the per-correlation
 * weights are permuted by P (Eq. jonesconj, Eq. permutation), i.e.
 * (w0, w2, w1, w3).
 */
int oc_normal_equations(const oc_problem *P, const oc_term *terms, int n_terms, int n,
                        const unsigned char *active, cplx *jhj, cplx *jhr)
{
    if (!P || !terms || n < 0 || n >= n_terms) return OC_EINVAL;
    const oc_term *T = &terms[n];
    const int np = n_param(T->type);
    const size_t n_bins = (size_t)T->n_tint * T->n_fint;
    memset(jhj, 0, sizeof(cplx) * n_bins * P->n_ant * np * np);
    memset(jhr, 0, sizeof(cplx) * n_bins * P->n_ant * np);
    static const int perm[4] = { 0, 2, 1, 3 };
    const int free_cols_diag[2] = { 0, 3 };

    for (int row = 0; row < P->n_row; ++row) {
        const int p = P->ant1[row], q = P->ant2[row], t = P->time_idx[row];
        if (p == q) continue;
        for (int c = 0; c < P->n_chan; ++c) {
            const size_t s = (size_t)row * P->n_chan + c;
            if (P->flag && P->flag[s]) continue;
            const size_t bin = bin_index(T, T->t_map[t], T->f_map[c]);
            if (active && !active[bin]) continue;
            for (int orient = 0; orient < 2; ++orient) {
                const int a = orient == 0 ? p : q;      /* antenna whose block receives the term */
                const int b = orient == 0 ? q : p;
                cplx Dm[4], Mm[4];
                double w[4];
                for (int k = 0; k < 4; ++k) {
                    Dm[k] = P->data[4 * s + k];
                    Mm[k] = P->model[4 * s + k];
                    w[k] = P->weight[4 * s + (orient == 0 ? k : perm[k])];
                }
                if (orient == 1) { mat_herm(Dm, Dm); mat_herm(Mm, Mm); }
                cplx L[4], G[4], R[4], Cb[4], CbH[4], X[4], V[4];
                chain_factors(terms, n_terms, n, P->n_ant, t, c, a, L, G, R);
                chain_product(terms, n_terms, P->n_ant, t, c, b, Cb);
                mat_herm(Cb, CbH);
                /* X = R_a M C_b^H ;  V = L_a G_a X  (Eq. chain_trick) */
                mat_mul(R, Mm, X);
                mat_mul(X, CbH, X);
                mat_mul(L, G, V);
                mat_mul(V, X, V);
                cplx r[4];
                for (int k = 0; k < 4; ++k) r[k] = Dm[k] - V[k];
                /* E = L_a (x) X^T (Eq. vectrick, Eq. g_derivative_dd): E[(i,j),(k,l)] = L[i][k] * X^T[j][l] = L[i][k] X[l][j] */
                cplx E[4][4];
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j)
                        for (int k = 0; k < 2; ++k)
                            for (int l = 0; l < 2; ++l)
                                E[2 * i + j][2 * k + l] = L[2 * i + k] * X[2 * l + j];
                /* restrict / reparameterise the columns for the term type */
                cplx Ef[4][4];
                for (int row4 = 0; row4 < 4; ++row4) {
                    for (int col = 0; col < np; ++col) {
                        if (T->type == OC_FULL) {
                            Ef[row4][col] = E[row4][col];
                        } else if (T->type == OC_DELAY) {
                            /* dg_c/dphi_c = i g_c,  dg_c/dtau_c = 2 pi nu i g_c  (Scenario 2) */
                            const int dc = col < 2 ? 0 : 3;
                            Ef[row4][col] = E[row4][dc] * I * G[dc];
                            if (col & 1) Ef[row4][col] *= TWO_PI * T->chan_freq[c];
                        } else {
                            Ef[row4][col] = E[row4][free_cols_diag[col]];
                            if (T->type == OC_PHASE)   /* dg/dphi = i g  (Scenario 1) */
                                Ef[row4][col] *= I * G[free_cols_diag[col] == 0 ? 0 : 3];
                        }
                    }
                }
                cplx *Ja = jhj + ((bin * P->n_ant) + a) * np * np;
                cplx *ra = jhr + ((bin * P->n_ant) + a) * np;
                for (int u = 0; u < np; ++u) {
                    for (int v = 0; v < np; ++v) {
                        cplx acc = 0;
                        for (int k = 0; k < 4; ++k) acc += conj(Ef[k][u]) * w[k] * Ef[k][v];
                        Ja[u * np + v] += acc;
                    }
                    cplx acc = 0;
                    for (int k = 0; k < 4; ++k) acc += conj(Ef[k][u]) * w[k] * r[k];
                    ra[u] += acc;
                }
            }
        }
    }
    if (T->type == OC_PHASE || T->type == OC_DELAY) {   /* 2 Re(.) of Eq. jhj_case1/2, Eq. jhwr_case1/2 */
        for (size_t i = 0; i < n_bins * P->n_ant * np * np; ++i) jhj[i] = 2.0 * creal(jhj[i]);
        for (size_t i = 0; i < n_bins * P->n_ant * np; ++i) jhr[i] = 2.0 * creal(jhr[i]);
    }
    return OC_OK;
}

/* ------------------------------------------------------------------------ */
/* Small dense solve: LU with partial pivoting (n <= 4)                        */
/* ------------------------------------------------------------------------ */

/*
 * Solve A x = b.  Returns 0 on success, 1 if A is treated as singular:
 * zero trace, a zero pivot, or reciprocal 1-norm condition number < 1e-12.
 */
int oc_block_solve(int n, const cplx *A_in, const cplx *b, cplx *x)
{
    cplx A[16], inv[16];
    int piv[4];
    double trace = 0, anorm = 0;
    for (int i = 0; i < n; ++i) trace += creal(A_in[i * n + i]);
    if (!(trace > 0)) return 1;
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < n; ++i) s += cabs(A_in[i * n + j]);
        if (s > anorm) anorm = s;
    }
    memcpy(A, A_in, sizeof(cplx) * n * n);
    for (int i = 0; i < n; ++i) piv[i] = i;
    for (int k = 0; k < n; ++k) {
        int m = k;
        for (int i = k + 1; i < n; ++i) if (cabs(A[i * n + k]) > cabs(A[m * n + k])) m = i;
        if (cabs(A[m * n + k]) == 0) return 1;
        if (m != k) {
            for (int j = 0; j < n; ++j) { cplx t = A[k * n + j]; A[k * n + j] = A[m * n + j]; A[m * n + j] = t; }
            int t = piv[k]; piv[k] = piv[m]; piv[m] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            A[i * n + k] /= A[k * n + k];
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= A[i * n + k] * A[k * n + j];
        }
    }
    /* inverse column by column (for the condition number), then x = A^{-1} b */
    for (int col = 0; col < n; ++col) {
        cplx y[4];
        for (int i = 0; i < n; ++i) {
            cplx s = (piv[i] == col) ? 1.0 : 0.0;
            for (int j = 0; j < i; ++j) s -= A[i * n + j] * y[j];
            y[i] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            cplx s = y[i];
            for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * y[j];
            y[i] = s / A[i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[i * n + col] = y[i];
    }
    double inorm = 0;
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < n; ++i) s += cabs(inv[i * n + j]);
        if (s > inorm) inorm = s;
    }
    if (!(1.0 / (anorm * inorm) >= 1e-12)) return 1;
    for (int i = 0; i < n; ++i) {
        cplx s = 0;
        for (int j = 0; j < n; ++j) s += inv[i * n + j] * b[j];
        x[i] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 for one term, then the chain schedule over epochs              */
/* ------------------------------------------------------------------------ */

/* gain flagging on divergence: last two updates against the first two (see oc_solve_term) */
#define DIV_RATIO 0.9

static double step_length(const oc_opts *o, int k /* 1-based iteration */)
{
    if (o && o->damping_mode == 1) return (k % 2 == 0) ? 0.5 : 1.0;
    return (o && o->damping > 0) ? o->damping : 1.0;
}

/* Gain of antenna a in bin as 4 complex entries (Eq. gvec), for the convergence norm. */
static void term_gain_vec(const oc_term *T, size_t idx, cplx g[4])
{
    if (T->type == OC_PHASE) {
        g[0] = cexp(I * T->params[2 * idx]); g[1] = 0; g[2] = 0; g[3] = cexp(I * T->params[2 * idx + 1]);
        return;
    }
    for (int k = 0; k < 4; ++k) g[k] = T->params[8 * idx + 2 * k] + I * T->params[8 * idx + 2 * k + 1];
}

/*
 * Solve term n of the chain with Algorithm 1, every solution interval
 * independently (Section 2.3, last paragraph: solution intervals).  iters (nullable) receives
 * the iteration count per interval [n_tint*n_fint].
 *
 * Gain flagging on divergence (Section 4.3: a gain whose updates do not tend to zero), when
 * o->div_flag is set, for diagonal, full and phase-only terms: the relative update of antenna
 * a in an interval at iteration k is d_a(k) = ||g_a(k) - g_a(k-1)||_F / ||g_a(k)||_F.  An
 * interval that ends at max_iter = K >= 4 without converging flags each antenna whose last two
 * updates have not shrunk by more than a tenth from its first two,
 * max(d_a(K-1), d_a(K)) >= 0.9 max(d_a(1), d_a(2)) > 0 (pairs, so that a period-2 oscillation
 * and the alternating step length compare like with like; the margin keeps an exact
 * oscillation from being decided by rounding): its gain flag becomes 2 and its gain is
 * restored to its value before this solve.
 */
int oc_solve_term(const oc_problem *P, oc_term *terms, int n_terms, int n, const oc_opts *o, int *iters)
{
    oc_term *T = &terms[n];
    const int np = n_param(T->type), na = P->n_ant;
    const size_t n_bins = (size_t)T->n_tint * T->n_fint;
    cplx *jhj = malloc(sizeof(cplx) * n_bins * na * np * np);
    cplx *jhr = malloc(sizeof(cplx) * n_bins * na * np);
    unsigned char *active = malloc(n_bins);
    if (!jhj || !jhr || !active) { free(jhj); free(jhr); free(active); return OC_ENOMEM; }
    memset(active, 1, n_bins);
    if (iters) memset(iters, 0, sizeof(int) * n_bins);
    /* divergence tracking: first and latest relative update per (interval, antenna), initial gains */
    const int track = o && o->div_flag && T->type != OC_DELAY && T->max_iter >= 4;
    const size_t pstride = T->type == OC_PHASE ? 2 : 8;
    double *d_first = NULL, *d_last = NULL, *p0 = NULL;
    if (track) {
        d_first = calloc(n_bins * na, sizeof(double));
        d_last = calloc(n_bins * na, sizeof(double));
        p0 = malloc(sizeof(double) * n_bins * na * pstride);
        if (!d_first || !d_last || !p0) {
            free(jhj); free(jhr); free(active); free(d_first); free(d_last); free(p0);
            return OC_ENOMEM;
        }
        memcpy(p0, T->params, sizeof(double) * n_bins * na * pstride);
    }

    for (int k = 1; k <= T->max_iter; ++k) {
        int any = 0;
        for (size_t b = 0; b < n_bins; ++b) any |= active[b];
        if (!any) break;
        oc_normal_equations(P, terms, n_terms, n, active, jhj, jhr);
        const double alpha = step_length(o, k);
        for (size_t b = 0; b < n_bins; ++b) {
            if (!active[b]) continue;
            double num = 0, den = 0;
            for (int a = 0; a < na; ++a) {
                const size_t idx = b * na + a;
                cplx g_old[4], g_new[4], dx[4];
                if (T->type == OC_DELAY) {
                    /* the gains change per channel: sum the change over the interval's channels */
                    double u_old[4];
                    memcpy(u_old, T->params + 4 * idx, sizeof u_old);
                    int singular = oc_block_solve(np, jhj + idx * np * np, jhr + idx * np, dx);
                    if (T->gain_flags) T->gain_flags[idx] = (signed char)singular;
                    if (!singular)
                        for (int e = 0; e < 4; ++e) T->params[4 * idx + e] += alpha * creal(dx[e]);
                    const int jf = (int)(b % T->n_fint);
                    for (int c = 0; c < P->n_chan; ++c) {
                        if (T->f_map[c] != jf) continue;
                        cplx ox, oy, nx, ny;
                        delay_gains(u_old, T->chan_freq[c], &ox, &oy);
                        delay_gains(T->params + 4 * idx, T->chan_freq[c], &nx, &ny);
                        num += creal((nx - ox) * conj(nx - ox)) + creal((ny - oy) * conj(ny - oy));
                        den += creal(nx * conj(nx)) + creal(ny * conj(ny));
                    }
                    continue;
                }
                term_gain_vec(T, idx, g_old);
                int singular = oc_block_solve(np, jhj + idx * np * np, jhr + idx * np, dx);
                if (T->gain_flags) T->gain_flags[idx] = (signed char)singular;
                if (!singular) {
                    if (T->type == OC_PHASE) {
                        T->params[2 * idx] += alpha * creal(dx[0]);
                        T->params[2 * idx + 1] += alpha * creal(dx[1]);
                    } else if (T->type == OC_DIAG) {
                        T->params[8 * idx + 0] += alpha * creal(dx[0]);
                        T->params[8 * idx + 1] += alpha * cimag(dx[0]);
                        T->params[8 * idx + 6] += alpha * creal(dx[1]);
                        T->params[8 * idx + 7] += alpha * cimag(dx[1]);
                    } else {
                        for (int e = 0; e < 4; ++e) {
                            T->params[8 * idx + 2 * e] += alpha * creal(dx[e]);
                            T->params[8 * idx + 2 * e + 1] += alpha * cimag(dx[e]);
                        }
                    }
                }
                term_gain_vec(T, idx, g_new);
                double na_ = 0, da_ = 0;
                for (int e = 0; e < 4; ++e) {
                    na_ += creal((g_new[e] - g_old[e]) * conj(g_new[e] - g_old[e]));
                    da_ += creal(g_new[e] * conj(g_new[e]));
                }
                num += na_;
                den += da_;
                if (track) {
                    const double da = da_ > 0 ? sqrt(na_ / da_) : 0.0;
                    if (k <= 2) d_first[idx] = fmax(d_first[idx], da);       /* max(d(1), d(2)) */
                    if (k >= T->max_iter - 1) d_last[idx] = fmax(d_last[idx], da); /* max(d(K-1), d(K)) */
                }
            }
            if (iters) iters[b] = k;
            const double delta = den > 0 ? sqrt(num / den) : 0.0;
            if (delta < T->tol) active[b] = 0;
        }
    }
    if (track) {
        /* intervals still active ran to max_iter without converging */
        for (size_t b = 0; b < n_bins; ++b) {
            if (!active[b]) continue;
            for (int a = 0; a < na; ++a) {
                const size_t idx = b * na + a;
                if (d_first[idx] > 0 && d_last[idx] >= DIV_RATIO * d_first[idx]) {
                    memcpy(T->params + pstride * idx, p0 + pstride * idx, sizeof(double) * pstride);
                    if (T->gain_flags) T->gain_flags[idx] = 2;
                }
            }
        }
    }
    free(jhj); free(jhr); free(active); free(d_first); free(d_last); free(p0);
    return OC_OK;
}

/*
 * Chain schedule (Section 4.3): for each epoch, each solvable term in chain
 * order is solved to convergence / max_iter before moving to the next.
 * iters (nullable): per term, per interval counts of the last epoch, packed
 * term after term.
 */
int oc_solve(const oc_problem *P, oc_term *terms, int n_terms, const oc_opts *o, int *iters)
{
    const int n_epochs = (o && o->n_epochs > 0) ? o->n_epochs : 1;
    for (int e = 0; e < n_epochs; ++e) {
        size_t off = 0;
        for (int n = 0; n < n_terms; ++n) {
            const size_t nb = (size_t)terms[n].n_tint * terms[n].n_fint;
            if (terms[n].solve) {
                int rc = oc_solve_term(P, terms, n_terms, n, o, iters ? iters + off : NULL);
                if (rc) return rc;
            }
            off += nb;
        }
    }
    return OC_OK;
}

/* ------------------------------------------------------------------------ */
/* Residual and chi^2 (Eq. min and Eq. baselineresidual)                       */
/* ------------------------------------------------------------------------ */

/*
 * chi2 = sum over unflagged cross-correlation samples and correlations of
 * w |d - v|^2.  resid (nullable) receives r = D - C_p M C_q^H for every
 * sample (zero for flagged samples and autocorrelations).
 */
int oc_residual(const oc_problem *P, const oc_term *terms, int n_terms, cplx *resid, double *chi2)
{
    double acc = 0;
    for (int row = 0; row < P->n_row; ++row) {
        const int p = P->ant1[row], q = P->ant2[row], t = P->time_idx[row];
        for (int c = 0; c < P->n_chan; ++c) {
            const size_t s = (size_t)row * P->n_chan + c;
            const int skip = (p == q) || (P->flag && P->flag[s]);
            if (skip) { if (resid) for (int k = 0; k < 4; ++k) resid[4 * s + k] = 0; continue; }
            cplx Cp[4], Cq[4], CqH[4], V[4];
            chain_product(terms, n_terms, P->n_ant, t, c, p, Cp);
            chain_product(terms, n_terms, P->n_ant, t, c, q, Cq);
            mat_herm(Cq, CqH);
            mat_mul(Cp, P->model + 4 * s, V);
            mat_mul(V, CqH, V);
            for (int k = 0; k < 4; ++k) {
                cplx r = P->data[4 * s + k] - V[k];
                if (resid) resid[4 * s + k] = r;
                acc += P->weight[4 * s + k] * creal(r * conj(r));
            }
        }
    }
    *chi2 = acc;
    return OC_OK;
}
