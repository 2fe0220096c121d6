/*
 * evsl_gb300.h -- C ABI of the GB300 (sm_103a) implementation of polynomial-filtered spectrum
 * slicing for large sparse symmetric eigenproblems (Li, Xi, Erlandson, Saad, "The Eigenvalues
 * Slicing Library (EVSL)", arXiv:1802.05215).
 *
 * Problem (Sec. 1, Eq. (1.2); Sec. 2.1): find all eigenpairs (lambda, x) of a real symmetric
 * sparse A with lambda in [xi, eta].  Workflow of the paper's Example 1 (Sec. 3.1):
 *   evsl_create -> evsl_set_csr -> evsl_bounds -> evsl_kpm_dos -> evsl_slice_by_dos ->
 *   for each slice: evsl_cheb_filter_build -> evsl_chebLanTr -> evsl_destroy.
 *
 * Conventions for every call:
 *   - Return value is an evsl_status (0 = EVSL_OK, negative = error).  On error the context's
 *     message is available from evsl_last_error(); output arguments are left unspecified
 *     unless the call says otherwise.
 *   - Host pointers are read or written only during the call and never retained.
 *   - Device memory is owned by the context and freed by evsl_destroy.
 *   - A context is bound to one CUDA device and one CUDA stream; use it from one host thread
 *     at a time.  Calls are synchronous with respect to the host unless stated otherwise.
 *   - The context's own stream is created non-blocking: it does not wait for work queued on
 *     other streams, the legacy default stream included.  Device buffers passed to a call must
 *     be complete when the call is made: synchronise their producer first, or produce them on
 *     the context's stream (evsl_set_stream).
 *   - Dense vectors and blocks are column-major (vector j of an n x k block starts at j*n).
 *   - Nothing in this library falls back to the CPU: without a usable GPU the calls that need
 *     one return EVSL_ERR_CUDA.
 */
#ifndef EVSL_GB300_H
#define EVSL_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct evsl_ctx evsl_ctx;

typedef enum {
    EVSL_OK = 0,
    EVSL_ERR_ARG = -1,      /* invalid argument (sizes, pointers, intervals)            */
    EVSL_ERR_NOMEM = -2,    /* device allocation failed or the HBM budget is exceeded   */
    EVSL_ERR_CUDA = -3,     /* a CUDA runtime call or kernel launch failed              */
    EVSL_ERR_NOCONV = -4,   /* iteration limit reached; partial results are returned    */
    EVSL_ERR_CAPACITY = -5, /* caller buffer too small; the needed size is reported     */
    EVSL_ERR_TIMEOUT = -6,  /* a bounded device-side wait gave up                       */
    EVSL_ERR_STATE = -7     /* call out of order (e.g. no matrix set)                   */
} evsl_status;

typedef enum { EVSL_DAMP_NONE = 0, EVSL_DAMP_JACKSON = 1, EVSL_DAMP_SIGMA = 2 } evsl_damping;
typedef enum { EVSL_FP64 = 0, EVSL_FP32 = 1 } evsl_precision;

/* ---------------------------------------------------------------------------------------- */
/* Context.  Replaces the paper's global state (EVSLStart/EVSLFinish, Sec. 3.1).
 * device: CUDA ordinal.  hbm_budget_bytes: cap on the device memory the context may hold
 * (0 = no cap); allocations beyond it fail with EVSL_ERR_NOMEM.  *ctx is set to NULL on error. */
int evsl_create(evsl_ctx **ctx, int device, size_t hbm_budget_bytes);
/* Frees everything the context holds, including batches created on it that were not destroyed
 * (their unfinished jobs are discarded; the batch handles become invalid). */
void evsl_destroy(evsl_ctx *ctx);
/* Message of the last failed call on ctx (empty string if none); valid until the next call. */
const char *evsl_last_error(const evsl_ctx *ctx);
/* Run the context's work on an existing stream (a cudaStream_t passed as void*); NULL restores
 * the context's own stream.  The caller keeps ownership of the stream. */
int evsl_set_stream(evsl_ctx *ctx, void *cuda_stream);

/* ---------------------------------------------------------------------------------------- */
/* Matrix (Sec. 3.1: CSR storage; SetAMatrix).  A is symmetric with both triangles stored,
 * 0-based, column indices sorted within each row.  row_ptr[n+1] (row_ptr[0] = 0,
 * non-decreasing), col_idx[nnz], val[nnz] are HOST arrays, copied in; the caller keeps them.
 * The device copy is a sliced ELLPACK layout (32-row slices) in FP64 with an FP32 mirror.
 * Replaces any previous matrix.  Symmetry is assumed, not checked.  Errors: EVSL_ERR_ARG for
 * n < 1, nnz >= 2^31, a bad row_ptr or an out-of-range column index. */
int evsl_set_csr(evsl_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                 const double *val);

/* Spectral bounds (Sec. 2.2.1, text after Eq. (2.3); LanTrbounds, Sec. 3.1): `steps` Lanczos
 * steps (full reorthogonalisation) from the seeded start vector; returns the extreme Ritz values
 * widened by their residual bounds, lmin = theta_1 - |beta s_{m,1}|, lmax = theta_m +
 * |beta s_{m,m}|.  lmin/lmax are host pointers. */
int evsl_bounds(evsl_ctx *ctx, int steps, uint64_t seed, double *lmin, double *lmax);

/* KPM spectral density (Sec. 2.1; kpmdos): with Ahat = (A - cI)/d, c and d the centre and
 * half-width of [lmin, lmax] (Eq. (2.3)), and nvec Rademacher probes v_l drawn by SplitMix64
 * from `seed` (sign of draw(seed, 2, l*n + i)),
 *     mu[k] = (1/nvec) * sum_l v_l^T T_k(Ahat) v_l ,   k = 0..degree   (so mu[0] == n).
 * mu[degree+1] is a HOST array.  prec selects FP64 or FP32 vectors and matrix values in the
 * recurrence (per-row dot products are accumulated in FP64 either way). */
int evsl_kpm_dos(evsl_ctx *ctx, int degree, int nvec, uint64_t seed, double lmin, double lmax,
                 evsl_precision prec, double *mu);

/* KPM moments by the doubling identities (the moment-doubling variant the KPM literature uses
 * with T_{2k} = 2 T_k^2 - T_0 and T_{2k+1} = 2 T_{k+1} T_k - T_1): the same mu[0..degree], same
 * probes, from ceil(degree/2) recurrence steps instead of degree:
 * mu_{2k} = (1/nvec) sum_l (2 ||w_k||^2 - n), mu_{2k+1} = (1/nvec) sum_l (2 w_{k+1}^T w_k - v_l^T w_1)
 * with w_k = T_k(Ahat) v_l.  Results differ from evsl_kpm_dos by rounding only (the identities
 * are exact); arguments and errors as evsl_kpm_dos. */
int evsl_kpm_dos_doubling(evsl_ctx *ctx, int degree, int nvec, uint64_t seed, double lmin, double lmax,
                          evsl_precision prec, double *mu);

/* Per-probe KPM sums (Sec. 2.1: the terms of the estimator before averaging), for spreading the
 * probes over processes (Sec. 2.6's first level of parallelism): for probes first .. first +
 * nprobe - 1, the same probes as evsl_kpm_dos (probe index first + l draws its signs at counter
 * (first + l) n + i),
 *     out[l * (degree + 1) + k] = v_{first+l}^T T_k(Ahat) v_{first+l},   k = 0..degree.
 * Each probe's values are formed in an order that depends on n only, not on first or nprobe,
 * so gathering every process's rows and adding them in probe order gives the same moments
 * bitwise however the probes were split.  out: HOST array of nprobe (degree + 1) doubles.
 * prec as in evsl_kpm_dos.  Errors: EVSL_ERR_ARG, EVSL_ERR_STATE without a matrix. */
int evsl_kpm_probe_moments(evsl_ctx *ctx, int degree, int64_t first, int nprobe, uint64_t seed, double lmin,
                           double lmax, evsl_precision prec, double *out);

/* DOS slicer (Sec. 2.1, Eq. (2.2); spslicer).  Pure host function, no context.  From the
 * Jackson-damped KPM density it places npts evenly spaced points on [xi, eta], and puts the
 * slice ends t_1..t_{ns-1} where the cumulative count crosses i/ns of the total (first crossing,
 * refined by linear interpolation); sli[0] = xi, sli[nslices] = eta.  est[i] is the estimated
 * eigenvalue count of slice i.  sli[nslices+1] and est[nslices] are caller-owned host arrays.
 * n is the matrix order (mu[0] should equal it).  npts <= 0 selects max(2001, 100*nslices). */
int evsl_slice_by_dos(const double *mu, int degree, int64_t n, double lmin, double lmax,
                      double xi, double eta, int nslices, int npts, double *sli, double *est);

/* ---------------------------------------------------------------------------------------- */
/* Chebyshev delta filter (Sec. 2.2.1, Eqs. (2.4)-(2.7); find_pol).
 * rho(t) = sum_{j<=deg} coef[j] T_j((t - c)/d).  Interior slices: for deg = 2, 3, ... the
 * centre gamma is balanced by Newton's method so that rho(a) = rho(b) (Eq. (2.7)), and the
 * first degree with end value bar <= tau (default 0.8) is kept.  Slices whose mapped left end
 * is <= -1 (right end >= 1) are boundary slices: gamma = -1 (+1), same damping, and the degree
 * grows until rho(inner end) <= tau_ext (default 0.4).  `bar` is the end value, i.e. the
 * threshold that separates wanted from unwanted Ritz values of rho(A). */
typedef struct {
    double tau;             /* end-value threshold for interior slices (0.8)            */
    double tau_ext;         /* end-value threshold for boundary slices (0.4)            */
    evsl_damping damping;   /* EVSL_DAMP_JACKSON (default), EVSL_DAMP_SIGMA, NONE       */
    int max_deg;            /* largest degree tried (10000)                             */
} evsl_filter_opts;

typedef struct {
    int deg;                /* polynomial degree                                        */
    int boundary;           /* -1 left boundary slice, +1 right, 0 interior             */
    double gamma;           /* centre in the mapped variable                            */
    double bar;             /* rho at the slice ends (interior) / inner end (boundary)  */
    double lmin, lmax;      /* spectral interval used for the mapping                   */
    double a, b;            /* the slice                                                */
    const double *coef;     /* deg+1 Chebyshev coefficients (caller-owned host memory)  */
} evsl_polfilt;

/* Pure host function.  opts may be NULL (defaults).  coef[cap] is a caller-owned host array;
 * on success pol->coef == coef.  Errors: EVSL_ERR_ARG (b <= a, lmax <= lmin, or [a, b]
 * covering the whole spectral interval or lying outside it); EVSL_ERR_CAPACITY if cap < deg+1 (pol->deg then
 * holds the degree needed); EVSL_ERR_NOCONV if max_deg was reached (the max_deg filter is
 * returned). */
int evsl_cheb_filter_build(double a, double b, double lmin, double lmax,
                           const evsl_filter_opts *opts, evsl_polfilt *pol, double *coef, int cap);

/* Filter application (Eq. (2.4) with the three-term Chebyshev recurrence): Y = rho(Ahat) X for
 * nvec columns.  X and Y are DEVICE pointers to n x nvec column-major FP64 blocks (Y must not
 * overlap X).  prec = EVSL_FP32 runs the recurrence in FP32 (X/Y stay FP64).
 * Execution: a single column of degree >= 8 replays a CUDA graph of the degree launches that the
 * context captures on first use and caches (keyed by filter, buffers and matrix; dropped by
 * evsl_set_csr and evsl_destroy).  The first block of a given width on a matrix times five tile
 * shapes of the block kernel once (synchronously) and keeps the fastest; results do not depend
 * on the shape.  Neither happens while the context's stream is being captured by the caller
 * (then the launches are issued directly). */
int evsl_filter_apply(evsl_ctx *ctx, const evsl_polfilt *pol, int nvec, const double *X,
                      double *Y, evsl_precision prec);

/* Multi-slice filter application: column t of X gets filter pols[t] (the slices of one
 * interval are independent, Sec. 2.1 and 2.6, so their filters can share each pass over the
 * matrix).  All filters must use the same [lmin, lmax].  Columns are processed in order of
 * decreasing degree; at degree j one launch updates every column whose degree is >= j, so the
 * matrix is read once per degree for all slices.  X, Y: DEVICE n x npol column-major FP64
 * (non-overlapping); prec as in evsl_filter_apply. */
int evsl_filter_apply_multi(evsl_ctx *ctx, int npol, const evsl_polfilt *pols, const double *X,
                            double *Y, evsl_precision prec);

/* Allocation-free form of evsl_filter_apply (the paper has no counterpart).  For callers that
 * must not allocate device memory once set up: hosts whose device memory belongs to another
 * allocator (a framework's caching pool that owns the GPU, so a cudaMalloc by this library
 * would fail or fragment that pool), and real-time or embedded loops that forbid allocation
 * after initialisation because cudaMalloc/cudaFree can block and synchronise the device.
 * Same operation, arguments and layout as evsl_filter_apply with prec = EVSL_FP64:
 * Y = rho(Ahat) X on nvec columns, X and Y device pointers (n x nvec, column-major,
 * non-overlapping), matrix from the context.  The two recurrence temporaries live in one fixed
 * device array of 2 * EVSL_NOALLOC_MAX_ELEMS doubles (32 MiB) that this library reserves on
 * every GPU where its kernels are loaded, until the process exits; this call allocates nothing
 * (no cudaMalloc/cudaFree, no workspace growth, no event creation).  Its first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device current and keeps
 * it for the life of the process; the kept address is valid only until the device is reset
 * (cudaDeviceReset), after which this entry point must not be used in the same process.  Every
 * call shares the array: calls that can overlap on the GPU (several contexts or threads on one
 * device) race and must be serialised by the caller.  The array keeps the previous call's
 * contents; nothing in it has to start at zero, because each temporary entry is written before
 * it is read.  The call is synchronous: it waits on the context's stream for its kernels to
 * finish before it returns.  It makes the context's device current while it runs and restores
 * the calling thread's previous current device before returning.  Errors: EVSL_ERR_ARG if
 * n * nvec > EVSL_NOALLOC_MAX_ELEMS (the message names the limit), EVSL_ERR_STATE without a
 * matrix, EVSL_ERR_CUDA if the address lookup fails. */
#define EVSL_NOALLOC_MAX_ELEMS (1 << 21)
int evsl_filter_apply_noalloc(evsl_ctx *ctx, const evsl_polfilt *pol, int nvec, const double *X,
                              double *Y);

/* ---------------------------------------------------------------------------------------- */
/* Filtered thick-restart Lanczos with locking (Sec. 2.5, Algorithm 2; ChebLanTr) on the slice
 * [a, b] with filter pol (built for the same slice).  Candidates are the Ritz values of
 * rho(A) at or above pol->bar; their Rayleigh quotients u^T A u outside the slice are ignored;
 * pairs with ||A u - lambda u|| <= tol * max(|lmin|, |lmax|) are locked and deflated.
 * The run stops after two consecutive restarts without candidates (a restart without
 * candidates makes the next cycle start from a fresh seeded vector orthogonal to the locked
 * ones), or with EVSL_ERR_NOCONV when maxit filtered matvec steps were spent.
 * Outputs: *nev pairs, eigenvalues ascending in lam[cap] and res[cap] (relative residuals) on
 * the HOST, eigenvectors in Y (n x cap column-major), which may be host or device memory
 * (detected).  If more than cap pairs converge: EVSL_ERR_CAPACITY, *nev = cap, outputs hold
 * the first cap found.
 * prec = EVSL_FP32 (not in the paper): the filter runs in FP32 and everything else in FP64.  The
 * Lanczos phase then locks at max(tol, 1e-6) (relaxed up to 1e-4 if candidates stall) in the slice
 * widened by that level times ||A||, and an FP64 polish (restarted block Krylov iteration with
 * the FP64 filter, Rayleigh-Ritz with A on the converged Ritz vectors of rho) brings the pairs to
 * tol and decides membership.  If the polish cannot bring every in-slice pair to tol (or its
 * workspace does not fit under the HBM budget), the slice is solved again with the FP64 filter
 * and that run's pairs are returned, so the FP32 mode never returns fewer pairs than the FP64
 * one.  The polish holds about 6 n (p + max(16, p/4)) doubles of workspace for p locked pairs. */
typedef struct {
    int m;                  /* Krylov dimension before a restart                        */
    int maxit;              /* limit on Lanczos steps (0 = 20*m)                        */
    int ncycle;             /* early-restart test period (10)                           */
    double tol;             /* residual tolerance relative to ||A|| (1e-8)              */
    double tau1;            /* early-restart tolerance on the Ritz-value sum (1e-10)     */
    uint64_t seed;          /* start vectors: SplitMix64 stream 3                       */
    evsl_precision prec;    /* filter precision: EVSL_FP64 or EVSL_FP32                 */
    int right_closed;       /* 1: lambda in [a, b]; 0: lambda in [a, b)                 */
} evsl_lan_opts;

typedef struct {
    int64_t niter;          /* Lanczos steps                                            */
    int64_t nmv;            /* sparse matrix-vector products inside the filter          */
    int64_t nrestart;       /* restarts                                                 */
    int64_t npass;          /* Gram-Schmidt passes                                      */
    double t_filter;        /* seconds in filter application                            */
    double t_orth;          /* seconds in reorthogonalisation                           */
    double t_restart;       /* seconds in restarts (small eigensolves, Ritz vectors)     */
    double t_total;         /* seconds in the call                                      */
} evsl_stats;

int evsl_chebLanTr(evsl_ctx *ctx, double a, double b, const evsl_polfilt *pol,
                   const evsl_lan_opts *opts, int cap, int *nev, double *lam, double *Y,
                   double *res, evsl_stats *stats);

/* Lanczos spectral density (landos; Sec. 2.1 names the Lanczos / Gaussian-quadrature method of
 * Lin, Saad and Yang as the alternative to KPM).  For each of nvec seeded unit vectors (stream 5),
 * an m-step Lanczos run on A with full reorthogonalisation gives T = S diag(theta) S^T; the
 * quadrature of v^T f(A) v has nodes theta_j and weights S_{1j}^2, and the density is
 * (n / nvec) sum_l sum_j w_lj delta(t - theta_lj).  Outputs on the HOST (row l = vector l,
 * m entries): nodes (ascending within a row), their weights, and mused[l] <= m, the steps actually run (a breakdown, beta <=
 * 1e-13 ||A q||, ends a run early: the quadrature is then exact for that vector). */
int evsl_landos(evsl_ctx *ctx, int m, int nvec, uint64_t seed, double *nodes, double *weights, int *mused);

/* Slicer on the Lanczos density (spslicer2; host only, no context).  The cumulative count is the
 * step function N(t) = (n / nvec) sum of the weights of the nodes <= t; with C0 = N just below xi
 * and C1 = N(eta), boundary t_i (0 < i < nslices) lies midway between the first node in [xi, eta]
 * where N reaches C0 + (i / nslices)(C1 - C0) and the node before it.  sli[nslices + 1] and
 * est[nslices] (estimated count per slice) caller-owned.  EVSL_ERR_ARG if no node lies in
 * [xi, eta] or the arguments are invalid. */
int evsl_slice_by_landos(const double *nodes, const double *weights, const int *mused, int m, int nvec,
                         int64_t n, double xi, double eta, int nslices, double *sli, double *est);

/* Filtered non-restart Lanczos (ChebLanNr, the variant the paper times in Tables 2 and 4; the
 * paper gives it no listing, and this is Algorithm 2 without restarts or locking).  One Krylov
 * basis of rho(A) with full reorthogonalisation grows up to opts->m vectors (opts->maxit is not
 * used).  Every ncycle steps the sum of the Ritz values >= pol->bar is formed; when it is stable
 * (relative change < tau1) the candidates are extracted as in evsl_chebLanTr (Rayleigh quotients
 * with A, pairs outside the slice dropped).  If every in-slice candidate has
 * ||A u - lambda u|| <= tol ||A|| the run returns them; otherwise the same basis keeps growing.
 * With a full basis the converged in-slice pairs are returned and the status is EVSL_ERR_NOCONV
 * if some in-slice candidate did not converge.  A slice with no Ritz value >= bar at two
 * consecutive tests after max(2 ncycle, m/4) steps returns 0 pairs.  Arguments, outputs,
 * EVSL_ERR_CAPACITY and the FP32 filter mode are as in evsl_chebLanTr; stats->nrestart counts
 * the extractions.  Device memory: about 2 n (m + 1) doubles for the basis and the Ritz block,
 * plus n cap for the result. */
int evsl_chebLanNr(evsl_ctx *ctx, double a, double b, const evsl_polfilt *pol,
                   const evsl_lan_opts *opts, int cap, int *nev, double *lam, double *Y,
                   double *res, evsl_stats *stats);

/* Polynomial filtered subspace iteration (ChebSI; the paper lists it among EVSL's projection
 * methods and notes that its subspace dimension comes from the DOS count, but gives no listing).
 * A block of opts->m vectors (about 1.5 times the slice's estimated count plus a margin) starts
 * from seeded random vectors; each pass applies rho(A) to the block, orthonormalises it and
 * performs Rayleigh-Ritz with A.  The filter's Rayleigh quotient mu = v^T rho(A) v of each Ritz
 * vector (free from the next pass) separates wanted pairs (mu >= pol->bar) from mixtures of
 * eigenvectors outside the slice (mu < bar); the run stops when every in-slice Ritz pair with
 * mu >= bar meets tol, after at most opts->maxit passes (0 = 100; then EVSL_ERR_NOCONV with the
 * converged pairs).  FP64 filter only (EVSL_ERR_ARG otherwise); outputs and EVSL_ERR_CAPACITY
 * as in evsl_chebLanTr; stats->niter counts passes, stats->nmv all filter matvecs.  Device
 * memory: about 4 n m doubles. */
int evsl_chebSI(evsl_ctx *ctx, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *opts,
                int cap, int *nev, double *lam, double *Y, double *res, evsl_stats *stats);

/* Several slices of one matrix solved together (Sec. 2.6: slices are independent; here they
 * share the GPU instead of separate processes).  Each job is one slice with its own filter,
 * Krylov dimension and outputs; the slices advance in lockstep and every Lanczos step applies
 * all their filters in one multi-slice pass per degree (as evsl_filter_apply_multi), while
 * reorthogonalisation, restarts and locking stay per slice exactly as in evsl_chebLanTr.
 * All filters must share [lmin, lmax].  opts supplies maxit (per slice), ncycle, tol, tau1,
 * seed and prec; opts->m and opts->right_closed are taken from each job instead.  Device
 * memory: each slice holds n x (cap + m + 1) doubles for its bases.  The call returns the first
 * failing job's status (EVSL_OK if all succeeded); each job's own status is in job.status. */
typedef struct {
    double a, b;                /* the slice                                                */
    const evsl_polfilt *pol;    /* its filter                                               */
    int m;                      /* Krylov dimension for this slice                          */
    int cap;                    /* capacity of lam, res and Y                               */
    int right_closed;           /* 1: lambda in [a, b]; 0: lambda in [a, b)                 */
    int *nev;                   /* out: number of pairs                                     */
    double *lam, *res;          /* out: host arrays of cap entries                          */
    double *Y;                  /* out: n x cap column-major, host or device memory         */
    evsl_stats *stats;          /* out: may be NULL                                         */
    int status;                 /* out: this slice's evsl_status                            */
} evsl_slice_job;

int evsl_chebLanTr_batch(evsl_ctx *ctx, int njobs, evsl_slice_job *jobs, const evsl_lan_opts *opts);

/* Incremental form of evsl_chebLanTr_batch, for serving: jobs (slice solves on the context's
 * matrix) join between steps and leave when finished, so requests that arrive while others run
 * are admitted as soon as device memory allows (continuous batching).  evsl_batch_add allocates
 * the job's bases (EVSL_ERR_NOMEM if the context's HBM budget would be exceeded; the job is then
 * not admitted and the caller may retry later) and RETAINS the job pointer until the job
 * finishes.  evsl_batch_step performs one Lanczos step of every active job (one multi-slice
 * filter pass per degree, then each job's reorthogonalisation and, where a cycle ends, its
 * restart); finished jobs get their outputs and status written, their device memory released,
 * and are counted in *nfinished.  *nactive is the number of jobs still running.  Results of a
 * job do not depend on which other jobs share its steps.  Destroying a batch discards the
 * unfinished jobs without writing their outputs. */
typedef struct evsl_batch evsl_batch;
int evsl_batch_create(evsl_ctx *ctx, const evsl_lan_opts *opts, evsl_batch **batch);
int evsl_batch_add(evsl_batch *batch, evsl_slice_job *job);
int evsl_batch_step(evsl_batch *batch, int *nactive, int *nfinished);
void evsl_batch_destroy(evsl_batch *batch);

/* ---------------------------------------------------------------------------------------- */
/* Generalized problems A x = lambda B x (Sec. 2.4-2.5) with B symmetric positive definite and
 * well conditioned, whose inverse is replaced by a polynomial (Sec. 4.3, the lsPol solve).
 *
 * evsl_lspol (host only): Chebyshev coefficients c_0..c_deg of p(t) ~ 1/t on [bmin, bmax]
 * (0 < bmin < bmax) in the variable (t - (bmax + bmin)/2) / ((bmax - bmin)/2): the interpolant at
 * the deg + 1 Chebyshev-Gauss points, deg the smallest degree <= maxdeg whose relative error
 * max |t p(t) - 1| over 2001 equispaced points of [bmin, bmax] is <= eps.  coef: host array of
 * cap >= maxdeg + 1 doubles; *err (may be NULL) receives that error.  Errors: EVSL_ERR_ARG;
 * EVSL_ERR_CAPACITY if cap < maxdeg + 1; EVSL_ERR_NOCONV if maxdeg was reached (the degree-maxdeg
 * interpolant is returned). */
int evsl_lspol(double bmin, double bmax, double eps, int maxdeg, int *deg, double *coef, int cap,
               double *err);

/* evsl_lspol_isqrt (host only): as evsl_lspol for q(t) ~ t^{-1/2} (relative error
 * max |sqrt(t) q(t) - 1|): the polynomial B^{-1/2} that builds the starting vectors of the
 * pencil's density (Sec. 2.1). */
int evsl_lspol_isqrt(double bmin, double bmax, double eps, int maxdeg, int *deg, double *coef,
                     int cap, double *err);

/* Mass matrix B (host CSR, same conventions and errors as evsl_set_csr) with its spectrum inside
 * [bmin, bmax], and its polynomial inverse p(B) (evsl_lspol with eps, maxdeg; *deg and *err may be
 * NULL, and report p) and inverse square root q(B) (evsl_lspol_isqrt, same eps and maxdeg).  Replaces any previous B; evsl_set_csr leaves B in place.  The solvers below need B and
 * A of the same order.  Errors: those of evsl_set_csr; EVSL_ERR_ARG if not 0 < bmin < bmax,
 * eps <= 0 or maxdeg < 1; EVSL_ERR_NOCONV if maxdeg did not reach eps (B and the degree-maxdeg
 * polynomial are set all the same). */
int evsl_set_csr_b(evsl_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                   const double *val, double bmin, double bmax, double eps, int maxdeg, int *deg,
                   double *err);

/* y = p(B) x (the approximate solve with B): x, y DEVICE pointers to n doubles, y distinct from
 * x.  Synchronous.  Errors: EVSL_ERR_ARG, EVSL_ERR_STATE without B. */
int evsl_polyB_apply(evsl_ctx *ctx, const double *x, double *y);

/* KPM moments of the pencil (Sec. 2.1's density extended to A x = lambda B x): the moments of the
 * density of S = B^{-1/2} A B^{-1/2} on [lmin, lmax] (the pencil's bounds, evsl_bounds_gen),
 * mu[k] = (1/nvec) sum_l v_l^T T_k((S - cI)/d) v_l for the Rademacher probes of evsl_kpm_dos, so
 * mu[0] = n up to the polynomials' accuracy.  Computed as u_l^T T_k((A B^{-1} - cI)/d) B u_l with
 * u_l = q(B) v_l and B^{-1} by p(B) (every degree one solve with B and one product with A).  mu:
 * host array of degree + 1 doubles; FP64; the moments feed evsl_slice_by_dos unchanged.  Errors:
 * EVSL_ERR_ARG, EVSL_ERR_STATE (as evsl_bounds_gen). */
int evsl_kpm_dos_gen(evsl_ctx *ctx, int degree, int nvec, uint64_t seed, double lmin, double lmax,
                     double *mu);

/* Lanczos quadrature density of the pencil (Sec. 2.1's Lanczos density extended to A x = lambda B x;
 * the lanDos step of the paper's Example 1): for each of nvec unit start vectors v_l (those of
 * evsl_landos), m steps of the B-inner-product Lanczos (Algorithm 3) on B^{-1} A from
 * w_1 = q(B) v_l (q ~ t^{-1/2}, set by evsl_set_csr_b) give the Gauss quadrature of
 * v_l^T f(B^{-1/2} A B^{-1/2}) v_l.  Outputs, layout and breakdown rule as evsl_landos (the
 * breakdown norm is ||A w_i|| / sqrt(bmax)); the result feeds evsl_slice_by_landos unchanged.
 * Errors: EVSL_ERR_ARG, EVSL_ERR_STATE (as evsl_bounds_gen). */
int evsl_landos_gen(evsl_ctx *ctx, int m, int nvec, uint64_t seed, double *nodes, double *weights,
                    int *mused);

/* Spectral bounds of the pencil: `steps` unfiltered steps of the B-inner-product Lanczos
 * (Algorithm 3) on B^{-1} A from a seeded start (Lanczos stream, index 0), with p(B) for B^{-1};
 * lmin = theta_1 - |beta s_{m,1}|, lmax = theta_m + |beta s_{m,m}|.  Errors: EVSL_ERR_ARG,
 * EVSL_ERR_STATE without A or B or with orders that differ. */
int evsl_bounds_gen(evsl_ctx *ctx, int steps, uint64_t seed, double *lmin, double *lmax);

/* Filtered non-restart Lanczos for the pencil on [a, b] (Sec. 2.5 with Algorithm 3): the
 * operator rho((A B^{-1} - c I) / d) (pol built on the pencil's bounds; every filter degree is
 * one solve with p(B) and one product with A) applied in the B-inner product with two full
 * reorthogonalisation passes, at most opts->m steps.  Every opts->ncycle steps the sum of the
 * Ritz values >= pol->bar is compared with the previous one (relative change < opts->tau1
 * triggers an extraction); a run with no Ritz value >= bar for max(2 ncycle, m/4) steps ends
 * with none.  Extraction: x = W y with (x, B x) = 1, lambda = x^T A x, kept in the slice,
 * converged when ||A x - lambda B x|| <= tol * bmax * max(|lmin|, |lmax|); unconverged candidates
 * continue the basis.  Outputs as evsl_chebLanNr (ascending; Y host or device, n x cap, the
 * eigenvectors B-orthonormal); stats: niter, nmv (products with A), t_total.  FP64 only.
 * Errors: EVSL_ERR_ARG, EVSL_ERR_STATE (as evsl_bounds_gen), EVSL_ERR_NOCONV (basis limit with
 * unconverged candidates; the converged ones are returned), EVSL_ERR_CAPACITY. */
int evsl_chebLanNr_gen(evsl_ctx *ctx, double a, double b, const evsl_polfilt *pol,
                       const evsl_lan_opts *opts, int cap, int *nev, double *lam, double *Y,
                       double *res, evsl_stats *stats);

/* Filtered thick-restart Lanczos with locking for the pencil on [a, b] (Algorithm 2 in the
 * B-inner product; Sec. 2.5 describes the generalized TR and locking scheme, with deflation
 * (I - B U U^T) A x = lambda B x for the B-orthonormal locked vectors U).  Vectors are kept in
 * pairs (w, z = B w); the operator is evsl_chebLanNr_gen's; two reorthogonalisation passes against
 * the locked pairs and the basis.  Restarts keep at most opts->m / 2 unconverged Ritz pairs
 * (thick restart with the arrow matrix); early restart, candidates and locking as evsl_chebLanTr
 * with the residual of evsl_chebLanNr_gen; fresh start vectors after a breakdown or a cycle
 * without candidates, stop after two such cycles; opts->maxit bounds the Lanczos steps (0 = 20 m).
 * No refinement of stalled candidates.  Outputs, stats (niter, nmv, nrestart, t_total) and errors as
 * evsl_chebLanNr_gen. */
int evsl_chebLanTr_gen(evsl_ctx *ctx, double a, double b, const evsl_polfilt *pol,
                       const evsl_lan_opts *opts, int cap, int *nev, double *lam, double *Y,
                       double *res, evsl_stats *stats);

/* ---------------------------------------------------------------------------------------- */
/* Instrumentation (no counterpart in the paper).
 * evsl_launch_count: kernels launched by this context since its creation.
 * evsl_profile: 1 starts timing the launch groups of each kernel family with CUDA events on
 * the context's stream, 0 stops; evsl_profile_get returns, for family `kernel` (EVSL_K_*),
 * the launches timed and their summed device time in milliseconds since profiling started. */
typedef enum {
    EVSL_K_CHEB_STEP = 0,   /* fused Chebyshev filter step (SpMM + recurrence + axpy)   */
    EVSL_K_KPM_STEP = 1,    /* KPM moment step (SpMM + recurrence + probe dots)         */
    EVSL_K_REORTH = 2,      /* Gram-Schmidt projections against the basis               */
    EVSL_K_RITZ_GEMM = 3,   /* Ritz vectors Y = Q S                                     */
    EVSL_K_SMALL_EIG = 4,   /* Jacobi / bisection on the projected matrix               */
    EVSL_K_GEN_STEP = 5,    /* generalized filter degree steps (solve with B, product with A) */
    EVSL_K_COUNT = 6
} evsl_kernel_family;

int64_t evsl_launch_count(const evsl_ctx *ctx);
/* Device memory accounting (no counterpart in the paper; the paper notes that memory grows
 * with the number of eigenvalues a slice holds, Sec. 4.2, which is what admission must bound).
 * evsl_set_device_budget caps the device memory held by ALL of this library's contexts on CUDA
 * device `device` together (0 = no cap, the default): an allocation by any of them that would
 * pass it fails with EVSL_ERR_NOMEM, and evsl_batch_add refuses a job whose bases and step
 * workspaces would not fit.  It is checked in addition to each context's own budget; lowering it
 * frees nothing.  EVSL_ERR_ARG for a device ordinal outside [0, 64).  evsl_device_used: bytes
 * held by the library's contexts on that device; evsl_mem_used: bytes held by one context. */
int evsl_set_device_budget(int device, size_t bytes);
size_t evsl_device_used(int device);
size_t evsl_mem_used(const evsl_ctx *ctx);

/* Dense FP64 products (Algorithm 2's "compute candidate Ritz pairs" step forms Y = Q S; the
 * Rayleigh-Ritz and Gram projections form W^T Z): C {=, -=, +=} op(A) B for DEVICE column-major
 * FP64 matrices, op(A) = A (M x K, lda >= M) when trans_a = 0, op(A) = A^T (A is K x M,
 * lda >= K) when trans_a = 1; B is K x N (ldb >= K); C is M x N (ldc >= M); mode 0 stores,
 * 1 subtracts, 2 adds.  With the tensor-core path enabled (the default) the product runs on the
 * BF16 tensor cores by exact digit splitting (Ozaki scheme I: nine 6-bit digits per element
 * against per-row / per-column power-of-two scales, exact FP32 sums per 448-long chunk, exact
 * 128-bit integer accumulation across chunks) and is rounded once to FP64: each element is
 * within about 2^-52 of sum_k |a_ik| |b_kj| of the exact product, and the result does not
 * depend on the tiling.  The solvers use the same path for their large products
 * (2 M N K >= 1e9).  evsl_set_tensor_gemm(ctx, 0) switches them (and this call, mode 0 only)
 * to the plain FP64 kernels.  Synchronous.  Workspace: the digits of at most 2 GiB of operand
 * panels.  Errors: EVSL_ERR_ARG, EVSL_ERR_NOMEM, EVSL_ERR_TIMEOUT (a bounded wait inside the
 * kernel's pipeline expired; C is then unspecified). */
int evsl_dense_gemm(evsl_ctx *ctx, int trans_a, int64_t M, int N, int64_t K, const double *A, int64_t lda,
                    const double *B, int64_t ldb, double *C, int64_t ldc, int mode);
int evsl_set_tensor_gemm(evsl_ctx *ctx, int enable);
/* evsl_set_graphs: 1 (the default) lets single-vector filter applications replay cached CUDA
 * graphs; 0 drops the cached graphs and makes every application launch its kernels directly.
 * Both give bitwise the same results. */
int evsl_set_graphs(evsl_ctx *ctx, int enable);
int evsl_profile(evsl_ctx *ctx, int enable);
int evsl_profile_get(evsl_ctx *ctx, int kernel, int64_t *launches, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* EVSL_GB300_H */
