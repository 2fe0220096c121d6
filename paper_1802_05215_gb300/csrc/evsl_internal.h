// Internal declarations of the GB300 spectrum-slicing library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <map>
#include <vector>

#include "../../include/evsl_gb300.h"

// SplitMix64 stream tags (must agree with the seeded-input definition used by callers).
enum { SM_STREAM_ANDERSON = 1, SM_STREAM_KPM = 2, SM_STREAM_LANCZOS = 3, SM_STREAM_BOUNDS = 4,
       SM_STREAM_LANDOS = 5 };

constexpr int SELL_C = 32;  // rows per ELLPACK slice (one warp)

// Device copy of the symmetric matrix in sliced ELLPACK form, 32-row slices, unsorted (the
// CSR row order is kept).  Slice s holds rows [32 s, 32 s + 32); its entries are stored
// column-major inside the slice: element j of lane l sits at sptr[s] + 32 j + l.  Padding
// entries have value 0 and repeat a valid column index of the same row.
struct DevMatrix {
    int64_t n = 0, nnz = 0, nslices = 0, nstored = 0;
    int maxw = 0;
    int64_t *sptr = nullptr;     // nslices + 1 offsets (elements)
    int32_t *col = nullptr;      // nstored
    double *val = nullptr;       // nstored
    float *val32 = nullptr;      // nstored
    int32_t *rlen = nullptr;     // n: stored (non-padding) entries of each row
    bool has_diag = false;       // every row stores its diagonal entry
    // mapped copy (2/d)(A - c I) of the values for the filter recurrence, for one (c, d)
    double *vhat = nullptr;
    float *vhat32 = nullptr;
    double hat_c = 0.0, hat_d = 0.0;
};

struct ProfGroup {
    cudaEvent_t a, b;
    int family;
    int launches;
};

struct evsl_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    size_t budget = 0, used = 0;
    std::string err;
    int64_t launches = 0;
    DevMatrix A;
    // generalized problems A x = lambda B x: the mass matrix and p(t) ~ 1/t on [b_min, b_max]
    // (Chebyshev coefficients, degree b_coef.size() - 1)
    DevMatrix B;
    double b_min = 0.0, b_max = 0.0;
    std::vector<double> b_coef;
    std::vector<double> b_coef_isqrt;  // q(t) ~ t^{-1/2} on the same interval (density of the pencil)
    // grow-only workspaces, indexed by WS_* slots
    std::vector<void *> ws_ptr;
    std::vector<size_t> ws_bytes;
    // profiling
    bool prof = false;
    std::vector<ProfGroup> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    int64_t prof_launches[EVSL_K_COUNT] = {0};
    double prof_ms[EVSL_K_COUNT] = {0};
    int dev_sm_count = 0;
    int64_t l2_bytes = 0;               // the device's L2 size
    std::vector<evsl_batch *> batches;  // live batches, destroyed with the context
    // CUDA graphs of single-vector filter applications, keyed by filter, buffers and matrix
    struct FilterGraph {
        uint64_t key = 0;
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;  // kernels in the graph
    };
    std::vector<FilterGraph> fgraphs;
    bool graphs_off = false;  // set when capture is not possible on the context's stream
    bool tc_gemm = true;      // large FP64 GEMMs on the tensor cores (digit splitting)
    // autotuned tile shape of the multi-column filter step, per (n, columns, precision)
    std::map<uint64_t, int> tune;
};

// autotuner of the multi-column filter step (kernels_sparse.cu): times the tile shapes on the
// block X once per (matrix, nvec, precision); tune_lookup gives the chosen shape (0 = default)
int tune_block_f64(evsl_ctx *c, int nvec, const double *X);
int tune_block_f32(evsl_ctx *c, int nvec, const float *X);
int tune_lookup(evsl_ctx *c, int nvec, int bytes);

// drop the cached filter graphs (they hold device addresses of the matrix and workspaces)
void filter_graphs_clear(evsl_ctx *c);
// Replays the cached graph `key` (capturing the kernel launches of issue() on the context's
// stream the first time), timed as one group of `launches` launches of `family`.  Returns 1
// when graphs cannot be used (the stream is being captured by the caller, or capture failed):
// the caller then launches directly.
int graph_replay(evsl_ctx *c, uint64_t key, int family, int launches, const std::function<int()> &issue);
// FNV-1a step for graph keys
uint64_t graph_key_hash(uint64_t h, const void *p, size_t len);

enum WsSlot {
    WS_PARTIAL = 0, WS_SCAL, WS_W0, WS_W1, WS_W2, WS_KPM_PART, WS_F32_X, WS_F32_Y,
    WS_LAN_U, WS_LAN_Q, WS_LAN_Y, WS_LAN_Z, WS_LAN_VEC, WS_LAN_T, WS_LAN_S, WS_LAN_IDX,
    WS_JAC_PAIRS, WS_BIS, WS_TMP_STAGE, WS_LAN_G, WS_POL_V, WS_POL_W, WS_POL_B, WS_POL_S, WS_POL_Y, WS_POL_R, WS_TUNE, WS_POL_H,
    WS_GEN_BASIS, WS_GEN_VEC, WS_GEN_SCAL, WS_GEN_MU,
    WS_OZ_A, WS_OZ_B, WS_OZ_E, WS_OZ_FLAG,
    WS_COUNT
};

// ---- context helpers (capi.cu)
int ctx_fail(evsl_ctx *c, int code, const char *fmt, ...);
int ctx_cuda(evsl_ctx *c, cudaError_t e, const char *what);
void *ctx_ws(evsl_ctx *c, int slot, size_t bytes, int *status);
int ctx_alloc(evsl_ctx *c, void **p, size_t bytes);
void ctx_free(evsl_ctx *c, void *p, size_t bytes);
// device-wide budget (0 = none) and the bytes all contexts hold on a device
size_t dev_budget_bytes(int device);
size_t dev_used_bytes(int device);
// profiling: begin/end a group of `launches` launches of one kernel family
void prof_begin(evsl_ctx *c, int family, ProfGroup *g);
void prof_end(evsl_ctx *c, ProfGroup *g, int launches);
int check_launch(evsl_ctx *c, const char *what);

// ---- sparse kernels (kernels_sparse.cu)
int sell_upload(evsl_ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col,
                const double *val);
void sell_free(evsl_ctx *c);
// the mass matrix B of a generalized problem, in the same layout (c->B)
int sell_upload_b(evsl_ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col,
                  const double *val);
void dev_matrix_free(evsl_ctx *c, DevMatrix &M);
// One fused Chebyshev step on nvec columns (ld = n).  mode 0: out = sc (A x - cc x),
// y = c0 x + cj out.  mode 1: out = sc (A x - cc x) - xprev, y += cj out.  out may alias xprev.
// hat = true uses the mapped values made current by ensure_mapped(c, cc, d) (same result up to
// rounding, two FP64 operations fewer per row).
int cheb_step_f64(evsl_ctx *c, int mode, int nvec, const double *x, const double *xprev,
                  double *out, double *y, double cc, double sc, double c0, double cj, bool hat);
int cheb_step_f32(evsl_ctx *c, int mode, int nvec, const float *x, const float *xprev,
                  float *out, float *y, double cc, double sc, double c0, double cj, bool hat);
// Multi-filter form: column l uses coefficient ctab[l] (and c0tab[l] in mode 0), device tables
int cheb_step_multi_f64(evsl_ctx *c, int mode, int nvec, const double *x, const double *xprev,
                        double *out, double *y, double cc, double sc, const double *ctab,
                        const double *c0tab, bool hat);
int cheb_step_multi_f32(evsl_ctx *c, int mode, int nvec, const float *x, const float *xprev,
                        float *out, float *y, double cc, double sc, const float *ctab,
                        const float *c0tab, bool hat);
// Make the mapped values (2/d)(A - cc I) current; returns false when the matrix lacks stored
// diagonal entries (the unscaled kernels are used then).
bool ensure_mapped(evsl_ctx *c, double cc, double d, int *status);
// Y = A X (FP64), nvec columns
int spmv_f64(evsl_ctx *c, int nvec, const double *X, double *Y);
// KPM: fill W0 with the probes, then steps
// KPM probe blocks are row-major with leading dimension kpm_ld(nvec) (nvec rounded up to 4)
int kpm_ld(int nvec);
// probes first .. first + nvec - 1 (global probe indices of the KPM random stream)
int kpm_init_f64(evsl_ctx *c, int nvec, uint64_t seed, double *W0, uint64_t first = 0);
int kpm_init_f32(evsl_ctx *c, int nvec, uint64_t seed, float *W0, uint64_t first = 0);
// out[l] = sum_r v_l[r] W[r, l] for the np probes of the block made by kpm_init (fixed order per
// probe); part: kpm_probe_dot_blocks(c) * np doubles of scratch
int kpm_probe_dots_f64(evsl_ctx *c, int np, const double *W, double *part, double *out);
int kpm_probe_dots_f32(evsl_ctx *c, int np, const float *W, double *part, double *out);
int kpm_probe_dot_blocks(evsl_ctx *c);
int drv_kpm_probe(evsl_ctx *c, int degree, int64_t first, int nprobe, uint64_t seed, double lmin, double lmax,
                  evsl_precision prec, double *out);
// mode 0: out = (A x - cc x) sc; mode 1: out = (A x - cc x) sc - xprev.  Writes, for moment
// index k, per-block partial sums of sum_l sum_i v_l[i] out_l[i] into part + k*nblk.
int kpm_step_f64(evsl_ctx *c, int mode, int nvec, uint64_t seed, const double *x,
                 const double *xprev, double *out, double cc, double sc, double *part, int k,
                 int nblk, bool hat,
                 bool dbl = false);
int kpm_step_f32(evsl_ctx *c, int mode, int nvec, uint64_t seed, const float *x,
                 const float *xprev, float *out, double cc, double sc, double *part, int k,
                 int nblk, bool hat,
                 bool dbl = false);
bool stream_matrix(const evsl_ctx *c, int64_t nstored, int64_t n, int value_bytes);
int kpm_nblocks(evsl_ctx *c);
int convert_f64_to_f32(evsl_ctx *c, int64_t count, const double *x, float *y);
int convert_f32_to_f64(evsl_ctx *c, int64_t count, const float *x, double *y);
int fill_uniform_f64(evsl_ctx *c, int64_t n, uint64_t seed, int stream, uint64_t index,
                     double *x);
// x[i] = +-1 by the top bit of draw(seed, stream, index*n + i) (KPM probe `index`)
int fill_rademacher_f64(evsl_ctx *c, int64_t n, uint64_t seed, int stream, uint64_t index,
                        double *x);

// ---- dense kernels (kernels_dense.cu)
// Deterministic reductions: partial sums per row chunk, then a fixed-order sum per output.
int64_t red_nchunks(int64_t n);
// out[j] = sum_c part[j * nch + c], j < k, fixed summation order
int reduce_rows(evsl_ctx *c, int k, int64_t nch, const double *part, double *out);
// out[j] = sum_r X[r,j] Y[r,j], j < k (device out)
int coldot(evsl_ctx *c, int64_t n, int k, const double *X, int64_t ldx, const double *Y,
           int64_t ldy, double *out);
// out[j] = || Z[:,j] - lam[j] Y[:,j] ||^2 (lam device)
int colres2(evsl_ctx *c, int64_t n, int k, const double *Z, const double *Y, int64_t ld,
            const double *lam, double *out);
// z = y - beta * qprev (qprev may be null); out[0] = q . z
int lan_three_term(evsl_ctx *c, int64_t n, const double *y, const double *qprev, double beta,
                   const double *q, double *z, double *out_dot);
// z -= (*alpha) q ; out[0] = ||z||^2  (alpha device scalar)
int lan_sub_alpha(evsl_ctx *c, int64_t n, double *z, const double *q, const double *alpha,
                  double *out_nrm2);
// h = [B1 B2]^T z  (h device, length k1 + k2)
int gemv_t2(evsl_ctx *c, int64_t n, const double *B1, int k1, const double *B2, int k2,
            const double *z, double *h);
// z -= [B1 B2] h ; out[0] = ||z||^2
int gemv_n2(evsl_ctx *c, int64_t n, const double *B1, int k1, const double *B2, int k2,
            const double *h, double *z, double *out_nrm2);
// x *= s (device scalar pointer or host value)
int scale_vec(evsl_ctx *c, int64_t n, double *x, double s, double *dst);
// Y[:, j] *= 1/sqrt(nrm2[j])
int colscale_inv_sqrt(evsl_ctx *c, int64_t n, int k, double *Y, const double *nrm2);
// C (n x l) = A (n x k, lda) * B (k x l, ldb)
int gemm_nn(evsl_ctx *c, int64_t n, int l, int k, const double *A, int64_t lda,
            const double *B, int64_t ldb, double *C, int64_t ldc);
// C -= A B (same shapes as gemm_nn)
int gemm_nn_sub(evsl_ctx *c, int64_t n, int l, int k, const double *A, int64_t lda,
                const double *B, int64_t ldb, double *C, int64_t ldc);
// Y[:, j] *= scale[j] (rows x k, ld rows), scale device
int colscale(evsl_ctx *c, int64_t rows, int k, double *Y, const double *scale);
// C (p x q, ldc) = A^T B, A: n x p (lda), B: n x q (ldb); split over rows, fixed-order sums
int gemm_tn(evsl_ctx *c, int64_t n, int p, int q, const double *A, int64_t lda,
            const double *B, int64_t ldb, double *C, int64_t ldc);
// dst[:, t] = src[:, idx[t]] (columns of length rows), idx device
int gather_cols(evsl_ctx *c, int64_t rows, int k, const double *src, int64_t lds,
                const int *idx, double *dst, int64_t ldd);
// FP64-accurate GEMM on the tensor cores (ozaki_gemm.cu): C (M x N, ldc) {=, -=, +=} op(A) B with
// op(A) = A (M x K, lda) or A^T (A K x M, lda), B K x N (ldb); mode 0 store, 1 subtract, 2 add.
// Synchronous (reads back the pipeline's timeout flag).
int gemm_tc(evsl_ctx *c, bool trans_a, int64_t M, int N, int64_t K, const double *A, int64_t lda, const double *B,
            int64_t ldb, double *C, int64_t ldc, int mode);
// Jacobi eigensolver for a dense symmetric m x m matrix (device, col-major, ld m).
// On return Tm's diagonal holds eigenvalues, V (ld M, M = m rounded to even) the vectors.
int jacobi_eig(evsl_ctx *c, int m, const double *Tdev_in, double *w_host, double *V, int *ldv,
               int *sweeps);
// eigenvalues k0..k1-1 (ascending index) of the arrow+tridiagonal matrix: diag d[k],
// e[i] (i < l: coupling of i with l; i >= l: coupling of i with i+1)
int bisect_eigs(evsl_ctx *c, int k, int l, const double *d_host, const double *e_host,
                int k0, int k1, double lo, double hi, double *w_host);

// ---- host-side numerics (host_filter.cpp)
int host_filter_build(double a, double b, double lmin, double lmax, const evsl_filter_opts *o,
                      evsl_polfilt *pol, double *coef, int cap);
int host_slicer(const double *mu, int degree, int64_t n, double lmin, double lmax, double xi,
                double eta, int ns, int npts, double *sli, double *est);
// number of eigenvalues < sigma of the arrow + tridiagonal matrix (Sylvester inertia)
int host_count_below(int k, int l, const double *d, const double *e, double sigma);

// ---- drivers (lanczos.cu, tr_lanczos.cu)
int filter_apply_dev(evsl_ctx *c, const evsl_polfilt *pol, int nvec, const double *X, double *Y,
                     evsl_precision prec, double *B0, double *B1, float *fbuf);
int filter_apply_multi_dev(evsl_ctx *c, int npol, const evsl_polfilt *pols, const double *X,
                           double *Y, evsl_precision prec);
int drv_chebLanTr_batch(evsl_ctx *c, int njobs, evsl_slice_job *jobs, const evsl_lan_opts *o);
int drv_landos(evsl_ctx *c, int m, int nvec, uint64_t seed, double *nodes, double *weights, int *mused);
int host_slicer_landos(const double *nodes, const double *weights, const int *mused, int m, int nvec,
                       int64_t n, double xi, double eta, int ns, double *sli, double *est);
int drv_chebSI(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *o, int cap,
               int *nev, double *lam, double *Y, double *res, evsl_stats *st);
int batch_create(evsl_ctx *c, const evsl_lan_opts *o, evsl_batch **out);
void batch_destroy(evsl_batch *bt);
int batch_add(evsl_batch *bt, evsl_slice_job *job);
int batch_step(evsl_batch *bt, int *nactive, int *nfinished);
evsl_ctx *batch_ctx(evsl_batch *bt);
int drv_bounds(evsl_ctx *c, int steps, uint64_t seed, double *lmin, double *lmax);
int drv_chebLanTr(evsl_ctx *c, double a, double b, const evsl_polfilt *pol,
                  const evsl_lan_opts *o, int cap, int *nev, double *lam, double *Y,
                  double *res, evsl_stats *st, bool nonrestart = false);
int drv_filter_apply(evsl_ctx *c, const evsl_polfilt *pol, int nvec, const double *X,
                     double *Y, evsl_precision prec);
int drv_filter_apply_multi(evsl_ctx *c, int npol, const evsl_polfilt *pols, const double *X,
                           double *Y, evsl_precision prec);
// generalized problems (generalized.cu)
// kind 0: p(t) ~ 1/t; kind 1: p(t) ~ t^{-1/2}
int host_lspol(double bmin, double bmax, double eps, int maxdeg, int *deg, double *coef, double *err, int kind = 0);
int gen_map_b(evsl_ctx *c);
int drv_polyB_apply(evsl_ctx *c, const double *x, double *y);
int drv_kpm_gen(evsl_ctx *c, int degree, int nvec, uint64_t seed, double lmin, double lmax, double *mu);
int drv_landos_gen(evsl_ctx *c, int m, int nvec, uint64_t seed, double *nodes, double *weights, int *mused);
int drv_chebLanTr_gen(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *o,
                      int cap, int *nev, double *lam, double *Y, double *res, evsl_stats *st);
int drv_bounds_gen(evsl_ctx *c, int steps, uint64_t seed, double *lmin, double *lmax);
int drv_chebLanNr_gen(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *o,
                      int cap, int *nev, double *lam, double *Y, double *res, evsl_stats *st);
int drv_kpm(evsl_ctx *c, int degree, int nvec, uint64_t seed, double lmin, double lmax,
            evsl_precision prec, double *mu,
            bool doubling = false);

#define EVSL_TRY(expr)                  \
    do {                                \
        int _st = (expr);               \
        if (_st != EVSL_OK) return _st; \
    } while (0)
