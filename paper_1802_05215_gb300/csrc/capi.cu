// C ABI entry points (include/evsl_gb300.h) and context services: error reporting, the
// HBM budget, grow-only workspaces and event-based kernel timing.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "evsl_internal.h"

int ctx_fail(evsl_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int ctx_cuda(evsl_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return ctx_fail(c, EVSL_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return ctx_fail(c, EVSL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int check_launch(evsl_ctx *c, const char *what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, what);
}

// Device-wide accounting: the bytes held by all contexts on one device, and an optional cap on
// them shared by those contexts (evsl_set_device_budget).
namespace {
constexpr int DEV_SLOTS = 64;
std::atomic<size_t> g_dev_budget[DEV_SLOTS];
std::atomic<size_t> g_dev_used[DEV_SLOTS];
inline bool dev_slot_ok(int d) { return d >= 0 && d < DEV_SLOTS; }
}  // namespace

size_t dev_budget_bytes(int device) { return dev_slot_ok(device) ? g_dev_budget[device].load() : 0; }
size_t dev_used_bytes(int device) { return dev_slot_ok(device) ? g_dev_used[device].load() : 0; }

int ctx_alloc(evsl_ctx *c, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return EVSL_OK;
    if (c->budget && c->used + bytes > c->budget)
        return ctx_fail(c, EVSL_ERR_NOMEM, "HBM budget exceeded (%zu + %zu > %zu bytes)", c->used,
                        bytes, c->budget);
    const bool slot = dev_slot_ok(c->device);
    if (slot) {
        // reserve the bytes against the device-wide budget before allocating
        const size_t cap = g_dev_budget[c->device].load();
        size_t cur = g_dev_used[c->device].load();
        do {
            if (cap && cur + bytes > cap)
                return ctx_fail(c, EVSL_ERR_NOMEM, "device HBM budget exceeded (%zu + %zu > %zu bytes)", cur,
                                bytes, cap);
        } while (!g_dev_used[c->device].compare_exchange_weak(cur, cur + bytes));
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        if (slot) g_dev_used[c->device] -= bytes;
        return ctx_fail(c, EVSL_ERR_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->used += bytes;
    return EVSL_OK;
}

void ctx_free(evsl_ctx *c, void *p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    c->used -= std::min(c->used, bytes);
    if (dev_slot_ok(c->device)) g_dev_used[c->device] -= bytes;
}

// Grow-only workspace: the returned buffer holds at least `bytes`; growing discards contents.
void *ctx_ws(evsl_ctx *c, int slot, size_t bytes, int *status)
{
    if (c->ws_ptr.size() < WS_COUNT) {
        c->ws_ptr.resize(WS_COUNT, nullptr);
        c->ws_bytes.resize(WS_COUNT, 0);
    }
    if (c->ws_bytes[slot] >= bytes && c->ws_ptr[slot]) return c->ws_ptr[slot];
    if (c->ws_ptr[slot]) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            *status = ctx_cuda(c, e, "workspace sync");
            return nullptr;
        }
        ctx_free(c, c->ws_ptr[slot], c->ws_bytes[slot]);
        c->ws_ptr[slot] = nullptr;
        c->ws_bytes[slot] = 0;
    }
    size_t want = bytes < 256 ? 256 : bytes;
    void *p = nullptr;
    int st = ctx_alloc(c, &p, want);
    if (st != EVSL_OK) {
        *status = st;
        return nullptr;
    }
    c->ws_ptr[slot] = p;
    c->ws_bytes[slot] = want;
    return p;
}

static cudaEvent_t take_event(evsl_ctx *c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static void prof_resolve(evsl_ctx *c)
{
    for (ProfGroup &g : c->prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(g.b) == cudaSuccess && cudaEventElapsedTime(&ms, g.a, g.b) == cudaSuccess) {
            c->prof_ms[g.family] += ms;
            c->prof_launches[g.family] += g.launches;
        }
        c->ev_pool.push_back(g.a);
        c->ev_pool.push_back(g.b);
    }
    c->prof_pending.clear();
}

void prof_begin(evsl_ctx *c, int family, ProfGroup *g)
{
    g->family = family;
    g->launches = 0;
    g->a = g->b = nullptr;
    if (!c->prof) return;
    g->a = take_event(c);
    g->b = take_event(c);
    cudaEventRecord(g->a, c->stream);
}

void prof_end(evsl_ctx *c, ProfGroup *g, int launches)
{
    if (!c->prof || !g->a) return;
    cudaEventRecord(g->b, c->stream);
    g->launches = launches;
    c->prof_pending.push_back(*g);
    if (c->prof_pending.size() > 4096) prof_resolve(c);
}

// ------------------------------------------------------------------------------------------
extern "C" {

int evsl_create(evsl_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out) return EVSL_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return EVSL_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return EVSL_ERR_CUDA;
    evsl_ctx *c = new evsl_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return EVSL_ERR_CUDA;
    }
    c->stream = c->own_stream;
    cudaDeviceGetAttribute(&c->dev_sm_count, cudaDevAttrMultiProcessorCount, device);
    if (c->dev_sm_count <= 0) c->dev_sm_count = 1;
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    c->l2_bytes = l2 > 0 ? l2 : 0;
    *out = c;
    return EVSL_OK;
}

void evsl_destroy(evsl_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    while (!c->batches.empty()) batch_destroy(c->batches.back());  // unfinished jobs are discarded
    cudaStreamSynchronize(c->stream);
    prof_resolve(c);
    sell_free(c);
    dev_matrix_free(c, c->B);
    filter_graphs_clear(c);
    for (size_t i = 0; i < c->ws_ptr.size(); i++) ctx_free(c, c->ws_ptr[i], c->ws_bytes[i]);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

const char *evsl_last_error(const evsl_ctx *c) { return c ? c->err.c_str() : "null context"; }

int evsl_set_stream(evsl_ctx *c, void *stream)
{
    if (!c) return EVSL_ERR_ARG;
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "set_stream");
    c->stream = stream ? (cudaStream_t)stream : c->own_stream;
    return EVSL_OK;
}

int evsl_set_csr(evsl_ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                 const double *val)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    cudaSetDevice(c->device);
    return sell_upload(c, n, row_ptr, col_idx, val);
}

int evsl_bounds(evsl_ctx *c, int steps, uint64_t seed, double *lmin, double *lmax)
{
    if (!c || !lmin || !lmax || steps < 2) return c ? ctx_fail(c, EVSL_ERR_ARG, "bounds: bad arguments") : EVSL_ERR_ARG;
    c->err.clear();
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "bounds: no matrix set");
    cudaSetDevice(c->device);
    return drv_bounds(c, steps, seed, lmin, lmax);
}

int evsl_kpm_dos(evsl_ctx *c, int degree, int nvec, uint64_t seed, double lmin, double lmax,
                 evsl_precision prec, double *mu)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!mu || degree < 0 || nvec < 1 || !(lmax > lmin) || (prec != EVSL_FP64 && prec != EVSL_FP32))
        return ctx_fail(c, EVSL_ERR_ARG, "kpm_dos: bad arguments");
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "kpm_dos: no matrix set");
    cudaSetDevice(c->device);
    return drv_kpm(c, degree, nvec, seed, lmin, lmax, prec, mu);
}

int evsl_kpm_dos_doubling(evsl_ctx *c, int degree, int nvec, uint64_t seed, double lmin, double lmax,
                          evsl_precision prec, double *mu)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!mu || degree < 0 || nvec < 1 || !(lmax > lmin) || (prec != EVSL_FP64 && prec != EVSL_FP32))
        return ctx_fail(c, EVSL_ERR_ARG, "kpm_dos_doubling: bad arguments");
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "kpm_dos_doubling: no matrix set");
    cudaSetDevice(c->device);
    return drv_kpm(c, degree, nvec, seed, lmin, lmax, prec, mu, true);
}

int evsl_kpm_probe_moments(evsl_ctx *c, int degree, int64_t first, int nprobe, uint64_t seed, double lmin,
                           double lmax, evsl_precision prec, double *out)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!out || degree < 0 || first < 0 || nprobe < 1 || !(lmax > lmin) || (prec != EVSL_FP64 && prec != EVSL_FP32))
        return ctx_fail(c, EVSL_ERR_ARG, "kpm_probe_moments: bad arguments");
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "kpm_probe_moments: no matrix set");
    cudaSetDevice(c->device);
    return drv_kpm_probe(c, degree, first, nprobe, seed, lmin, lmax, prec, out);
}

int evsl_slice_by_dos(const double *mu, int degree, int64_t n, double lmin, double lmax,
                      double xi, double eta, int nslices, int npts, double *sli, double *est)
{
    return host_slicer(mu, degree, n, lmin, lmax, xi, eta, nslices, npts, sli, est);
}

int evsl_cheb_filter_build(double a, double b, double lmin, double lmax,
                           const evsl_filter_opts *opts, evsl_polfilt *pol, double *coef, int cap)
{
    return host_filter_build(a, b, lmin, lmax, opts, pol, coef, cap);
}

int evsl_filter_apply(evsl_ctx *c, const evsl_polfilt *pol, int nvec, const double *X, double *Y,
                      evsl_precision prec)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!pol || !pol->coef || pol->deg < 0 || nvec < 1 || !X || !Y)
        return ctx_fail(c, EVSL_ERR_ARG, "filter_apply: bad arguments");
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "filter_apply: no matrix set");
    cudaSetDevice(c->device);
    return drv_filter_apply(c, pol, nvec, X, Y, prec);
}

int evsl_filter_apply_multi(evsl_ctx *c, int npol, const evsl_polfilt *pols, const double *X,
                            double *Y, evsl_precision prec)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!pols || npol < 1 || !X || !Y || (prec != EVSL_FP64 && prec != EVSL_FP32))
        return ctx_fail(c, EVSL_ERR_ARG, "filter_apply_multi: bad arguments");
    for (int t = 0; t < npol; t++)
        if (!pols[t].coef || pols[t].deg < 0)
            return ctx_fail(c, EVSL_ERR_ARG, "filter_apply_multi: filter %d has no coefficients", t);
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "filter_apply_multi: no matrix set");
    cudaSetDevice(c->device);
    return drv_filter_apply_multi(c, npol, pols, X, Y, prec);
}

int evsl_chebLanTr(evsl_ctx *c, double a, double b, const evsl_polfilt *pol,
                   const evsl_lan_opts *opts, int cap, int *nev, double *lam, double *Y,
                   double *res, evsl_stats *stats)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!pol || !pol->coef || !opts || !nev || !lam || !res || cap < 1 || !(b > a) || opts->m < 2)
        return ctx_fail(c, EVSL_ERR_ARG, "chebLanTr: bad arguments");
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "chebLanTr: no matrix set");
    cudaSetDevice(c->device);
    return drv_chebLanTr(c, a, b, pol, opts, cap, nev, lam, Y, res, stats);
}

int evsl_chebLanNr(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *opts,
                   int cap, int *nev, double *lam, double *Y, double *res, evsl_stats *stats)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!pol || !pol->coef || !opts || !nev || !lam || !res || cap < 1 || !(b > a) || opts->m < 2)
        return ctx_fail(c, EVSL_ERR_ARG, "chebLanNr: bad arguments");
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "chebLanNr: no matrix set");
    cudaSetDevice(c->device);
    return drv_chebLanTr(c, a, b, pol, opts, cap, nev, lam, Y, res, stats, true);
}

int evsl_landos(evsl_ctx *c, int m, int nvec, uint64_t seed, double *nodes, double *weights, int *mused)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (m < 1 || nvec < 1 || !nodes || !weights || !mused) return ctx_fail(c, EVSL_ERR_ARG, "landos: bad arguments");
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "landos: no matrix set");
    cudaSetDevice(c->device);
    return drv_landos(c, m, nvec, seed, nodes, weights, mused);
}

int evsl_slice_by_landos(const double *nodes, const double *weights, const int *mused, int m, int nvec,
                         int64_t n, double xi, double eta, int nslices, double *sli, double *est)
{
    if (!nodes || !weights || !mused || m < 1 || nvec < 1 || n < 1 || !(eta > xi) || nslices < 1 || !sli || !est)
        return EVSL_ERR_ARG;
    for (int l = 0; l < nvec; l++)
        if (mused[l] < 0 || mused[l] > m) return EVSL_ERR_ARG;
    return host_slicer_landos(nodes, weights, mused, m, nvec, n, xi, eta, nslices, sli, est);
}

int evsl_chebSI(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *opts,
                int cap, int *nev, double *lam, double *Y, double *res, evsl_stats *stats)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!pol || !pol->coef || !opts || !nev || !lam || !res || cap < 1 || !(b > a) || opts->m < 1)
        return ctx_fail(c, EVSL_ERR_ARG, "chebSI: bad arguments");
    if (opts->prec != EVSL_FP64) return ctx_fail(c, EVSL_ERR_ARG, "chebSI: only the FP64 filter is supported");
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "chebSI: no matrix set");
    cudaSetDevice(c->device);
    return drv_chebSI(c, a, b, pol, opts, cap, nev, lam, Y, res, stats);
}

int evsl_chebLanTr_batch(evsl_ctx *c, int njobs, evsl_slice_job *jobs, const evsl_lan_opts *opts)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (njobs < 1 || !jobs || !opts) return ctx_fail(c, EVSL_ERR_ARG, "chebLanTr_batch: bad arguments");
    for (int j = 0; j < njobs; j++) {
        const evsl_slice_job &J = jobs[j];
        if (!J.pol || !J.pol->coef || !J.nev || !J.lam || !J.res || J.cap < 1 || !(J.b > J.a) || J.m < 2)
            return ctx_fail(c, EVSL_ERR_ARG, "chebLanTr_batch: job %d has bad arguments", j);
        if (J.pol->lmin != jobs[0].pol->lmin || J.pol->lmax != jobs[0].pol->lmax)
            return ctx_fail(c, EVSL_ERR_ARG, "chebLanTr_batch: job %d uses another [lmin, lmax]", j);
        jobs[j].status = EVSL_OK;
        *J.nev = 0;
    }
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "chebLanTr_batch: no matrix set");
    cudaSetDevice(c->device);
    return drv_chebLanTr_batch(c, njobs, jobs, opts);
}

int evsl_batch_create(evsl_ctx *c, const evsl_lan_opts *opts, evsl_batch **batch)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!opts || !batch) return ctx_fail(c, EVSL_ERR_ARG, "batch_create: bad arguments");
    *batch = nullptr;
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "batch_create: no matrix set");
    cudaSetDevice(c->device);
    return batch_create(c, opts, batch);
}

int evsl_batch_add(evsl_batch *batch, evsl_slice_job *J)
{
    if (!batch) return EVSL_ERR_ARG;
    evsl_ctx *c = batch_ctx(batch);
    c->err.clear();
    if (!J || !J->pol || !J->pol->coef || !J->nev || !J->lam || !J->res || J->cap < 1 || !(J->b > J->a) || J->m < 2)
        return ctx_fail(c, EVSL_ERR_ARG, "batch_add: bad job");
    cudaSetDevice(c->device);
    return batch_add(batch, J);
}

int evsl_batch_step(evsl_batch *batch, int *nactive, int *nfinished)
{
    if (!batch) return EVSL_ERR_ARG;
    evsl_ctx *c = batch_ctx(batch);
    c->err.clear();
    cudaSetDevice(c->device);
    return batch_step(batch, nactive, nfinished);
}

void evsl_batch_destroy(evsl_batch *batch)
{
    if (!batch) return;
    cudaSetDevice(batch_ctx(batch)->device);
    batch_destroy(batch);
}

int64_t evsl_launch_count(const evsl_ctx *c) { return c ? c->launches : 0; }

int evsl_set_device_budget(int device, size_t bytes)
{
    if (!dev_slot_ok(device)) return EVSL_ERR_ARG;
    g_dev_budget[device] = bytes;
    return EVSL_OK;
}

size_t evsl_device_used(int device) { return dev_used_bytes(device); }

size_t evsl_mem_used(const evsl_ctx *c) { return c ? c->used : 0; }

int evsl_set_tensor_gemm(evsl_ctx *c, int enable)
{
    if (!c) return EVSL_ERR_ARG;
    c->tc_gemm = enable != 0;
    return EVSL_OK;
}

int evsl_dense_gemm(evsl_ctx *c, int trans_a, int64_t M, int N, int64_t K, const double *A, int64_t lda,
                    const double *B, int64_t ldb, double *C, int64_t ldc, int mode)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (M < 0 || N < 0 || K < 0 || mode < 0 || mode > 2 || (M > 0 && N > 0 && (!C || ldc < M)) ||
        (M > 0 && N > 0 && K > 0 && (!A || !B || ldb < K || lda < (trans_a ? K : M))))
        return ctx_fail(c, EVSL_ERR_ARG, "dense_gemm: bad arguments");
    cudaSetDevice(c->device);
    int st = c->tc_gemm ? gemm_tc(c, trans_a != 0, M, N, K, A, lda, B, ldb, C, ldc, mode)
                        : (mode == 0 ? (trans_a ? gemm_tn(c, K, (int)M, N, A, lda, B, ldb, C, ldc)
                                                : gemm_nn(c, M, N, (int)K, A, lda, B, ldb, C, ldc))
                                     : ctx_fail(c, EVSL_ERR_ARG, "dense_gemm: modes 1 and 2 need the tensor-core path"));
    if (st != EVSL_OK) return st;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "dense_gemm");
}

int evsl_profile(evsl_ctx *c, int enable)
{
    if (!c) return EVSL_ERR_ARG;
    cudaSetDevice(c->device);
    if (enable) {
        prof_resolve(c);
        for (int i = 0; i < EVSL_K_COUNT; i++) {
            c->prof_ms[i] = 0.0;
            c->prof_launches[i] = 0;
        }
        c->prof = true;
    } else {
        prof_resolve(c);
        c->prof = false;
    }
    return EVSL_OK;
}

int evsl_profile_get(evsl_ctx *c, int kernel, int64_t *launches, double *ms)
{
    if (!c || kernel < 0 || kernel >= EVSL_K_COUNT || !launches || !ms) return EVSL_ERR_ARG;
    cudaSetDevice(c->device);
    prof_resolve(c);
    *launches = c->prof_launches[kernel];
    *ms = c->prof_ms[kernel];
    return EVSL_OK;
}

// ---- generalized problems A x = lambda B x
int evsl_lspol(double bmin, double bmax, double eps, int maxdeg, int *deg, double *coef, int cap, double *err)
{
    if (!(bmin > 0.0) || !(bmax > bmin) || !(eps > 0.0) || maxdeg < 1 || !deg || !coef) return EVSL_ERR_ARG;
    if (cap < maxdeg + 1) {
        *deg = maxdeg;
        return EVSL_ERR_CAPACITY;
    }
    return host_lspol(bmin, bmax, eps, maxdeg, deg, coef, err);
}

int evsl_lspol_isqrt(double bmin, double bmax, double eps, int maxdeg, int *deg, double *coef, int cap, double *err)
{
    if (!(bmin > 0.0) || !(bmax > bmin) || !(eps > 0.0) || maxdeg < 1 || !deg || !coef) return EVSL_ERR_ARG;
    if (cap < maxdeg + 1) {
        *deg = maxdeg;
        return EVSL_ERR_CAPACITY;
    }
    return host_lspol(bmin, bmax, eps, maxdeg, deg, coef, err, 1);
}

int evsl_kpm_dos_gen(evsl_ctx *c, int degree, int nvec, uint64_t seed, double lmin, double lmax, double *mu)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (degree < 0 || nvec < 1 || !mu || !(lmax > lmin)) return ctx_fail(c, EVSL_ERR_ARG, "kpm_dos_gen: bad arguments");
    cudaSetDevice(c->device);
    return drv_kpm_gen(c, degree, nvec, seed, lmin, lmax, mu);
}

int evsl_set_csr_b(evsl_ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                   double bmin, double bmax, double eps, int maxdeg, int *deg, double *err)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!(bmin > 0.0) || !(bmax > bmin) || !(eps > 0.0) || maxdeg < 1)
        return ctx_fail(c, EVSL_ERR_ARG, "set_csr_b: need 0 < bmin < bmax, eps > 0 and maxdeg >= 1");
    std::vector<double> coef((size_t)maxdeg + 1), coef_s((size_t)maxdeg + 1);
    int d = 0, ds = 0;
    filter_graphs_clear(c);  // cached generalized-filter graphs hold B's device addresses
    double e = 0.0, es = 0.0;
    const int pst = host_lspol(bmin, bmax, eps, maxdeg, &d, coef.data(), &e);
    const int sst = host_lspol(bmin, bmax, eps, maxdeg, &ds, coef_s.data(), &es, 1);
    cudaSetDevice(c->device);
    EVSL_TRY(sell_upload_b(c, n, row_ptr, col_idx, val));
    coef.resize((size_t)d + 1);
    coef_s.resize((size_t)ds + 1);
    c->b_coef = coef;
    c->b_coef_isqrt = coef_s;
    c->b_min = bmin;
    c->b_max = bmax;
    EVSL_TRY(gen_map_b(c));
    if (deg) *deg = d;
    if (err) *err = e;
    if (pst != EVSL_OK) return ctx_fail(c, pst, "set_csr_b: degree %d reached with error %g > eps %g", d, e, eps);
    if (sst != EVSL_OK)
        return ctx_fail(c, sst, "set_csr_b: B^{-1/2} polynomial degree %d reached with error %g > eps %g", ds, es, eps);
    return EVSL_OK;
}

int evsl_polyB_apply(evsl_ctx *c, const double *x, double *y)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!x || !y || x == y) return ctx_fail(c, EVSL_ERR_ARG, "polyB_apply: bad arguments");
    cudaSetDevice(c->device);
    return drv_polyB_apply(c, x, y);
}

int evsl_bounds_gen(evsl_ctx *c, int steps, uint64_t seed, double *lmin, double *lmax)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!lmin || !lmax || steps < 2) return ctx_fail(c, EVSL_ERR_ARG, "bounds_gen: bad arguments");
    cudaSetDevice(c->device);
    return drv_bounds_gen(c, steps, seed, lmin, lmax);
}

int evsl_chebLanNr_gen(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *opts,
                       int cap, int *nev, double *lam, double *Y, double *res, evsl_stats *stats)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!pol || !pol->coef || pol->deg < 0 || !opts || !nev || !lam || !res || cap < 1 || !(b > a) || opts->m < 2 ||
        !(pol->lmax > pol->lmin))
        return ctx_fail(c, EVSL_ERR_ARG, "chebLanNr_gen: bad arguments");
    if (opts->prec != EVSL_FP64) return ctx_fail(c, EVSL_ERR_ARG, "chebLanNr_gen: only the FP64 filter is supported");
    cudaSetDevice(c->device);
    return drv_chebLanNr_gen(c, a, b, pol, opts, cap, nev, lam, Y, res, stats);
}

int evsl_chebLanTr_gen(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *opts,
                       int cap, int *nev, double *lam, double *Y, double *res, evsl_stats *stats)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!pol || !pol->coef || pol->deg < 0 || !opts || !nev || !lam || !res || cap < 1 || !(b > a) || opts->m < 2 ||
        !(pol->lmax > pol->lmin))
        return ctx_fail(c, EVSL_ERR_ARG, "chebLanTr_gen: bad arguments");
    if (opts->prec != EVSL_FP64) return ctx_fail(c, EVSL_ERR_ARG, "chebLanTr_gen: only the FP64 filter is supported");
    cudaSetDevice(c->device);
    return drv_chebLanTr_gen(c, a, b, pol, opts, cap, nev, lam, Y, res, stats);
}

int evsl_landos_gen(evsl_ctx *c, int m, int nvec, uint64_t seed, double *nodes, double *weights, int *mused)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (m < 1 || nvec < 1 || !nodes || !weights || !mused) return ctx_fail(c, EVSL_ERR_ARG, "landos_gen: bad arguments");
    cudaSetDevice(c->device);
    return drv_landos_gen(c, m, nvec, seed, nodes, weights, mused);
}

int evsl_set_graphs(evsl_ctx *c, int enable)
{
    if (!c) return EVSL_ERR_ARG;
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "set_graphs");
    if (!enable) filter_graphs_clear(c);
    c->graphs_off = !enable;
    return EVSL_OK;
}

}  // extern "C"
