// Drivers of the hot path: spectral bounds (Sec. 2.2.1), KPM moments (Sec. 2.1), filter
// application (Eq. (2.4)) and filtered thick-restart Lanczos with locking (Algorithm 2).
// All vector work runs in the kernels of kernels_sparse.cu / kernels_dense.cu on the
// context's stream; the host keeps only the small projected matrix and the control flow.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "evsl_internal.h"

namespace {

constexpr double DGKS_ETA2 = 0.5;  // (1/sqrt(2))^2: second Gram-Schmidt pass when ||z'||^2 < 0.5 ||z||^2

struct Scal {  // device scalar area layout (doubles)
    enum { ALPHA = 0, NRM_BEFORE = 1, NRM_AFTER = 2, NRM_Y = 3, TMP = 4, H = 16 };
};

int d2h(evsl_ctx *c, void *dst, const void *src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "device-to-host copy");
}

int h2d(evsl_ctx *c, void *dst, const void *src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "host-to-device copy");
}

}  // namespace

// Y = rho(Ahat) X on nvec columns with the three-term recurrence; one fused launch per degree.
// B0, B1: n*nvec FP64 temporaries; fbuf: 4*n*nvec floats (FP32 mode only).  Asynchronous.
namespace {

constexpr int GRAPH_MIN_DEG = 8;   // filters of lower degree launch directly
constexpr size_t GRAPH_CACHE = 16;  // graphs kept per context (oldest dropped first)

uint64_t fnv1a(uint64_t h, const void *p, size_t len)
{
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < len; i++) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

// Issues the recurrence of one filter application on one vector whose input already sits in
// the second recurrence buffer (FP64: B1; FP32: f1): the same kernels, arguments and buffer
// rotation as the direct path (from degree 2 on, the direct path also writes w_{j+1} over
// w_{j-1}), so both give identical results.
int issue_filter_staged(evsl_ctx *c, const evsl_polfilt *pol, double *Y, evsl_precision prec, double *B0,
                        double *B1, float *fbuf, bool hat)
{
    const int64_t n = c->A.n;
    const double cc = 0.5 * (pol->lmax + pol->lmin), d = 0.5 * (pol->lmax - pol->lmin);
    const double *coef = pol->coef;
    if (prec == EVSL_FP64) {
        EVSL_TRY(cheb_step_f64(c, 0, 1, B1, nullptr, B0, Y, cc, 1.0 / d, coef[0], coef[1], hat));
        double *prev = B1, *cur = B0;
        for (int j = 2; j <= pol->deg; j++) {
            EVSL_TRY(cheb_step_f64(c, 1, 1, cur, prev, prev, Y, cc, 2.0 / d, 0.0, coef[j], hat));
            std::swap(prev, cur);
        }
        return EVSL_OK;
    }
    float *f0 = fbuf + n, *f1 = fbuf + 2 * n, *fy = fbuf + 3 * n;
    EVSL_TRY(cheb_step_f32(c, 0, 1, f1, nullptr, f0, fy, cc, 1.0 / d, coef[0], coef[1], hat));
    float *prev = f1, *cur = f0;
    for (int j = 2; j <= pol->deg; j++) {
        EVSL_TRY(cheb_step_f32(c, 1, 1, cur, prev, prev, fy, cc, 2.0 / d, 0.0, coef[j], hat));
        std::swap(prev, cur);
    }
    return convert_f32_to_f64(c, n, fy, Y);
}

// Replays the cached CUDA graph with key h, capturing it from issue() (kernel launches only,
// on the context's stream) the first time.  The launches are timed as one filter group of
// `degree` steps.  Returns 1 if graphs cannot be used here (the caller then launches directly).
template <typename F>
int launch_graph(evsl_ctx *c, uint64_t h, int degree, F issue, int family = EVSL_K_CHEB_STEP)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return 1;
    }
    cudaGraphExec_t exec = nullptr;
    int64_t nl = 0;
    for (auto &g : c->fgraphs)
        if (g.key == h) {
            exec = g.exec;
            nl = g.launches;
        }
    if (!exec) {
        const int64_t launches0 = c->launches;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->graphs_off = true;
            return 1;
        }
        int st = issue();
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(c->stream, &graph);
        nl = c->launches - launches0;
        c->launches = launches0;
        if (st != EVSL_OK || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            if (st != EVSL_OK) return st;
            c->graphs_off = true;
            return 1;
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->graphs_off = true;
            return 1;
        }
        if (c->fgraphs.size() >= GRAPH_CACHE) {
            cudaGraphExecDestroy(c->fgraphs.front().exec);
            c->fgraphs.erase(c->fgraphs.begin());
        }
        c->fgraphs.push_back({h, exec, nl});
    }
    ProfGroup g;
    prof_begin(c, family, &g);
    cudaError_t e = cudaGraphLaunch(exec, c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "filter graph launch");
    c->launches += nl;
    prof_end(c, &g, degree);
    return EVSL_OK;
}

// Single-vector filter application through a cached CUDA graph of its deg (+1) launches; the
// input is copied (FP64) or converted (FP32) into the second recurrence buffer first.
// Returns 1 if graphs cannot be used here (the caller then launches directly).
int filter_apply_graph(evsl_ctx *c, const evsl_polfilt *pol, const double *X, double *Y, evsl_precision prec,
                       double *B0, double *B1, float *fbuf, bool hat)
{
    const int64_t n = c->A.n;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return 1;
    }
    uint64_t h = 1469598103934665603ull;
    const void *ptrs[] = {Y, B0, B1, fbuf, c->A.sptr, c->A.col, c->A.val, c->A.val32, c->A.vhat, c->A.vhat32};
    h = fnv1a(h, ptrs, sizeof(ptrs));
    const int64_t meta[] = {n, pol->deg, (int64_t)prec, (int64_t)hat};
    h = fnv1a(h, meta, sizeof(meta));
    const double dm[] = {pol->lmin, pol->lmax};
    h = fnv1a(h, dm, sizeof(dm));
    h = fnv1a(h, pol->coef, sizeof(double) * (size_t)(pol->deg + 1));
    // stage the input
    if (prec == EVSL_FP64) {
        cudaError_t e = cudaMemcpyAsync(B1, X, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "filter input staging");
    } else {
        EVSL_TRY(convert_f64_to_f32(c, n, X, fbuf + 2 * n));
    }
    return launch_graph(c, h, pol->deg, [&]() { return issue_filter_staged(c, pol, Y, prec, B0, B1, fbuf, hat); });
}

// The recurrence of a multi-slice filter application on the degree-sorted block Xs (the
// coefficient tables at dtab, active[j] columns still running at degree j), into Ys.
int issue_filter_multi(evsl_ctx *c, int npol, const std::vector<int> &active, int maxdeg, const double *Xs,
                       double *Ys, const void *dtab, evsl_precision prec, bool hat, double cc, double d,
                       double *B0, double *B1, float *fb)
{
    const int64_t N = c->A.n * (int64_t)npol;
    if (prec == EVSL_FP64) {
        const double *t64 = (const double *)dtab;
        EVSL_TRY(cheb_step_multi_f64(c, 0, npol, Xs, nullptr, B0, Ys, cc, 1.0 / d, t64 + npol, t64, hat));
        const double *prev = Xs;
        double *cur = B0;
        for (int j = 2; j <= maxdeg; j++) {
            double *out = (j == 2) ? B1 : const_cast<double *>(prev);
            EVSL_TRY(cheb_step_multi_f64(c, 1, active[j], cur, prev, out, Ys, cc, 2.0 / d,
                                         t64 + (size_t)j * npol, nullptr, hat));
            prev = cur;
            cur = out;
        }
        return EVSL_OK;
    }
    float *fx = fb, *f0 = fb + N, *f1 = fb + 2 * N, *fy = fb + 3 * N;
    const float *t32 = (const float *)dtab;
    EVSL_TRY(convert_f64_to_f32(c, N, Xs, fx));
    EVSL_TRY(cheb_step_multi_f32(c, 0, npol, fx, nullptr, f0, fy, cc, 1.0 / d, t32 + npol, t32, hat));
    const float *prev = fx;
    float *cur = f0;
    for (int j = 2; j <= maxdeg; j++) {
        float *out = (j == 2) ? f1 : const_cast<float *>(prev);
        EVSL_TRY(cheb_step_multi_f32(c, 1, active[j], cur, prev, out, fy, cc, 2.0 / d,
                                     t32 + (size_t)j * npol, nullptr, hat));
        prev = cur;
        cur = out;
    }
    return convert_f32_to_f64(c, N, fy, Ys);
}

}  // namespace

int graph_replay(evsl_ctx *c, uint64_t key, int family, int launches, const std::function<int()> &issue)
{
    return launch_graph(c, key, launches, [&]() { return issue(); }, family);
}

uint64_t graph_key_hash(uint64_t h, const void *p, size_t len) { return fnv1a(h, p, len); }

void filter_graphs_clear(evsl_ctx *c)
{
    for (auto &g : c->fgraphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    c->fgraphs.clear();
}

int filter_apply_dev(evsl_ctx *c, const evsl_polfilt *pol, int nvec, const double *X, double *Y,
               evsl_precision prec, double *B0, double *B1, float *fbuf)
{
    const int64_t n = c->A.n, N = n * (int64_t)nvec;
    const double cc = 0.5 * (pol->lmax + pol->lmin), d = 0.5 * (pol->lmax - pol->lmin);
    const double *coef = pol->coef;
    const int deg = pol->deg;
    if (deg == 0) return scale_vec(c, N, const_cast<double *>(X), coef[0], Y);
    int st = EVSL_OK;
    const bool hat = ensure_mapped(c, cc, d, &st);
    if (st) return st;
    if (nvec > 1) {
        // tile shape of the block step (timed once per matrix, width and precision)
        if (prec == EVSL_FP64) EVSL_TRY(tune_block_f64(c, nvec, X));
        else EVSL_TRY(tune_block_f32(c, nvec, fbuf));
    }
    if (nvec == 1 && deg >= GRAPH_MIN_DEG && !c->graphs_off && X != B1 && X != B0 && X != Y) {
        const int r = filter_apply_graph(c, pol, X, Y, prec, B0, B1, fbuf, hat);
        if (r != 1) return r;
    }
    ProfGroup g;
    if (prec == EVSL_FP64) {
        prof_begin(c, EVSL_K_CHEB_STEP, &g);
        EVSL_TRY(cheb_step_f64(c, 0, nvec, X, nullptr, B0, Y, cc, 1.0 / d, coef[0], coef[1], hat));
        const double *prev = X;
        double *cur = B0;
        for (int j = 2; j <= deg; j++) {
            double *out = (j == 2) ? B1 : const_cast<double *>(prev);
            EVSL_TRY(cheb_step_f64(c, 1, nvec, cur, prev, out, Y, cc, 2.0 / d, 0.0, coef[j], hat));
            prev = cur;
            cur = out;
        }
        prof_end(c, &g, deg);
        return EVSL_OK;
    }
    float *fx = fbuf, *f0 = fbuf + N, *f1 = fbuf + 2 * N, *fy = fbuf + 3 * N;
    EVSL_TRY(convert_f64_to_f32(c, N, X, fx));
    prof_begin(c, EVSL_K_CHEB_STEP, &g);
    EVSL_TRY(cheb_step_f32(c, 0, nvec, fx, nullptr, f0, fy, cc, 1.0 / d, coef[0], coef[1], hat));
    const float *prev = fx;
    float *cur = f0;
    for (int j = 2; j <= deg; j++) {
        float *out = (j == 2) ? f1 : const_cast<float *>(prev);
        EVSL_TRY(cheb_step_f32(c, 1, nvec, cur, prev, out, fy, cc, 2.0 / d, 0.0, coef[j], hat));
        prev = cur;
        cur = out;
    }
    prof_end(c, &g, deg);
    return convert_f32_to_f64(c, N, fy, Y);
}

namespace {

// One classical Gram-Schmidt pass of z against [B1 (k1 cols), B2 (k2 cols)].
int cgs_pass(evsl_ctx *c, double *z, const double *B1, int k1, const double *B2, int k2,
             double *h, double *nrm2_out)
{
    const int64_t n = c->A.n;
    EVSL_TRY(gemv_t2(c, n, B1, k1, B2, k2, z, h));
    return gemv_n2(c, n, B1, k1, B2, k2, h, z, nrm2_out);
}

}  // namespace

// ------------------------------------------------------------------------------------------
int drv_filter_apply(evsl_ctx *c, const evsl_polfilt *pol, int nvec, const double *X, double *Y,
                     evsl_precision prec)
{
    const int64_t N = c->A.n * (int64_t)nvec;
    int st = EVSL_OK;
    double *B0 = (double *)ctx_ws(c, WS_W0, sizeof(double) * N, &st);
    if (st) return st;
    double *B1 = (double *)ctx_ws(c, WS_W1, sizeof(double) * N, &st);
    if (st) return st;
    float *fbuf = nullptr;
    if (prec == EVSL_FP32) {
        fbuf = (float *)ctx_ws(c, WS_F32_X, sizeof(float) * 4 * N, &st);
        if (st) return st;
    }
    EVSL_TRY(filter_apply_dev(c, pol, nvec, X, Y, prec, B0, B1, fbuf));
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "filter_apply");
}

// Several filters on one matrix at once (the slices of one interval): column t of X gets
// filter pols[t].  Columns are processed in order of decreasing degree, so the columns still
// active at degree j are a prefix and each degree is one block launch over that prefix.
int filter_apply_multi_dev(evsl_ctx *c, int npol, const evsl_polfilt *pols, const double *X,
                           double *Y, evsl_precision prec)
{
    const int64_t n = c->A.n, N = n * (int64_t)npol;
    const double lmin = pols[0].lmin, lmax = pols[0].lmax;
    for (int t = 0; t < npol; t++)
        if (std::fabs(pols[t].lmin - lmin) > 1e-12 * std::fabs(lmax - lmin) ||
            std::fabs(pols[t].lmax - lmax) > 1e-12 * std::fabs(lmax - lmin))
            return ctx_fail(c, EVSL_ERR_ARG, "filter_apply_multi: filters must share [lmin, lmax]");
    std::vector<int> perm(npol);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return pols[x].deg > pols[y].deg; });
    const int maxdeg = pols[perm[0]].deg;
    std::vector<int> active(maxdeg + 1, 0);
    for (int j = 0; j <= maxdeg; j++)
        for (int t = 0; t < npol; t++) active[j] += pols[perm[t]].deg >= j;
    std::vector<double> tab((size_t)(maxdeg + 1) * npol, 0.0);
    for (int j = 0; j <= maxdeg; j++)
        for (int t = 0; t < npol; t++)
            if (j <= pols[perm[t]].deg) tab[(size_t)j * npol + t] = pols[perm[t]].coef[j];
    int st = EVSL_OK;
    const size_t tbytes = (prec == EVSL_FP64 ? sizeof(double) : sizeof(float)) * tab.size();
    void *dtab = ctx_ws(c, WS_KPM_PART, tbytes + sizeof(int) * npol, &st);
    if (st) return st;
    int *dperm = (int *)((char *)dtab + tbytes);
    if (prec == EVSL_FP64) {
        EVSL_TRY(h2d(c, dtab, tab.data(), tbytes));
    } else {
        std::vector<float> tf(tab.begin(), tab.end());
        EVSL_TRY(h2d(c, dtab, tf.data(), tbytes));
    }
    EVSL_TRY(h2d(c, dperm, perm.data(), sizeof(int) * npol));
    double *Xs = (double *)ctx_ws(c, WS_W2, sizeof(double) * N * 2, &st);
    if (st) return st;
    double *Ys = Xs + N;
    EVSL_TRY(gather_cols(c, n, npol, X, n, dperm, Xs, n));
    const double cc = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    const bool hat = ensure_mapped(c, cc, d, &st);
    if (st) return st;
    if (maxdeg == 0) {
        for (int t = 0; t < npol; t++)
            EVSL_TRY(scale_vec(c, n, Xs + (int64_t)t * n, tab[t], Ys + (int64_t)t * n));
    } else {
        double *B0 = nullptr, *B1 = nullptr;
        float *fb = nullptr;
        if (prec == EVSL_FP64) {
            B0 = (double *)ctx_ws(c, WS_W0, sizeof(double) * N, &st);
            if (st) return st;
            B1 = (double *)ctx_ws(c, WS_W1, sizeof(double) * N, &st);
            if (st) return st;
        } else {
            fb = (float *)ctx_ws(c, WS_F32_X, sizeof(float) * 4 * N, &st);
            if (st) return st;
        }
        // tile shape of the block step (timed once per matrix, width and precision)
        if (prec == EVSL_FP64) EVSL_TRY(tune_block_f64(c, npol, Xs));
        else EVSL_TRY(tune_block_f32(c, npol, fb));
        auto issue = [&]() -> int {
            return issue_filter_multi(c, npol, active, maxdeg, Xs, Ys, dtab, prec, hat, cc, d, B0, B1, fb);
        };
        int r = 1;
        if (maxdeg >= GRAPH_MIN_DEG && !c->graphs_off) {
            uint64_t h = 1469598103934665603ull;
            const void *ptrs[] = {Xs, Ys, dtab, B0, B1, fb, c->A.sptr, c->A.col, c->A.val, c->A.val32,
                                  c->A.vhat, c->A.vhat32};
            h = fnv1a(h, ptrs, sizeof(ptrs));
            const int64_t meta[] = {-1, n, npol, maxdeg, (int64_t)prec, (int64_t)hat};
            h = fnv1a(h, meta, sizeof(meta));
            const double dm[] = {cc, d};
            h = fnv1a(h, dm, sizeof(dm));
            h = fnv1a(h, active.data(), sizeof(int) * active.size());
            r = launch_graph(c, h, maxdeg, issue);
        }
        if (r == 1) {
            ProfGroup g;
            prof_begin(c, EVSL_K_CHEB_STEP, &g);
            EVSL_TRY(issue());
            prof_end(c, &g, maxdeg);
        } else if (r != EVSL_OK) {
            return r;
        }
    }
    // scatter back: Y[:, perm[t]] = Ys[:, t]
    std::vector<int> inv(npol);
    for (int t = 0; t < npol; t++) inv[perm[t]] = t;
    EVSL_TRY(h2d(c, dperm, inv.data(), sizeof(int) * npol));
    return gather_cols(c, n, npol, Ys, n, dperm, Y, n);
}

int drv_filter_apply_multi(evsl_ctx *c, int npol, const evsl_polfilt *pols, const double *X,
                           double *Y, evsl_precision prec)
{
    EVSL_TRY(filter_apply_multi_dev(c, npol, pols, X, Y, prec));
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "filter_apply_multi");
}

// KPM moments mu_0..M.  doubling: only ceil(M/2) recurrence steps; step j yields
// sum_l w_j^T w_{j-1} and sum_l ||w_j||^2, from which T_{2j} = 2 T_j^2 - T_0 and
// T_{2j-1} = 2 T_j T_{j-1} - T_1 give mu_{2j} and mu_{2j-1}.
template <typename T>
static int kpm_run(evsl_ctx *c, int M, int nvec, uint64_t seed, double lmin, double lmax,
                   double *mu, bool doubling)
{
    const int64_t n = c->A.n, N = n * (int64_t)kpm_ld(nvec);   // row-major probe blocks
    const double cc = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    int st = EVSL_OK;
    T *W0 = (T *)ctx_ws(c, WS_W0, sizeof(T) * N, &st);
    if (st) return st;
    T *W1 = (T *)ctx_ws(c, WS_W1, sizeof(T) * N, &st);
    if (st) return st;
    const int nb = kpm_nblocks(c);
    const int K = doubling ? (M + 1) / 2 : M;          // recurrence steps
    const int rows = doubling ? 2 * K + 1 : M + 1;     // partial-sum rows 0..rows-1
    double *part = (double *)ctx_ws(c, WS_KPM_PART, sizeof(double) * (size_t)rows * nb, &st);
    if (st) return st;
    double *dmu = (double *)ctx_ws(c, WS_SCAL, sizeof(double) * (rows + 16), &st);
    if (st) return st;
    const bool hat = ensure_mapped(c, cc, d, &st);
    if (st) return st;
    if constexpr (sizeof(T) == 8)
        EVSL_TRY(kpm_init_f64(c, nvec, seed, (double *)W0));
    else
        EVSL_TRY(kpm_init_f32(c, nvec, seed, (float *)W0));
    ProfGroup g;
    prof_begin(c, EVSL_K_KPM_STEP, &g);
    T *prev = W0, *cur = W1;
    for (int k = 1; k <= K; k++) {
        // k = 1: cur = Ahat W0 ; k >= 2: prev <- 2 Ahat cur - prev, then swap
        if constexpr (sizeof(T) == 8) {
            if (k == 1)
                EVSL_TRY(kpm_step_f64(c, 0, nvec, seed, (double *)W0, nullptr, (double *)W1, cc, 1.0 / d, part, 1, nb, hat, doubling));
            else
                EVSL_TRY(kpm_step_f64(c, 1, nvec, seed, (double *)cur, (double *)prev, (double *)prev, cc, 2.0 / d, part, k, nb, hat, doubling));
        } else {
            if (k == 1)
                EVSL_TRY(kpm_step_f32(c, 0, nvec, seed, (float *)W0, nullptr, (float *)W1, cc, 1.0 / d, part, 1, nb, hat, doubling));
            else
                EVSL_TRY(kpm_step_f32(c, 1, nvec, seed, (float *)cur, (float *)prev, (float *)prev, cc, 2.0 / d, part, k, nb, hat, doubling));
        }
        if (k >= 2) std::swap(prev, cur);
    }
    prof_end(c, &g, K);
    std::vector<double> hs(rows, 0.0);
    if (rows > 1) {
        // fixed-order sums of the per-block partials
        EVSL_TRY(reduce_rows(c, rows - 1, nb, part + nb, dmu + 1));
        EVSL_TRY(d2h(c, hs.data() + 1, dmu + 1, sizeof(double) * (rows - 1)));
    }
    mu[0] = (double)n;  // v^T v = n exactly for Rademacher probes
    if (!doubling) {
        for (int k = 1; k <= M; k++) mu[k] = hs[k] / nvec;
        return EVSL_OK;
    }
    if (M >= 1) mu[1] = hs[1] / nvec;
    for (int j = 1; j <= K; j++) {
        if (2 * j <= M) mu[2 * j] = (2.0 * hs[2 * j] - (double)n * nvec) / nvec;
        if (j >= 2 && 2 * j - 1 <= M) mu[2 * j - 1] = (2.0 * hs[2 * j - 1] - hs[1]) / nvec;
    }
    return EVSL_OK;
}

// Per-probe KPM sums for probes first .. first + np - 1: the same recurrence as kpm_run on a
// block of only these probes, with each probe's dot product v_l^T w_k formed separately in a
// fixed order (kpm_probe_dots), so that a probe's values do not depend on the block it is in.
template <typename T>
static int kpm_probe_run(evsl_ctx *c, int M, int64_t first, int np, uint64_t seed, double lmin, double lmax,
                         double *out)
{
    const int64_t n = c->A.n, N = n * (int64_t)kpm_ld(np);
    const double cc = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    int st = EVSL_OK;
    T *W0 = (T *)ctx_ws(c, WS_W0, sizeof(T) * N, &st);
    if (st) return st;
    T *W1 = (T *)ctx_ws(c, WS_W1, sizeof(T) * N, &st);
    if (st) return st;
    const int nb = kpm_nblocks(c);
    double *part = (double *)ctx_ws(c, WS_KPM_PART, sizeof(double) * (size_t)(M + 1) * nb, &st);
    if (st) return st;
    const int nd = kpm_probe_dot_blocks(c);
    double *dpart = (double *)ctx_ws(c, WS_GEN_MU, sizeof(double) * ((size_t)nd * np + (size_t)(M + 1) * np), &st);
    if (st) return st;
    double *dk = dpart + (size_t)nd * np;      // (M + 1) x np: row k = the probes' sums of step k
    const bool hat = ensure_mapped(c, cc, d, &st);
    if (st) return st;
    auto dots = [&](const T *W, int k) {
        if constexpr (sizeof(T) == 8) return kpm_probe_dots_f64(c, np, (const double *)W, dpart, dk + (size_t)k * np);
        else return kpm_probe_dots_f32(c, np, (const float *)W, dpart, dk + (size_t)k * np);
    };
    if constexpr (sizeof(T) == 8)
        EVSL_TRY(kpm_init_f64(c, np, seed, (double *)W0, (uint64_t)first));
    else
        EVSL_TRY(kpm_init_f32(c, np, seed, (float *)W0, (uint64_t)first));
    ProfGroup g;
    prof_begin(c, EVSL_K_KPM_STEP, &g);
    T *prev = W0, *cur = W1;
    for (int k = 1; k <= M; k++) {
        if constexpr (sizeof(T) == 8) {
            if (k == 1)
                EVSL_TRY(kpm_step_f64(c, 0, np, seed, (double *)W0, nullptr, (double *)W1, cc, 1.0 / d, part, 1, nb, hat));
            else
                EVSL_TRY(kpm_step_f64(c, 1, np, seed, (double *)cur, (double *)prev, (double *)prev, cc, 2.0 / d, part, k, nb, hat));
        } else {
            if (k == 1)
                EVSL_TRY(kpm_step_f32(c, 0, np, seed, (float *)W0, nullptr, (float *)W1, cc, 1.0 / d, part, 1, nb, hat));
            else
                EVSL_TRY(kpm_step_f32(c, 1, np, seed, (float *)cur, (float *)prev, (float *)prev, cc, 2.0 / d, part, k, nb, hat));
        }
        if (k >= 2) std::swap(prev, cur);
        // the newest block: W1 after step 1, `cur` after the swap of every later step
        EVSL_TRY(dots(k == 1 ? W1 : cur, k));
    }
    prof_end(c, &g, M);
    std::vector<double> h((size_t)(M + 1) * np, 0.0);
    if (M >= 1) EVSL_TRY(d2h(c, h.data() + np, dk + np, sizeof(double) * (size_t)M * np));
    for (int l = 0; l < np; l++) {
        out[(size_t)l * (M + 1)] = (double)n;   // v^T v = n exactly for Rademacher probes
        for (int k = 1; k <= M; k++) out[(size_t)l * (M + 1) + k] = h[(size_t)k * np + l];
    }
    return EVSL_OK;
}

int drv_kpm_probe(evsl_ctx *c, int degree, int64_t first, int nprobe, uint64_t seed, double lmin, double lmax,
                  evsl_precision prec, double *out)
{
    if (prec == EVSL_FP64) return kpm_probe_run<double>(c, degree, first, nprobe, seed, lmin, lmax, out);
    return kpm_probe_run<float>(c, degree, first, nprobe, seed, lmin, lmax, out);
}

int drv_kpm(evsl_ctx *c, int degree, int nvec, uint64_t seed, double lmin, double lmax,
            evsl_precision prec, double *mu, bool doubling)
{
    if (prec == EVSL_FP64) return kpm_run<double>(c, degree, nvec, seed, lmin, lmax, mu, doubling);
    return kpm_run<float>(c, degree, nvec, seed, lmin, lmax, mu, doubling);
}

// ------------------------------------------------------------------------------------------
// Lanczos / Gaussian-quadrature density: for each of nvec seeded unit vectors, an m-step Lanczos
// run on A with full reorthogonalisation; T = S diag(theta) S^T gives the quadrature nodes theta_j
// and weights S_{1j}^2.  A breakdown (beta <= 1e-13 ||A q_j||) ends that vector's run early.
int drv_landos(evsl_ctx *c, int m, int nvec, uint64_t seed, double *nodes, double *weights, int *mused)
{
    const int64_t n = c->A.n;
    const int mm = (int)std::min<int64_t>(m, n);
    int st = EVSL_OK;
    double *Q = (double *)ctx_ws(c, WS_LAN_Q, sizeof(double) * n * (mm + 1), &st);
    if (st) return st;
    double *z = (double *)ctx_ws(c, WS_LAN_VEC, sizeof(double) * n * 3, &st);
    if (st) return st;
    double *sc = (double *)ctx_ws(c, WS_SCAL, sizeof(double) * (Scal::H + mm + 8), &st);
    if (st) return st;
    double *h = sc + Scal::H;
    const int M = std::max(2, mm + (mm & 1));
    double *V = (double *)ctx_ws(c, WS_LAN_T, sizeof(double) * (size_t)M * M, &st);
    if (st) return st;
    for (int l = 0; l < nvec; l++) {
        EVSL_TRY(fill_uniform_f64(c, n, seed, SM_STREAM_LANDOS, (uint64_t)l, Q));
        EVSL_TRY(coldot(c, n, 1, Q, n, Q, n, sc + Scal::TMP));
        double nq2 = 0;
        EVSL_TRY(d2h(c, &nq2, sc + Scal::TMP, sizeof(double)));
        EVSL_TRY(scale_vec(c, n, Q, 1.0 / std::sqrt(nq2), nullptr));
        std::vector<double> T((size_t)mm * mm, 0.0);
        double beta = 0.0;
        int k = 0;
        for (int j = 0; j < mm; j++) {
            double *qj = Q + (int64_t)j * n;
            EVSL_TRY(spmv_f64(c, 1, qj, z));
            EVSL_TRY(coldot(c, n, 1, z, n, z, n, sc + Scal::NRM_Y));
            EVSL_TRY(lan_three_term(c, n, z, j > 0 ? Q + (int64_t)(j - 1) * n : nullptr, beta, qj, z, sc + Scal::ALPHA));
            EVSL_TRY(lan_sub_alpha(c, n, z, qj, sc + Scal::ALPHA, sc + Scal::NRM_BEFORE));
            EVSL_TRY(cgs_pass(c, z, Q, j + 1, nullptr, 0, h, sc + Scal::NRM_AFTER));
            double hs[4];
            EVSL_TRY(d2h(c, hs, sc, sizeof(double) * 4));
            double nrm2 = hs[2];
            if (hs[2] < DGKS_ETA2 * hs[1]) {
                EVSL_TRY(cgs_pass(c, z, Q, j + 1, nullptr, 0, h, sc + Scal::NRM_AFTER));
                EVSL_TRY(d2h(c, &nrm2, sc + Scal::NRM_AFTER, sizeof(double)));
            }
            T[(size_t)j * mm + j] = hs[0];
            k = j + 1;
            beta = std::sqrt(nrm2);
            if (j + 1 == mm || beta <= 1e-13 * std::sqrt(hs[3])) break;
            T[(size_t)(j + 1) * mm + j] = beta;
            T[(size_t)j * mm + j + 1] = beta;
            EVSL_TRY(scale_vec(c, n, z, 1.0 / beta, Q + (int64_t)(j + 1) * n));
        }
        std::vector<double> Tk((size_t)k * k), w(k), s0(k);
        for (int jj = 0; jj < k; jj++)
            for (int ii = 0; ii < k; ii++) Tk[(size_t)jj * k + ii] = T[(size_t)jj * mm + ii];
        int ldv = 0, sweeps = 0;
        EVSL_TRY(jacobi_eig(c, k, Tk.data(), w.data(), V, &ldv, &sweeps));
        // first row of the eigenvector matrix
        cudaError_t e = cudaMemcpy2DAsync(s0.data(), sizeof(double), V, sizeof(double) * ldv, sizeof(double), k,
                                          cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "landos first row");
        std::vector<int> order(k);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] < w[y]; });
        for (int j = 0; j < mm; j++) {
            nodes[(size_t)l * m + j] = j < k ? w[order[j]] : 0.0;
            weights[(size_t)l * m + j] = j < k ? s0[order[j]] * s0[order[j]] : 0.0;
        }
        for (int j = mm; j < m; j++) {
            nodes[(size_t)l * m + j] = 0.0;
            weights[(size_t)l * m + j] = 0.0;
        }
        mused[l] = k;
    }
    return EVSL_OK;
}

int drv_bounds(evsl_ctx *c, int steps, uint64_t seed, double *lmin, double *lmax)
{
    const int64_t n = c->A.n;
    if (steps > n) steps = (int)n;
    int st = EVSL_OK;
    double *Q = (double *)ctx_ws(c, WS_LAN_Q, sizeof(double) * n * (steps + 1), &st);
    if (st) return st;
    double *z = (double *)ctx_ws(c, WS_LAN_VEC, sizeof(double) * n * 3, &st);
    if (st) return st;
    double *sc = (double *)ctx_ws(c, WS_SCAL, sizeof(double) * (Scal::H + steps + 8), &st);
    if (st) return st;
    double *h = sc + Scal::H;
    EVSL_TRY(fill_uniform_f64(c, n, seed, SM_STREAM_BOUNDS, 0, Q));
    EVSL_TRY(coldot(c, n, 1, Q, n, Q, n, sc + Scal::TMP));
    double nq2 = 0;
    EVSL_TRY(d2h(c, &nq2, sc + Scal::TMP, sizeof(double)));
    EVSL_TRY(scale_vec(c, n, Q, 1.0 / std::sqrt(nq2), nullptr));
    std::vector<double> T((size_t)steps * steps, 0.0);
    double beta = 0.0;
    int m = 0;
    for (int j = 0; j < steps; j++) {
        double *qj = Q + (int64_t)j * n;
        EVSL_TRY(spmv_f64(c, 1, qj, z));
        EVSL_TRY(lan_three_term(c, n, z, j > 0 ? Q + (int64_t)(j - 1) * n : nullptr, beta, qj, z, sc + Scal::ALPHA));
        EVSL_TRY(lan_sub_alpha(c, n, z, qj, sc + Scal::ALPHA, sc + Scal::NRM_BEFORE));
        EVSL_TRY(cgs_pass(c, z, Q, j + 1, nullptr, 0, h, sc + Scal::NRM_AFTER));
        double hs[3];
        EVSL_TRY(d2h(c, hs, sc, sizeof(double) * 3));
        double nrm2 = hs[2];
        if (hs[2] < DGKS_ETA2 * hs[1]) {
            EVSL_TRY(cgs_pass(c, z, Q, j + 1, nullptr, 0, h, sc + Scal::NRM_AFTER));
            EVSL_TRY(d2h(c, &nrm2, sc + Scal::NRM_AFTER, sizeof(double)));
        }
        T[(size_t)j * steps + j] = hs[0];
        beta = std::sqrt(nrm2);
        m = j + 1;
        if (j + 1 < steps) {
            T[(size_t)(j + 1) * steps + j] = beta;
            T[(size_t)j * steps + j + 1] = beta;
        }
        if (beta == 0.0) break;
        EVSL_TRY(scale_vec(c, n, z, 1.0 / beta, Q + (int64_t)(j + 1) * n));
    }
    std::vector<double> Tm((size_t)m * m), w(m);
    for (int j = 0; j < m; j++)
        for (int i = 0; i < m; i++) Tm[(size_t)j * m + i] = T[(size_t)j * steps + i];
    int M = m + (m & 1);
    if (M < 2) M = 2;
    double *V = (double *)ctx_ws(c, WS_LAN_T, sizeof(double) * (size_t)M * M, &st);
    if (st) return st;
    int ldv = 0, sweeps = 0;
    EVSL_TRY(jacobi_eig(c, m, Tm.data(), w.data(), V, &ldv, &sweeps));
    int imin = (int)(std::min_element(w.begin(), w.end()) - w.begin());
    int imax = (int)(std::max_element(w.begin(), w.end()) - w.begin());
    double smin = 0, smax = 0;
    EVSL_TRY(d2h(c, &smin, V + (int64_t)imin * ldv + (m - 1), sizeof(double)));
    EVSL_TRY(d2h(c, &smax, V + (int64_t)imax * ldv + (m - 1), sizeof(double)));
    *lmin = w[imin] - std::fabs(beta * smin);
    *lmax = w[imax] + std::fabs(beta * smax);
    return EVSL_OK;
}

