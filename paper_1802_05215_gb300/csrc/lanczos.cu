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

int d2d(evsl_ctx *c, void *dst, const void *src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "device-to-device copy");
}

// Y = rho(Ahat) X on nvec columns with the three-term recurrence; one fused launch per degree.
// B0, B1: n*nvec FP64 temporaries; fbuf: 4*n*nvec floats (FP32 mode only).
int filter_run(evsl_ctx *c, const evsl_polfilt *pol, int nvec, const double *X, double *Y,
               evsl_precision prec, double *B0, double *B1, float *fbuf)
{
    const int64_t n = c->A.n, N = n * (int64_t)nvec;
    const double cc = 0.5 * (pol->lmax + pol->lmin), d = 0.5 * (pol->lmax - pol->lmin);
    const double *coef = pol->coef;
    const int deg = pol->deg;
    if (deg == 0) return scale_vec(c, N, const_cast<double *>(X), coef[0], Y);
    ProfGroup g;
    if (prec == EVSL_FP64) {
        prof_begin(c, EVSL_K_CHEB_STEP, &g);
        EVSL_TRY(cheb_step_f64(c, 0, nvec, X, nullptr, B0, Y, cc, 1.0 / d, coef[0], coef[1]));
        const double *prev = X;
        double *cur = B0;
        for (int j = 2; j <= deg; j++) {
            double *out = (j == 2) ? B1 : const_cast<double *>(prev);
            EVSL_TRY(cheb_step_f64(c, 1, nvec, cur, prev, out, Y, cc, 2.0 / d, 0.0, coef[j]));
            prev = cur;
            cur = out;
        }
        prof_end(c, &g, deg);
        return EVSL_OK;
    }
    float *fx = fbuf, *f0 = fbuf + N, *f1 = fbuf + 2 * N, *fy = fbuf + 3 * N;
    EVSL_TRY(convert_f64_to_f32(c, N, X, fx));
    prof_begin(c, EVSL_K_CHEB_STEP, &g);
    EVSL_TRY(cheb_step_f32(c, 0, nvec, fx, nullptr, f0, fy, cc, 1.0 / d, coef[0], coef[1]));
    const float *prev = fx;
    float *cur = f0;
    for (int j = 2; j <= deg; j++) {
        float *out = (j == 2) ? f1 : const_cast<float *>(prev);
        EVSL_TRY(cheb_step_f32(c, 1, nvec, cur, prev, out, fy, cc, 2.0 / d, 0.0, coef[j]));
        prev = cur;
        cur = out;
    }
    prof_end(c, &g, deg);
    return convert_f32_to_f64(c, N, fy, Y);
}

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
    EVSL_TRY(filter_run(c, pol, nvec, X, Y, prec, B0, B1, fbuf));
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "filter_apply");
}

template <typename T>
static int kpm_run(evsl_ctx *c, int M, int nvec, uint64_t seed, double lmin, double lmax,
                   double *mu)
{
    const int64_t n = c->A.n, N = n * (int64_t)nvec;
    const double cc = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    int st = EVSL_OK;
    T *W0 = (T *)ctx_ws(c, WS_W0, sizeof(T) * N, &st);
    if (st) return st;
    T *W1 = (T *)ctx_ws(c, WS_W1, sizeof(T) * N, &st);
    if (st) return st;
    const int nb = kpm_nblocks(c);
    double *part = (double *)ctx_ws(c, WS_KPM_PART, sizeof(double) * (size_t)(M + 1) * nb, &st);
    if (st) return st;
    double *dmu = (double *)ctx_ws(c, WS_SCAL, sizeof(double) * (M + 1 + 16), &st);
    if (st) return st;
    if constexpr (sizeof(T) == 8)
        EVSL_TRY(kpm_init_f64(c, nvec, seed, (double *)W0));
    else
        EVSL_TRY(kpm_init_f32(c, nvec, seed, (float *)W0));
    ProfGroup g;
    prof_begin(c, EVSL_K_KPM_STEP, &g);
    T *prev = W0, *cur = W1;
    for (int k = 1; k <= M; k++) {
        // k = 1: cur = Ahat W0 ; k >= 2: prev <- 2 Ahat cur - prev, then swap
        if constexpr (sizeof(T) == 8) {
            if (k == 1)
                EVSL_TRY(kpm_step_f64(c, 0, nvec, seed, (double *)W0, nullptr, (double *)W1, cc, 1.0 / d, part, 1, nb));
            else
                EVSL_TRY(kpm_step_f64(c, 1, nvec, seed, (double *)cur, (double *)prev, (double *)prev, cc, 2.0 / d, part, k, nb));
        } else {
            if (k == 1)
                EVSL_TRY(kpm_step_f32(c, 0, nvec, seed, (float *)W0, nullptr, (float *)W1, cc, 1.0 / d, part, 1, nb));
            else
                EVSL_TRY(kpm_step_f32(c, 1, nvec, seed, (float *)cur, (float *)prev, (float *)prev, cc, 2.0 / d, part, k, nb));
        }
        if (k >= 2) std::swap(prev, cur);
    }
    prof_end(c, &g, M);
    std::vector<double> hmu(M + 1, 0.0);
    if (M >= 1) {
        // moments 1..M: fixed-order sums of the per-block partials
        EVSL_TRY(reduce_rows(c, M, nb, part + nb, dmu + 1));
        EVSL_TRY(d2h(c, hmu.data() + 1, dmu + 1, sizeof(double) * M));
    }
    mu[0] = (double)n;  // v^T v = n exactly for Rademacher probes
    for (int k = 1; k <= M; k++) mu[k] = hmu[k] / nvec;
    return EVSL_OK;
}

int drv_kpm(evsl_ctx *c, int degree, int nvec, uint64_t seed, double lmin, double lmax,
            evsl_precision prec, double *mu)
{
    if (prec == EVSL_FP64) return kpm_run<double>(c, degree, nvec, seed, lmin, lmax, mu);
    return kpm_run<float>(c, degree, nvec, seed, lmin, lmax, mu);
}

// ------------------------------------------------------------------------------------------
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

// ------------------------------------------------------------------------------------------
namespace {

struct LanState {
    evsl_ctx *c;
    int64_t n;
    int m, cap;
    double *U, *Q, *Yt, *Z, *y, *B0, *B1, *sc, *h, *Vj, *S, *lamd, *resd, *nrmd;
    int *idxd;
    float *fbuf;
    std::vector<double> T;  // (m+1) x (m+1) column-major
    double &t(int i, int j) { return T[(size_t)j * (m + 1) + i]; }
    int64_t nmv = 0, npass = 0;
    double t_filter = 0, t_orth = 0, t_restart = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
};

// fresh seeded vector in dst, orthogonalised (two passes) against U[:, :nlock] and Q[:, :nq]
int fresh_vector(LanState &S, uint64_t seed, uint64_t index, double *dst, int nlock, int nq)
{
    evsl_ctx *c = S.c;
    EVSL_TRY(fill_uniform_f64(c, S.n, seed, SM_STREAM_LANCZOS, index, dst));
    for (int p = 0; p < 2; p++)
        if (nlock + nq > 0) EVSL_TRY(cgs_pass(c, dst, S.U, nlock, S.Q, nq, S.h, S.sc + Scal::TMP));
    EVSL_TRY(coldot(c, S.n, 1, dst, S.n, dst, S.n, S.sc + Scal::TMP));
    double nr2 = 0;
    EVSL_TRY(d2h(c, &nr2, S.sc + Scal::TMP, sizeof(double)));
    return scale_vec(c, S.n, dst, 1.0 / std::sqrt(nr2), nullptr);
}

// Reorthogonalise z (CGS with the DGKS test, at most two passes) against [U, Q[:, :nq]];
// returns ||z||^2 after.  nrm_before2 is ||z||^2 before the first pass.
int reorth(LanState &S, double *z, int nlock, int nq, double nrm_before2, double *nrm2_out)
{
    evsl_ctx *c = S.c;
    EVSL_TRY(cgs_pass(c, z, S.U, nlock, S.Q, nq, S.h, S.sc + Scal::NRM_AFTER));
    S.npass++;
    double a2 = 0;
    EVSL_TRY(d2h(c, &a2, S.sc + Scal::NRM_AFTER, sizeof(double)));
    if (a2 < DGKS_ETA2 * nrm_before2) {
        EVSL_TRY(cgs_pass(c, z, S.U, nlock, S.Q, nq, S.h, S.sc + Scal::NRM_AFTER));
        S.npass++;
        EVSL_TRY(d2h(c, &a2, S.sc + Scal::NRM_AFTER, sizeof(double)));
    }
    *nrm2_out = a2;
    return EVSL_OK;
}

// Rayleigh-Ritz refinement with A over W = U[:, :p] (orthonormal columns): G = W^T A W =
// Z diag(theta) Z^T; the columns of W Z with theta in the slice and ||A w - theta w|| <= tol ||A||
// replace the locked set, in ascending theta.  lam/res are replaced accordingly.
int refine_locked(LanState &S, double a, double b, bool right_closed, double normA, double tol,
                  int p, std::vector<double> &lam, std::vector<double> &res, int *kept_out,
                  bool verbose)
{
    evsl_ctx *c = S.c;
    const int64_t n = S.n;
    int st = EVSL_OK;
    double *G = (double *)ctx_ws(c, WS_LAN_G, sizeof(double) * (size_t)p * p, &st);
    if (st) return st;
    const int zc = std::min(p, 128);
    S.Z = (double *)ctx_ws(c, WS_LAN_Z, sizeof(double) * n * zc, &st);
    if (st) return st;
    for (int j0 = 0; j0 < p; j0 += zc) {
        int nc = std::min(zc, p - j0);
        EVSL_TRY(spmv_f64(c, nc, S.U + (int64_t)j0 * n, S.Z));
        EVSL_TRY(gemm_tn(c, n, p, nc, S.U, n, S.Z, n, G + (int64_t)j0 * p, p));
    }
    std::vector<double> Gh((size_t)p * p), w(p);
    EVSL_TRY(d2h(c, Gh.data(), G, sizeof(double) * Gh.size()));
    for (int j = 0; j < p; j++)
        for (int i = 0; i < j; i++) {
            double v = 0.5 * (Gh[(size_t)j * p + i] + Gh[(size_t)i * p + j]);
            Gh[(size_t)j * p + i] = v;
            Gh[(size_t)i * p + j] = v;
        }
    int M = p + (p & 1);
    S.Vj = (double *)ctx_ws(c, WS_LAN_T, sizeof(double) * (size_t)M * M, &st);
    if (st) return st;
    S.S = (double *)ctx_ws(c, WS_LAN_S, sizeof(double) * (size_t)M * M, &st);
    if (st) return st;
    int ldv = 0, sweeps = 0;
    EVSL_TRY(jacobi_eig(c, p, Gh.data(), w.data(), S.Vj, &ldv, &sweeps));
    std::vector<int> order(p);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] < w[y]; });
    S.idxd = (int *)ctx_ws(c, WS_LAN_IDX, sizeof(int) * (size_t)(2 * p + 8), &st);
    if (st) return st;
    EVSL_TRY(h2d(c, S.idxd, order.data(), sizeof(int) * p));
    EVSL_TRY(gather_cols(c, p, p, S.Vj, ldv, S.idxd, S.S, p));
    S.Yt = (double *)ctx_ws(c, WS_LAN_Y, sizeof(double) * n * std::max(S.m, p), &st);
    if (st) return st;
    EVSL_TRY(gemm_nn(c, n, p, p, S.U, n, S.S, p, S.Yt, n));
    std::vector<double> th(p), r2(p);
    for (int j = 0; j < p; j++) th[j] = w[order[j]];
    double *lamd = (double *)ctx_ws(c, WS_KPM_PART, sizeof(double) * 2 * (size_t)p, &st);
    if (st) return st;
    EVSL_TRY(h2d(c, lamd, th.data(), sizeof(double) * p));
    for (int j0 = 0; j0 < p; j0 += zc) {
        int nc = std::min(zc, p - j0);
        EVSL_TRY(spmv_f64(c, nc, S.Yt + (int64_t)j0 * n, S.Z));
        EVSL_TRY(colres2(c, n, nc, S.Z, S.Yt + (int64_t)j0 * n, n, lamd + j0, lamd + p + j0));
    }
    EVSL_TRY(d2h(c, r2.data(), lamd + p, sizeof(double) * p));
    std::vector<int> keep;
    lam.clear();
    res.clear();
    for (int j = 0; j < p; j++) {
        bool inside = (th[j] >= a) && (right_closed ? (th[j] <= b) : (th[j] < b));
        double rj = std::sqrt(std::max(0.0, r2[j])) / normA;
        if (inside && rj <= tol && (int)keep.size() < S.cap) {
            keep.push_back(j);
            lam.push_back(th[j]);
            res.push_back(rj);
        }
    }
    if (!keep.empty()) {
        EVSL_TRY(h2d(c, S.idxd + p, keep.data(), sizeof(int) * keep.size()));
        EVSL_TRY(gather_cols(c, n, (int)keep.size(), S.Yt, n, S.idxd + p, S.U, n));
    }
    if (verbose) fprintf(stderr, "[evsl] refinement: p=%d kept=%zu sweeps=%d\n", p, keep.size(), sweeps);
    *kept_out = (int)keep.size();
    return EVSL_OK;
}

float ev_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

}  // namespace

int drv_chebLanTr(evsl_ctx *c, double a, double b, const evsl_polfilt *pol,
                  const evsl_lan_opts *o, int cap, int *nev_out, double *lam_out, double *Y_out,
                  double *res_out, evsl_stats *st_out)
{
    cudaEvent_t tstart, tend;
    cudaEventCreate(&tstart);
    cudaEventCreate(&tend);
    cudaEventRecord(tstart, c->stream);
    LanState S;
    S.c = c;
    S.n = c->A.n;
    const int64_t n = S.n;
    int m = o->m;
    if (m > n) m = (int)n;
    S.m = m;
    S.cap = cap;
    const int maxit = o->maxit > 0 ? o->maxit : 20 * m;
    const int ncycle = o->ncycle > 0 ? o->ncycle : 10;
    const double tol = o->tol > 0 ? o->tol : 1e-8;
    const double tau1 = o->tau1 > 0 ? o->tau1 : 1e-10;
    const double bar = pol->bar;
    const double normA = std::max(std::fabs(pol->lmin), std::fabs(pol->lmax));
    const int zcols = std::min(m, 128);
    int st = EVSL_OK;
#define WS(slot, bytes) ctx_ws(c, slot, bytes, &st); if (st) return st
    S.U = (double *)WS(WS_LAN_U, sizeof(double) * n * cap);
    S.Q = (double *)WS(WS_LAN_Q, sizeof(double) * n * (m + 1));
    S.Yt = (double *)WS(WS_LAN_Y, sizeof(double) * n * m);
    S.Z = (double *)WS(WS_LAN_Z, sizeof(double) * n * zcols);
    S.y = (double *)WS(WS_LAN_VEC, sizeof(double) * n * 3);
    S.B0 = S.y + n;
    S.B1 = S.y + 2 * n;
    const size_t nsc = Scal::H + (size_t)cap + m + 1 + 3 * (size_t)(m + 1) + 8;
    S.sc = (double *)WS(WS_SCAL, sizeof(double) * nsc);
    S.h = S.sc + Scal::H;
    S.lamd = S.h + cap + m + 1;
    S.resd = S.lamd + (m + 1);
    S.nrmd = S.resd + (m + 1);
    int Mpad = (m + 1) + ((m + 1) & 1);
    S.Vj = (double *)WS(WS_LAN_T, sizeof(double) * (size_t)Mpad * Mpad);
    S.S = (double *)WS(WS_LAN_S, sizeof(double) * (size_t)Mpad * Mpad);
    S.idxd = (int *)WS(WS_LAN_IDX, sizeof(int) * (size_t)(m + 1 + cap));
    S.fbuf = nullptr;
    if (o->prec == EVSL_FP32) S.fbuf = (float *)WS(WS_F32_X, sizeof(float) * 4 * n);
#undef WS
    cudaEventCreate(&S.e0);
    cudaEventCreate(&S.e1);
    cudaEventCreate(&S.e2);
    S.T.assign((size_t)(m + 1) * (m + 1), 0.0);
    std::vector<double> lam_l, res_l;  // locked pairs in locking order
    std::vector<double> trtheta, trs;
    int nlock = 0, l = 0, its = 0, nrestart = 0, nocand = 0, status = EVSL_OK, stall = 0, nrefine = 0;
    uint64_t fresh_index = 0;
    const uint64_t seed = o->seed;
    const char *venv = getenv("EVSL_VERBOSE");
    const bool verbose = venv && venv[0] == '1';

    // one filtered Lanczos step on column i (0-based); the caller sets up T's coupling
    auto apply_filter = [&](const double *q) -> int {
        cudaEventRecord(S.e0, c->stream);
        int r = filter_run(c, pol, 1, q, S.y, o->prec, S.B0, S.B1, S.fbuf);
        cudaEventRecord(S.e1, c->stream);
        S.nmv += pol->deg;
        return r;
    };

    EVSL_TRY(fresh_vector(S, seed, fresh_index++, S.Q, 0, 0));
    while (its <= maxit) {
        int k;
        std::fill(S.T.begin(), S.T.end(), 0.0);
        if (l > 0) {
            for (int j = 0; j < l; j++) {
                S.t(j, j) = trtheta[j];
                S.t(j, l) = trs[j];
                S.t(l, j) = trs[j];
            }
            double *ql = S.Q + (int64_t)l * n;
            EVSL_TRY(apply_filter(ql));
            its++;
            EVSL_TRY(coldot(c, n, 1, S.y, n, S.y, n, S.sc + Scal::NRM_Y));
            // z = y - sum_j s_j u_j ; alpha = q_l . z ; z -= alpha q_l
            EVSL_TRY(h2d(c, S.h, trs.data(), sizeof(double) * l));
            EVSL_TRY(gemv_n2(c, n, S.Q, l, nullptr, 0, S.h, S.y, S.sc + Scal::TMP));
            EVSL_TRY(lan_three_term(c, n, S.y, nullptr, 0.0, ql, S.y, S.sc + Scal::ALPHA));
            EVSL_TRY(lan_sub_alpha(c, n, S.y, ql, S.sc + Scal::ALPHA, S.sc + Scal::NRM_BEFORE));
            double hs[4];
            EVSL_TRY(d2h(c, hs, S.sc, sizeof(double) * 4));
            double nrm2;
            EVSL_TRY(reorth(S, S.y, nlock, l + 1, hs[1], &nrm2));
            cudaEventRecord(S.e2, c->stream);
            double beta = std::sqrt(nrm2);
            double *qn = S.Q + (int64_t)(l + 1) * n;
            if (beta <= 1e-13 * std::sqrt(hs[3])) {
                EVSL_TRY(fresh_vector(S, seed, fresh_index++, qn, nlock, l + 1));
                beta = 0.0;
            } else {
                EVSL_TRY(scale_vec(c, n, S.y, 1.0 / beta, qn));
            }
            cudaEventSynchronize(S.e2);
            S.t_filter += ev_ms(S.e0, S.e1) * 1e-3;
            S.t_orth += ev_ms(S.e1, S.e2) * 1e-3;
            S.t(l, l) = hs[0];
            S.t(l, l + 1) = beta;
            S.t(l + 1, l) = beta;
            k = l + 1;
        } else {
            k = 0;
        }
        const int lstart = k;
        double t_old = 0.0;
        bool have_old = false;
        int prev_nabove = 0;
        for (int i = k; i < m; i++) {
            its++;
            double *qi = S.Q + (int64_t)i * n;
            EVSL_TRY(apply_filter(qi));
            EVSL_TRY(coldot(c, n, 1, S.y, n, S.y, n, S.sc + Scal::NRM_Y));
            const double bi = (i > 0) ? S.t(i - 1, i) : 0.0;
            EVSL_TRY(lan_three_term(c, n, S.y, i > 0 ? S.Q + (int64_t)(i - 1) * n : nullptr, bi, qi,
                                    S.y, S.sc + Scal::ALPHA));
            EVSL_TRY(lan_sub_alpha(c, n, S.y, qi, S.sc + Scal::ALPHA, S.sc + Scal::NRM_BEFORE));
            double hs[4];
            EVSL_TRY(d2h(c, hs, S.sc, sizeof(double) * 4));
            double nrm2;
            EVSL_TRY(reorth(S, S.y, nlock, i + 1, hs[1], &nrm2));
            cudaEventRecord(S.e2, c->stream);
            double beta = std::sqrt(nrm2);
            double *qn = S.Q + (int64_t)(i + 1) * n;
            if (beta <= 1e-13 * std::sqrt(hs[3])) {
                EVSL_TRY(fresh_vector(S, seed, fresh_index++, qn, nlock, i + 1));
                beta = 0.0;
            } else {
                EVSL_TRY(scale_vec(c, n, S.y, 1.0 / beta, qn));
            }
            cudaEventSynchronize(S.e2);
            S.t_filter += ev_ms(S.e0, S.e1) * 1e-3;
            S.t_orth += ev_ms(S.e1, S.e2) * 1e-3;
            S.t(i, i) = hs[0];
            S.t(i, i + 1) = beta;
            S.t(i + 1, i) = beta;
            k = i + 1;
            if ((k - lstart) % ncycle == 0) {
                // early-restart test: sum of the Ritz values >= bar (bisection with inertia counts)
                std::vector<double> dd(k), ee(k, 0.0);
                for (int j = 0; j < k; j++) dd[j] = S.t(j, j);
                for (int j = 0; j < k; j++) {
                    if (j < l) ee[j] = S.t(j, l);
                    else if (j + 1 < k) ee[j] = S.t(j, j + 1);
                }
                int nbelow = host_count_below(k, l, dd.data(), ee.data(), bar);
                int nabove = k - nbelow;
                double t_new = 0.0;
                if (nabove > 0) {
                    double lo = 1e300, hi = -1e300;
                    double hub = 0.0;
                    for (int j = 0; j < l; j++) hub += std::fabs(ee[j]);
                    for (int j = 0; j < k; j++) {
                        double rr;
                        if (j < l) rr = std::fabs(ee[j]);
                        else if (j == l) rr = hub + std::fabs(ee[j]);
                        else rr = std::fabs(ee[j - 1]) + std::fabs(ee[j]);
                        lo = std::min(lo, dd[j] - rr);
                        hi = std::max(hi, dd[j] + rr);
                    }
                    std::vector<double> w(nabove);
                    EVSL_TRY(bisect_eigs(c, k, l, dd.data(), ee.data(), nbelow, k, lo, hi, w.data()));
                    for (double v : w) t_new += v;
                }
                if (verbose && (k - lstart) % (ncycle * 20) == 0)
                    fprintf(stderr, "[evsl]   check its=%d k=%d nabove=%d t=%.12f\n", its, k, nabove, t_new);
                if (have_old && nabove > 0 && std::fabs(t_new - t_old) < tau1 * std::max(1.0, std::fabs(t_new)))
                    break;
                // a cycle with nothing above bar ends once it had time for a missed eigenvalue to emerge
                if (have_old && nabove == 0 && prev_nabove == 0 && k - lstart >= std::max(2 * ncycle, m / 4))
                    break;
                t_old = t_new;
                prev_nabove = nabove;
                have_old = true;
            }
            if (its > maxit) break;
        }
        // ---- restart: Ritz pairs of T_k
        cudaEventRecord(S.e0, c->stream);
        nrestart++;
        std::vector<double> Tk((size_t)k * k), w(k);
        for (int j = 0; j < k; j++)
            for (int i = 0; i < k; i++) Tk[(size_t)j * k + i] = S.t(i, j);
        int ldv = 0, sweeps = 0;
        EVSL_TRY(jacobi_eig(c, k, Tk.data(), w.data(), S.Vj, &ldv, &sweeps));
        const double betak = S.t(k - 1, k);
        std::vector<int> order(k);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
        int ncand0 = 0;
        while (ncand0 < k && w[order[ncand0]] >= bar) ncand0++;
        int ncand = 0;
        const int nlock_before = nlock;
        std::vector<int> lock_idx, tr_idx;
        std::vector<double> new_trtheta, new_trs;
        if (ncand0 > 0) {
            EVSL_TRY(h2d(c, S.idxd, order.data(), sizeof(int) * ncand0));
            EVSL_TRY(gather_cols(c, k, ncand0, S.Vj, ldv, S.idxd, S.S, k));
            ProfGroup g;
            prof_begin(c, EVSL_K_RITZ_GEMM, &g);
            EVSL_TRY(gemm_nn(c, n, ncand0, k, S.Q, n, S.S, k, S.Yt, n));
            prof_end(c, &g, 1);
            EVSL_TRY(coldot(c, n, ncand0, S.Yt, n, S.Yt, n, S.nrmd));
            EVSL_TRY(colscale_inv_sqrt(c, n, ncand0, S.Yt, S.nrmd));
            std::vector<double> lamh(ncand0), resh(ncand0), slast(ncand0);
            for (int j0 = 0; j0 < ncand0; j0 += zcols) {
                int nc = std::min(zcols, ncand0 - j0);
                EVSL_TRY(spmv_f64(c, nc, S.Yt + (int64_t)j0 * n, S.Z));
                EVSL_TRY(coldot(c, n, nc, S.Yt + (int64_t)j0 * n, n, S.Z, n, S.lamd + j0));
                EVSL_TRY(colres2(c, n, nc, S.Z, S.Yt + (int64_t)j0 * n, n, S.lamd + j0, S.resd + j0));
            }
            EVSL_TRY(d2h(c, lamh.data(), S.lamd, sizeof(double) * ncand0));
            EVSL_TRY(d2h(c, resh.data(), S.resd, sizeof(double) * ncand0));
            {
                cudaError_t e = cudaMemcpy2DAsync(slast.data(), sizeof(double), S.S + (k - 1), sizeof(double) * k,
                                                  sizeof(double), ncand0, cudaMemcpyDeviceToHost, c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess) return ctx_cuda(c, e, "last-row readback");
            }
            for (int cnd = 0; cnd < ncand0; cnd++) {
                double lj = lamh[cnd];
                bool inside = (lj >= a) && (o->right_closed ? (lj <= b) : (lj < b));
                if (!inside) continue;
                ncand++;
                double rj = std::sqrt(std::max(0.0, resh[cnd])) / normA;
                if (rj <= tol) {
                    if (nlock + (int)lock_idx.size() >= cap) {
                        status = EVSL_ERR_CAPACITY;
                        break;
                    }
                    lock_idx.push_back(cnd);
                    lam_l.push_back(lj);
                    res_l.push_back(rj);
                } else if ((int)tr_idx.size() < m / 2) {
                    // thick-restart set, largest Ritz values first, at most m/2 vectors
                    tr_idx.push_back(cnd);
                    new_trtheta.push_back(w[order[cnd]]);
                    new_trs.push_back(betak * slast[cnd]);
                }
            }
            if (!lock_idx.empty()) {
                EVSL_TRY(h2d(c, S.idxd + (m + 1), lock_idx.data(), sizeof(int) * lock_idx.size()));
                EVSL_TRY(gather_cols(c, n, (int)lock_idx.size(), S.Yt, n, S.idxd + (m + 1),
                                     S.U + (int64_t)nlock * n, n));
                nlock += (int)lock_idx.size();
            }
        }
        if (status == EVSL_ERR_CAPACITY) break;
        const int ntr = (int)tr_idx.size();
        if (verbose)
            fprintf(stderr, "[evsl] restart %d: its=%d k=%d l=%d jacobi_sweeps=%d cand>=bar=%d in_slice=%d "
                            "locked+%d ntr=%d nlock=%d beta_k=%.3e\n",
                    nrestart, its, k, l, sweeps, ncand0, ncand, (int)lock_idx.size(), ntr,
                    nlock, betak);
        if (ncand == 0) nocand++; else nocand = 0;
        if (ncand > 0 && nlock == nlock_before) stall++; else stall = 0;
        bool refined = false;
        if (stall >= 2 && nrefine < 2 && ntr > 0 && nlock + ntr <= cap) {
            // stagnation: Rayleigh-Ritz with A over the locked set and the stuck candidates
            EVSL_TRY(h2d(c, S.idxd, tr_idx.data(), sizeof(int) * ntr));
            EVSL_TRY(gather_cols(c, n, ntr, S.Yt, n, S.idxd, S.U + (int64_t)nlock * n, n));
            int kept = 0;
            EVSL_TRY(refine_locked(S, a, b, o->right_closed != 0, normA, tol, nlock + ntr, lam_l, res_l, &kept, verbose));
            nlock = kept;
            nrefine++;
            stall = 0;
            nocand = 1;
            refined = true;
        }
        cudaEventRecord(S.e1, c->stream);
        cudaEventSynchronize(S.e1);
        S.t_restart += ev_ms(S.e0, S.e1) * 1e-3;
        if (nocand >= 2) break;
        if (its > maxit) {
            status = EVSL_ERR_NOCONV;
            break;
        }
        if (ncand == 0 || refined) {
            l = 0;
            EVSL_TRY(fresh_vector(S, seed, fresh_index++, S.Q, nlock, 0));
        } else {
            if (ntr != k) EVSL_TRY(d2d(c, S.Q + (int64_t)ntr * n, S.Q + (int64_t)k * n, sizeof(double) * n));
            if (ntr > 0) {
                EVSL_TRY(h2d(c, S.idxd, tr_idx.data(), sizeof(int) * ntr));
                EVSL_TRY(gather_cols(c, n, ntr, S.Yt, n, S.idxd, S.Q, n));
            }
            trtheta = new_trtheta;
            trs = new_trs;
            l = ntr;
            if (l == 0) {
                // continue from q_{k+1}, re-orthogonalised against the new locked vectors
                EVSL_TRY(coldot(c, n, 1, S.Q, n, S.Q, n, S.sc + Scal::TMP));
                double b2 = 0;
                EVSL_TRY(d2h(c, &b2, S.sc + Scal::TMP, sizeof(double)));
                double nrm2;
                EVSL_TRY(reorth(S, S.Q, nlock, 0, b2, &nrm2));
                EVSL_TRY(scale_vec(c, n, S.Q, 1.0 / std::sqrt(nrm2), nullptr));
            }
        }
    }
    // ---- outputs, sorted by eigenvalue
    std::vector<int> perm(nlock);
    std::iota(perm.begin(), perm.end(), 0);
    std::sort(perm.begin(), perm.end(), [&](int x, int y) { return lam_l[x] < lam_l[y]; });
    for (int i = 0; i < nlock; i++) {
        lam_out[i] = lam_l[perm[i]];
        res_out[i] = res_l[perm[i]];
    }
    if (Y_out && nlock > 0) {
        cudaPointerAttributes attr;
        bool ydev = (cudaPointerGetAttributes(&attr, Y_out) == cudaSuccess) &&
                    (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        if (ydev) {
            EVSL_TRY(h2d(c, S.idxd, perm.data(), sizeof(int) * nlock));
            EVSL_TRY(gather_cols(c, n, nlock, S.U, n, S.idxd, Y_out, n));
        } else {
            for (int i = 0; i < nlock; i++) {
                cudaError_t e = cudaMemcpyAsync(Y_out + (int64_t)i * n, S.U + (int64_t)perm[i] * n,
                                                sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
                if (e != cudaSuccess) return ctx_cuda(c, e, "eigenvector readback");
            }
        }
    }
    cudaEventRecord(tend, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanTr");
    *nev_out = nlock;
    if (st_out) {
        st_out->niter = its;
        st_out->nmv = S.nmv;
        st_out->nrestart = nrestart;
        st_out->npass = S.npass;
        st_out->t_filter = S.t_filter;
        st_out->t_orth = S.t_orth;
        st_out->t_restart = S.t_restart;
        st_out->t_total = ev_ms(tstart, tend) * 1e-3;
    }
    cudaEventDestroy(S.e0);
    cudaEventDestroy(S.e1);
    cudaEventDestroy(S.e2);
    cudaEventDestroy(tstart);
    cudaEventDestroy(tend);
    if (status == EVSL_ERR_CAPACITY) return ctx_fail(c, status, "more than cap=%d eigenpairs converged", cap);
    if (status == EVSL_ERR_NOCONV) return ctx_fail(c, status, "maxit=%d Lanczos steps reached", maxit);
    return EVSL_OK;
}
