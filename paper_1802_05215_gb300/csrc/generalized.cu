// Generalized symmetric-definite problems A x = lambda B x (Sec. 2.4-2.5) with a well-conditioned
// mass matrix B whose inverse is replaced by a polynomial (Sec. 4.3, lsPol): p(t) ~ 1/t on
// [bmin, bmax], applied to a vector with the Chebyshev three-term recurrence on
// Bhat = (B - bc I) / bh.  The filter is rho((A B^{-1} - c I) / d): every degree of its
// recurrence is one polynomial solve with B followed by one product with A, fused with the
// recurrence update and the coefficient accumulation.  On top of it:
//   - the pencil's spectral bounds by unfiltered Lanczos in the B-inner product (Algorithm 3);
//   - the pencil's KPM density (Sec. 2.1), with starting vectors q(B) v, q(t) ~ t^{-1/2};
//   - filtered non-restart Lanczos in the B-inner product with two full reorthogonalisation
//     passes (ChebLanNr);
//   - filtered thick-restart Lanczos with locking in the B-inner product (Algorithm 2).
// The eigenvectors come out B-orthonormal.
//
// Kernels: one sliced-ELLPACK step (k_gen_step, a warp per 32-row slice, lane = row) whose
// sparse operand u is separate from the shifted vector x, so that the same kernel serves the
// solve with B (u = x, on B's mapped values) and the filter degree with A (u = p(B) x).  The
// Lanczos vector updates, reorthogonalisation GEMVs, dot products and the small eigensolves are
// the dense helpers of the standard path.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "evsl_internal.h"

namespace {

constexpr int GTPB = 256;
constexpr double PI = 3.14159265358979323846;

// [gen_step begin] -- source region fingerprinted by the profile summaries
// Sparse step with M in sliced ELLPACK:
//   MODE 0: out = sc (M u - cc x);          y = c0 x + cj out
//   MODE 1: out = sc (M u - cc x) - xprev;  y += cj out
//   MODE 2: out = M u
// HAT: val holds the mapped (2/h)(M - c I) and u = x, so acc is already 2 Mhat x and the
// epilogue is out = acc / 2 (MODE 0) or out = acc - xprev (MODE 1); cc and sc are unused.
// out may alias xprev (each row reads xprev[r] before writing out[r]); u is gathered across
// rows and must not alias out or y.  STREAM: the matrix entries are loaded with the evict-first
// policy, so that the vectors, which the next step reads again, stay in L2 between launches
// (chosen by the launcher when one step's bytes exceed half of L2; below that, the normal
// policy keeps the matrix in L2 as well).
template <int MODE, bool HAT, bool STREAM>
__global__ void __launch_bounds__(GTPB)
k_gen_step(int64_t n, int64_t nslices, const int64_t *__restrict__ sptr, const int32_t *__restrict__ col,
           const double *__restrict__ val, const double *u, const double *x, const double *xprev,
           double *out, double *y, double cc, double sc, double c0, double cj)
{
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (s >= nslices) return;
    const int lane = threadIdx.x & 31;
    const int64_t b0 = sptr[s];
    const int w = (int)((sptr[s + 1] - b0) >> 5);
    double acc = 0.0;
#pragma unroll 4
    for (int j = 0; j < w; j++) {
        const int64_t p = b0 + 32 * (int64_t)j + lane;
        const double v = STREAM ? __ldcs(val + p) : val[p];
        const int ci = STREAM ? __ldcs(col + p) : col[p];
        acc = fma(v, u[ci], acc);
    }
    const int64_t r = s * 32 + lane;
    if (r >= n) return;
    if (MODE == 2) {
        out[r] = acc;
        return;
    }
    double wv;
    if (HAT) {
        wv = (MODE == 0) ? 0.5 * acc : acc - xprev[r];
    } else {
        wv = sc * (acc - cc * x[r]);
        if (MODE == 1) wv -= xprev[r];
    }
    out[r] = wv;
    y[r] = (MODE == 0) ? c0 * x[r] + cj * wv : y[r] + cj * wv;
}
// [gen_step end]

// vhat = (2/h)(M - c I) on the stored entries (padding stays 0); rows must store their diagonal
__global__ void k_gen_map(int64_t n, int64_t nslices, const int64_t *__restrict__ sptr, const int32_t *__restrict__ col,
                          const double *__restrict__ val, const int32_t *__restrict__ rlen, double c, double s2,
                          double *__restrict__ vhat)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t sl = r >> 5;
    if (sl >= nslices) return;
    const int lane = (int)(r & 31);
    const int w = (int)((sptr[sl + 1] - sptr[sl]) >> 5);
    const int len = (r < n) ? rlen[r] : 0;
    for (int j = 0; j < w; j++) {
        const int64_t e = sptr[sl] + 32 * (int64_t)j + lane;
        double v = 0.0;
        if (j < len) v = s2 * (val[e] - (col[e] == r ? c : 0.0));
        vhat[e] = v;
    }
}

template <int MODE, bool HAT = false>
int gen_step(evsl_ctx *c, const DevMatrix &M, const double *u, const double *x, const double *xprev,
             double *out, double *y, double cc, double sc, double c0, double cj)
{
    const unsigned grid = (unsigned)((M.nslices * 32 + GTPB - 1) / GTPB);
    const double *v = HAT ? M.vhat : M.val;
    if (stream_matrix(c, M.nstored, M.n, 8))
        k_gen_step<MODE, HAT, true><<<grid, GTPB, 0, c->stream>>>(M.n, M.nslices, M.sptr, M.col, v, u, x, xprev, out,
                                                                   y, cc, sc, c0, cj);
    else
        k_gen_step<MODE, HAT, false><<<grid, GTPB, 0, c->stream>>>(M.n, M.nslices, M.sptr, M.col, v, u, x, xprev, out,
                                                                    y, cc, sc, c0, cj);
    c->launches++;
    return check_launch(c, "generalized sparse step");
}

int d2h(evsl_ctx *c, void *dst, const void *src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "device-to-host copy");
}

// device scalars: alpha, a scratch norm, beta^2, (x, Bx), lambda, ||A x - lambda B x||^2,
// ||y||^2 of the filtered vector, then the projection coefficients h
enum { S_ALPHA = 0, S_TMP = 1, S_BETA2 = 2, S_NB2 = 3, S_LAM = 4, S_RES2 = 5, S_YN2 = 6, S_H = 8 };

// n-vectors of the generalized drivers (one workspace, carved); zs: fixed input of the
// filter graphs
struct Vecs {
    double *u, *t1, *t2, *f1, *f2, *z, *wt, *x, *ax, *bx, *zs;
    static constexpr int COUNT = 11;
};

int get_vecs(evsl_ctx *c, Vecs &v)
{
    const int64_t n = c->A.n;
    int st = EVSL_OK;
    double *p = (double *)ctx_ws(c, WS_GEN_VEC, sizeof(double) * (size_t)n * Vecs::COUNT, &st);
    if (st) return st;
    double **slots[Vecs::COUNT] = {&v.u, &v.t1, &v.t2, &v.f1, &v.f2, &v.z, &v.wt, &v.x, &v.ax, &v.bx, &v.zs};
    for (int i = 0; i < Vecs::COUNT; i++) *slots[i] = p + (int64_t)i * n;
    return EVSL_OK;
}

// y = p(B) x for a Chebyshev series p on [b_min, b_max]: y = c_0 x + c_1 w_1 + ...,
// w_1 = Bhat x, w_j = 2 Bhat w_{j-1} - w_{j-2}.  t1, t2: temporaries; y must not alias x, t1 or t2
// (x is only read).
int apply_poly_b(evsl_ctx *c, const std::vector<double> &cf, const double *x, double *y, double *t1, double *t2)
{
    const DevMatrix &B = c->B;
    const int deg = (int)cf.size() - 1;
    const double bc = 0.5 * (c->b_max + c->b_min), bh = 0.5 * (c->b_max - c->b_min);
    if (deg == 0) return scale_vec(c, B.n, const_cast<double *>(x), cf[0], y);
    const bool hat = B.vhat != nullptr;  // mapped values (2/bh)(B - bc I), made by set_csr_b
    if (hat) EVSL_TRY((gen_step<0, true>(c, B, x, x, nullptr, t1, y, bc, 1.0 / bh, cf[0], cf[1])));
    else EVSL_TRY(gen_step<0>(c, B, x, x, nullptr, t1, y, bc, 1.0 / bh, cf[0], cf[1]));
    const double *prev = x, *cur = t1;
    bool prev_tmp = false;  // prev is a temporary that the next term may overwrite
    for (int j = 2; j <= deg; j++) {
        double *out = prev_tmp ? const_cast<double *>(prev) : t2;
        if (hat) EVSL_TRY((gen_step<1, true>(c, B, cur, cur, prev, out, y, bc, 2.0 / bh, 0.0, cf[j])));
        else EVSL_TRY(gen_step<1>(c, B, cur, cur, prev, out, y, bc, 2.0 / bh, 0.0, cf[j]));
        prev = cur;
        cur = out;
        prev_tmp = true;
    }
    return EVSL_OK;
}

// y = p(B) x with the lsPol polynomial p ~ B^{-1} (the approximate solve with B)
int solve_b(evsl_ctx *c, const double *x, double *y, double *t1, double *t2)
{
    return apply_poly_b(c, c->b_coef, x, y, t1, t2);
}

// z = rho(Mhat) zi with Mhat = (A p(B) - cc I) / dd: f_1 = Mhat zi, f_j = 2 Mhat f_{j-1} - f_{j-2},
// z = sum_j c_j f_j.  z must not alias zi or the temporaries.  Counts deg products with A.
int filter_gen(evsl_ctx *c, const evsl_polfilt *pol, const double *zi, double *z, const Vecs &v, int64_t *nmv)
{
    const DevMatrix &A = c->A;
    const double cc = 0.5 * (pol->lmax + pol->lmin), dd = 0.5 * (pol->lmax - pol->lmin);
    const double *cf = pol->coef;
    const int deg = pol->deg;
    if (deg == 0) return scale_vec(c, A.n, const_cast<double *>(zi), cf[0], z);
    EVSL_TRY(solve_b(c, zi, v.u, v.t1, v.t2));
    EVSL_TRY(gen_step<0>(c, A, v.u, zi, nullptr, v.f1, z, cc, 1.0 / dd, cf[0], cf[1]));
    const double *prev = zi, *cur = v.f1;
    bool prev_tmp = false;
    for (int j = 2; j <= deg; j++) {
        EVSL_TRY(solve_b(c, cur, v.u, v.t1, v.t2));
        double *out = prev_tmp ? const_cast<double *>(prev) : v.f2;
        EVSL_TRY(gen_step<1>(c, A, v.u, cur, prev, out, z, cc, 2.0 / dd, 0.0, cf[j]));
        prev = cur;
        cur = out;
        prev_tmp = true;
    }
    *nmv += deg;
    return EVSL_OK;
}

// k_gen_step launches of one filter application: deg solves of deg(p) steps each, deg steps with A
int filter_gen_launches(const evsl_ctx *c, const evsl_polfilt *pol)
{
    return pol->deg * ((int)c->b_coef.size() - 1 + 1);
}

// z (= v.z) = rho(Mhat) zi.  Filters of degree >= 2 copy zi into v.zs and replay a cached CUDA
// graph of the launches (keyed by the filter, the polynomial inverse, both matrices and the
// buffers), which removes the host launch cost of the deg (deg(p) + 1) small launches; the
// kernels and their arguments are those of the direct path, so the results are bitwise equal.
int filter_gen_run(evsl_ctx *c, const evsl_polfilt *pol, const double *zi, const Vecs &v, int64_t *nmv)
{
    const int nl = filter_gen_launches(c, pol);
    if (pol->deg >= 2 && !c->graphs_off) {
        uint64_t h = 1469598103934665603ull;
        const char tag[] = "generalized filter";
        h = graph_key_hash(h, tag, sizeof tag);
        h = graph_key_hash(h, &pol->deg, sizeof pol->deg);
        h = graph_key_hash(h, &pol->lmin, sizeof pol->lmin);
        h = graph_key_hash(h, &pol->lmax, sizeof pol->lmax);
        h = graph_key_hash(h, pol->coef, sizeof(double) * (pol->deg + 1));
        h = graph_key_hash(h, c->b_coef.data(), sizeof(double) * c->b_coef.size());
        h = graph_key_hash(h, &c->b_min, sizeof c->b_min);
        h = graph_key_hash(h, &c->b_max, sizeof c->b_max);
        const void *ptrs[] = {c->A.sptr, c->A.col, c->A.val, c->B.sptr, c->B.col, c->B.val, c->B.vhat,
                              v.zs, v.z, v.u, v.t1, v.t2, v.f1, v.f2};
        h = graph_key_hash(h, ptrs, sizeof ptrs);
        h = graph_key_hash(h, &c->A.n, sizeof c->A.n);
        cudaError_t e = cudaMemcpyAsync(v.zs, zi, sizeof(double) * c->A.n, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "generalized filter input copy");
        const int r = graph_replay(c, h, EVSL_K_GEN_STEP, nl, [&]() {
            int64_t unused = 0;
            return filter_gen(c, pol, v.zs, v.z, v, &unused);
        });
        if (r != 1) {
            if (r == EVSL_OK) *nmv += pol->deg;
            return r;
        }
    }
    ProfGroup g;
    prof_begin(c, EVSL_K_GEN_STEP, &g);
    EVSL_TRY(filter_gen(c, pol, zi, v.z, v, nmv));
    prof_end(c, &g, nl);
    return EVSL_OK;
}

// Seeded start of Algorithm 3: w_1 uniform(-1, 1) (Lanczos stream, index 0), z_1 = B w_1, both
// scaled so that (w_1, z_1) = 1.
int lanab_start(evsl_ctx *c, uint64_t seed, double *W, double *Z, double *sc)
{
    const int64_t n = c->A.n;
    EVSL_TRY(fill_uniform_f64(c, n, seed, SM_STREAM_LANCZOS, 0, W));
    EVSL_TRY(gen_step<2>(c, c->B, W, nullptr, nullptr, Z, nullptr, 0.0, 0.0, 0.0, 0.0));
    EVSL_TRY(coldot(c, n, 1, W, n, Z, n, sc + S_NB2));
    double s2 = 0.0;
    EVSL_TRY(d2h(c, &s2, sc + S_NB2, sizeof(double)));
    if (!(s2 > 0.0)) return ctx_fail(c, EVSL_ERR_ARG, "generalized Lanczos: (w, B w) = %g; B is not positive definite", s2);
    const double inv = 1.0 / std::sqrt(s2);
    EVSL_TRY(scale_vec(c, n, W, inv, nullptr));
    return scale_vec(c, n, Z, inv, nullptr);
}

// One step of Algorithm 3 on z = Op w_i (already in z): z -= beta_i z_{i-1}; alpha = (z, w_i);
// z -= alpha z_i; two passes of z -= Z_{0..i} (W_{0..i}^T z); w = p(B) z;
// beta = (w, z)^{1/2}; w_{i+1} = w / beta, z_{i+1} = z / beta (skipped when beta = 0).
int lanab_step(evsl_ctx *c, int i, double *W, double *Z, double *z, double beta_i, const Vecs &v, double *sc,
               double *alpha, double *beta)
{
    const int64_t n = c->A.n;
    EVSL_TRY(lan_three_term(c, n, z, i > 0 ? Z + (int64_t)(i - 1) * n : nullptr, beta_i, W + (int64_t)i * n, z,
                            sc + S_ALPHA));
    EVSL_TRY(lan_sub_alpha(c, n, z, Z + (int64_t)i * n, sc + S_ALPHA, sc + S_TMP));
    for (int pass = 0; pass < 2; pass++) {
        EVSL_TRY(gemv_t2(c, n, W, i + 1, nullptr, 0, z, sc + S_H));
        EVSL_TRY(gemv_n2(c, n, Z, i + 1, nullptr, 0, sc + S_H, z, sc + S_TMP));
    }
    EVSL_TRY(solve_b(c, z, v.wt, v.t1, v.t2));
    EVSL_TRY(coldot(c, n, 1, v.wt, n, z, n, sc + S_BETA2));
    double hs[S_BETA2 + 1];
    EVSL_TRY(d2h(c, hs, sc, sizeof(hs)));
    *alpha = hs[S_ALPHA];
    const double b = std::sqrt(std::max(0.0, hs[S_BETA2]));
    if (b > 0.0) {
        EVSL_TRY(scale_vec(c, n, v.wt, 1.0 / b, W + (int64_t)(i + 1) * n));
        EVSL_TRY(scale_vec(c, n, z, 1.0 / b, Z + (int64_t)(i + 1) * n));
    }
    *beta = b;
    return EVSL_OK;
}

// bases W, Z (n x (k+1) each), extra_cols more columns at *X, and the device scalars with room
// for hcap projection coefficients
int get_basis(evsl_ctx *c, int k, int extra_cols, double **W, double **Z, double **X, double **sc, int hcap)
{
    const int64_t n = c->A.n;
    int st = EVSL_OK;
    double *p = (double *)ctx_ws(c, WS_GEN_BASIS, sizeof(double) * (size_t)n * (2 * (size_t)(k + 1) + extra_cols), &st);
    if (st) return st;
    *W = p;
    *Z = p + (int64_t)(k + 1) * n;
    if (X) *X = p + 2 * (int64_t)(k + 1) * n;
    *sc = (double *)ctx_ws(c, WS_GEN_SCAL, sizeof(double) * (S_H + (size_t)hcap + 8), &st);
    return st;
}

// eigenpairs of the leading k x k block of the tridiagonal (ld ldt, column-major, host):
// eigenvalues to w (host, unordered), vectors to the device buffer *V (ld *ldv)
int tri_eig(evsl_ctx *c, int k, const std::vector<double> &T, int ldt, std::vector<double> &w, double **V, int *ldv)
{
    std::vector<double> Tk((size_t)k * k);
    for (int j = 0; j < k; j++)
        for (int i = 0; i < k; i++) Tk[(size_t)j * k + i] = T[(size_t)j * ldt + i];
    const int M = std::max(2, k + (k & 1));
    int st = EVSL_OK;
    *V = (double *)ctx_ws(c, WS_LAN_T, sizeof(double) * (size_t)M * M, &st);
    if (st) return st;
    w.assign(k, 0.0);
    int sweeps = 0;
    return jacobi_eig(c, k, Tk.data(), w.data(), *V, ldv, &sweeps);
}

int check_pencil(evsl_ctx *c, const char *what)
{
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "%s: no matrix A set", what);
    if (c->B.n == 0 || c->b_coef.empty()) return ctx_fail(c, EVSL_ERR_STATE, "%s: no matrix B set", what);
    if (c->B.n != c->A.n)
        return ctx_fail(c, EVSL_ERR_STATE, "%s: A has %lld rows, B %lld", what, (long long)c->A.n, (long long)c->B.n);
    return EVSL_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Chebyshev interpolant of f(t) = 1/t (kind 0, the solve with B) or f(t) = t^{-1/2} (kind 1, the
// starting vectors of the pencil's density) on [bmin, bmax] at the N = k + 1 Chebyshev-Gauss points
// theta_q = pi (q + 1/2) / N: c_j = (2 - [j = 0]) / N sum_q cos(j theta_q) f(t(theta_q)),
// t(theta) = bc + bh cos(theta).  The degree is the smallest k <= maxdeg with
// max |p(t) / f(t) - 1| <= eps over 2001 equispaced points of [bmin, bmax] (p by Clenshaw's sum).
int host_lspol(double bmin, double bmax, double eps, int maxdeg, int *deg, double *coef, double *err, int kind)
{
    const double bc = 0.5 * (bmax + bmin), bh = 0.5 * (bmax - bmin);
    const int NPTS = 2001;
    double e = 0.0;
    for (int k = 1; k <= maxdeg; k++) {
        const int N = k + 1;
        std::vector<double> th(N), f(N);
        for (int q = 0; q < N; q++) {
            th[q] = PI * (q + 0.5) / N;
            const double t = bc + bh * std::cos(th[q]);
            f[q] = (kind == 0) ? 1.0 / t : 1.0 / std::sqrt(t);
        }
        for (int j = 0; j <= k; j++) {
            double s = 0.0;
            for (int q = 0; q < N; q++) s += std::cos(j * th[q]) * f[q];
            coef[j] = s * (j == 0 ? 1.0 : 2.0) / N;
        }
        e = 0.0;
        for (int q = 0; q < NPTS; q++) {
            const double t = bmin + (bmax - bmin) * q / (NPTS - 1);
            const double x = (t - bc) / bh;
            double b1 = 0.0, b2 = 0.0;  // Clenshaw: b_j = c_j + 2 x b_{j+1} - b_{j+2}
            for (int j = k; j >= 1; j--) {
                const double b0 = coef[j] + 2.0 * x * b1 - b2;
                b2 = b1;
                b1 = b0;
            }
            const double p = coef[0] + x * b1 - b2;
            e = std::max(e, std::fabs((kind == 0 ? t : std::sqrt(t)) * p - 1.0));
        }
        if (e <= eps) {
            *deg = k;
            if (err) *err = e;
            return EVSL_OK;
        }
    }
    *deg = maxdeg;
    if (err) *err = e;
    return EVSL_ERR_NOCONV;
}

// Mapped values (2/bh)(B - bc I) of the current B for the solve's recurrence, when every row
// of B stores its diagonal (else the solve uses B's values and the explicit shift).
int gen_map_b(evsl_ctx *c)
{
    DevMatrix &B = c->B;
    if (!B.has_diag || B.n == 0) return EVSL_OK;
    if (!B.vhat) EVSL_TRY(ctx_alloc(c, (void **)&B.vhat, sizeof(double) * B.nstored));
    const double bc = 0.5 * (c->b_max + c->b_min), bh = 0.5 * (c->b_max - c->b_min);
    k_gen_map<<<(unsigned)((B.nslices * 32 + 255) / 256), 256, 0, c->stream>>>(B.n, B.nslices, B.sptr, B.col, B.val,
                                                                               B.rlen, bc, 2.0 / bh, B.vhat);
    c->launches++;
    EVSL_TRY(check_launch(c, "generalized value mapping"));
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "generalized value mapping");
}

int drv_polyB_apply(evsl_ctx *c, const double *x, double *y)
{
    if (c->B.n == 0 || c->b_coef.empty()) return ctx_fail(c, EVSL_ERR_STATE, "polyB_apply: no matrix B set");
    const int64_t n = c->B.n;
    int st = EVSL_OK;
    double *t = (double *)ctx_ws(c, WS_GEN_VEC, sizeof(double) * (size_t)n * Vecs::COUNT, &st);
    if (st) return st;
    ProfGroup g;
    prof_begin(c, EVSL_K_GEN_STEP, &g);
    EVSL_TRY(solve_b(c, x, y, t, t + n));
    prof_end(c, &g, (int)c->b_coef.size() - 1);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "polyB_apply");
}

// Bounds of the pencil's spectrum from `steps` unfiltered steps of Algorithm 3 on B^{-1} A:
// lmin = theta_1 - |beta s_{m,1}|, lmax = theta_m + |beta s_{m,m}|.
int drv_bounds_gen(evsl_ctx *c, int steps, uint64_t seed, double *lmin, double *lmax)
{
    EVSL_TRY(check_pencil(c, "bounds_gen"));
    const int64_t n = c->A.n;
    if (steps > n) steps = (int)n;
    double *W, *Z, *sc;
    EVSL_TRY(get_basis(c, steps, 0, &W, &Z, nullptr, &sc, steps + 1));
    Vecs v;
    EVSL_TRY(get_vecs(c, v));
    EVSL_TRY(lanab_start(c, seed, W, Z, sc));
    std::vector<double> T((size_t)steps * steps, 0.0);
    double beta = 0.0;
    int m = 0;
    for (int i = 0; i < steps; i++) {
        EVSL_TRY(gen_step<2>(c, c->A, W + (int64_t)i * n, nullptr, nullptr, v.z, nullptr, 0.0, 0.0, 0.0, 0.0));
        double alpha = 0.0, bn = 0.0;
        EVSL_TRY(lanab_step(c, i, W, Z, v.z, beta, v, sc, &alpha, &bn));
        T[(size_t)i * steps + i] = alpha;
        m = i + 1;
        beta = bn;
        if (i + 1 < steps) {
            T[(size_t)(i + 1) * steps + i] = beta;
            T[(size_t)i * steps + i + 1] = beta;
        }
        if (!(beta > 0.0)) break;
    }
    std::vector<double> w;
    double *V = nullptr;
    int ldv = 0;
    EVSL_TRY(tri_eig(c, m, T, steps, w, &V, &ldv));
    const int imin = (int)(std::min_element(w.begin(), w.end()) - w.begin());
    const int imax = (int)(std::max_element(w.begin(), w.end()) - w.begin());
    double smin = 0.0, smax = 0.0;
    EVSL_TRY(d2h(c, &smin, V + (int64_t)imin * ldv + (m - 1), sizeof(double)));
    EVSL_TRY(d2h(c, &smax, V + (int64_t)imax * ldv + (m - 1), sizeof(double)));
    *lmin = w[imin] - std::fabs(beta * smin);
    *lmax = w[imax] + std::fabs(beta * smax);
    return EVSL_OK;
}

// Filtered non-restart Lanczos for A x = lambda B x: Algorithm 3 on the pencil (B rho, B) with
// the operator rho((A B^{-1} - c I) / d) applied to z_i.  Every ncycle steps the Ritz values
// >= bar of T_k are summed; extraction when the sum is stable (relative change < tau1), at the
// basis limit m, or on breakdown; a run whose Ritz values stayed below bar for
// max(2 ncycle, m / 4) steps ends with none.  Extraction: for Ritz values >= bar (largest
// first), x = W y scaled to (x, B x) = 1, lambda = x^T A x, kept inside the slice, converged if
// ||A x - lambda B x|| <= tol ||B|| max(|lmin|, |lmax|) (||B|| by bmax).  Unconverged
// candidates continue the basis.  Eigenpairs are returned in ascending order.
int drv_chebLanNr_gen(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *o, int cap,
                      int *nev, double *lam, double *Y, double *res, evsl_stats *stats)
{
    EVSL_TRY(check_pencil(c, "chebLanNr_gen"));
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t n = c->A.n;
    int m = o->m;
    if (m > n) m = (int)n;
    const int ncycle = o->ncycle > 0 ? o->ncycle : 10;
    const double bar = pol->bar;
    const double scale = c->b_max * std::max(std::fabs(pol->lmin), std::fabs(pol->lmax));
    double *W, *Z, *Xc, *sc;
    EVSL_TRY(get_basis(c, m, cap, &W, &Z, &Xc, &sc, m + 1));
    Vecs v;
    EVSL_TRY(get_vecs(c, v));
    EVSL_TRY(lanab_start(c, o->seed, W, Z, sc));
    const int ldt = m + 1;
    std::vector<double> T((size_t)ldt * ldt, 0.0), w;
    std::vector<double> lam_c(cap), res_c(cap);
    int64_t nmv = 0;
    int its = 0, status = EVSL_OK, found = 0, prev_nabove = 0;
    bool have_old = false;
    double t_old = 0.0, beta = 0.0;
    for (int i = 0; i < m; i++) {
        its++;
        EVSL_TRY(filter_gen_run(c, pol, Z + (int64_t)i * n, v, &nmv));
        double alpha = 0.0, bn = 0.0;
        EVSL_TRY(lanab_step(c, i, W, Z, v.z, beta, v, sc, &alpha, &bn));
        T[(size_t)i * ldt + i] = alpha;
        beta = bn;
        T[(size_t)(i + 1) * ldt + i] = beta;
        T[(size_t)i * ldt + i + 1] = beta;
        const int k = i + 1;
        bool extract = (k == m) || !(beta > 0.0);
        double *V = nullptr;
        int ldv = 0;
        if (!extract && k % ncycle == 0) {
            EVSL_TRY(tri_eig(c, k, T, ldt, w, &V, &ldv));
            double t_new = 0.0;
            int nabove = 0;
            for (double th : w)
                if (th >= bar) {
                    t_new += th;
                    nabove++;
                }
            const int min_empty = std::max(2 * ncycle, m / 4);
            if (have_old && nabove == 0 && prev_nabove == 0 && k >= min_empty) break;
            if (have_old && nabove > 0 && std::fabs(t_new - t_old) < o->tau1 * std::max(1.0, std::fabs(t_new)))
                extract = true;
            t_old = t_new;
            prev_nabove = nabove;
            have_old = true;
        }
        if (!extract) continue;
        EVSL_TRY(tri_eig(c, k, T, ldt, w, &V, &ldv));
        std::vector<int> order(k);
        for (int j = 0; j < k; j++) order[j] = j;
        std::sort(order.begin(), order.end(), [&](int p, int q) { return w[p] > w[q]; });
        int nconv = 0, nunconv = 0;
        for (int jj : order) {
            if (w[jj] < bar) break;
            EVSL_TRY(gemm_nn(c, n, 1, k, W, n, V + (int64_t)jj * ldv, ldv, v.x, n));
            EVSL_TRY(gen_step<2>(c, c->B, v.x, nullptr, nullptr, v.bx, nullptr, 0.0, 0.0, 0.0, 0.0));
            EVSL_TRY(coldot(c, n, 1, v.x, n, v.bx, n, sc + S_NB2));
            double nb2 = 0.0;
            EVSL_TRY(d2h(c, &nb2, sc + S_NB2, sizeof(double)));
            if (!(nb2 > 0.0)) return ctx_fail(c, EVSL_ERR_ARG, "chebLanNr_gen: (x, B x) = %g; B is not positive definite", nb2);
            const double inv = 1.0 / std::sqrt(nb2);
            EVSL_TRY(scale_vec(c, n, v.x, inv, nullptr));
            EVSL_TRY(scale_vec(c, n, v.bx, inv, nullptr));
            EVSL_TRY(gen_step<2>(c, c->A, v.x, nullptr, nullptr, v.ax, nullptr, 0.0, 0.0, 0.0, 0.0));
            EVSL_TRY(coldot(c, n, 1, v.x, n, v.ax, n, sc + S_LAM));
            EVSL_TRY(colres2(c, n, 1, v.ax, v.bx, n, sc + S_LAM, sc + S_RES2));
            double lr[2];
            EVSL_TRY(d2h(c, lr, sc + S_LAM, sizeof(lr)));
            const double lamj = lr[0];
            const bool inside = lamj >= a && (o->right_closed ? lamj <= b : lamj < b);
            if (!inside) continue;
            const double rj = std::sqrt(std::max(0.0, lr[1])) / scale;
            if (rj > o->tol) {
                nunconv++;
                continue;
            }
            if (nconv >= cap) {
                status = EVSL_ERR_CAPACITY;
                break;
            }
            cudaError_t e = cudaMemcpyAsync(Xc + (int64_t)nconv * n, v.x, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                            c->stream);
            if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanNr_gen eigenvector copy");
            lam_c[nconv] = lamj;
            res_c[nconv] = rj;
            nconv++;
        }
        found = nconv;
        if (status == EVSL_ERR_CAPACITY) break;
        if (nunconv == 0 || k == m || !(beta > 0.0)) {
            if (nunconv > 0) status = EVSL_ERR_NOCONV;
            break;
        }
        have_old = false;
    }
    std::vector<int> perm(found);
    for (int i = 0; i < found; i++) perm[i] = i;
    std::sort(perm.begin(), perm.end(), [&](int p, int q) { return lam_c[p] < lam_c[q]; });
    for (int i = 0; i < found; i++) {
        lam[i] = lam_c[perm[i]];
        res[i] = res_c[perm[i]];
        if (Y) {
            cudaError_t e = cudaMemcpyAsync(Y + (int64_t)i * n, Xc + (int64_t)perm[i] * n, sizeof(double) * n,
                                            cudaMemcpyDefault, c->stream);
            if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanNr_gen eigenvector readback");
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanNr_gen outputs");
    *nev = found;
    if (stats) {
        *stats = evsl_stats();
        stats->niter = its;
        stats->nmv = nmv;
        stats->t_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

// KPM moments of the pencil (the density of S = B^{-1/2} A B^{-1/2}, whose eigenvalues are the
// pencil's): for Rademacher probes v_l (the KPM stream and indexing of the standard moments),
// u_l = q(B) v_l ~ B^{-1/2} v_l and y_0 = B u_l, mu_k = (1/nvec) sum_l u_l^T y_k with
// y_1 = Mhat y_0, y_{k+1} = 2 Mhat y_k - y_{k-1}, Mhat = (A p(B) - cI)/d -- the generalized
// filter's step, since v^T T_k(Shat) v = u^T B T_k((B^{-1}A - cI)/d) u = u^T T_k(Mhat) B u.
// Each probe's moments go to a device row (deterministic dot products); the host adds the rows
// in probe order.  The recurrence steps write their unused y accumulator into a scratch vector.
int drv_kpm_gen(evsl_ctx *c, int M, int nvec, uint64_t seed, double lmin, double lmax, double *mu)
{
    EVSL_TRY(check_pencil(c, "kpm_dos_gen"));
    if (c->b_coef_isqrt.empty()) return ctx_fail(c, EVSL_ERR_STATE, "kpm_dos_gen: no B^{-1/2} polynomial");
    const int64_t n = c->A.n;
    int st = EVSL_OK;
    double *p = (double *)ctx_ws(c, WS_GEN_VEC, sizeof(double) * (size_t)n * Vecs::COUNT, &st);
    if (st) return st;
    double *v = p, *u = p + n, *ya = p + 2 * n, *yb = p + 3 * n, *sv = p + 4 * n, *t1 = p + 5 * n,
           *t2 = p + 6 * n, *scr = p + 7 * n;
    const size_t rows = (size_t)nvec * (M + 1);
    double *mud = (double *)ctx_ws(c, WS_GEN_MU, sizeof(double) * rows, &st);
    if (st) return st;
    const double cc = 0.5 * (lmax + lmin), dd = 0.5 * (lmax - lmin);
    const DevMatrix &A = c->A;
    for (int l = 0; l < nvec; l++) {
        double *row = mud + (size_t)l * (M + 1);
        EVSL_TRY(fill_rademacher_f64(c, n, seed, SM_STREAM_KPM, (uint64_t)l, v));
        EVSL_TRY(apply_poly_b(c, c->b_coef_isqrt, v, u, t1, t2));                       // u = q(B) v
        EVSL_TRY(gen_step<2>(c, c->B, u, nullptr, nullptr, ya, nullptr, 0.0, 0.0, 0.0, 0.0));  // y_0 = B u
        EVSL_TRY(coldot(c, n, 1, u, n, ya, n, row));
        const double *prev = nullptr;
        double *cur = ya;
        for (int k = 1; k <= M; k++) {
            EVSL_TRY(solve_b(c, cur, sv, t1, t2));                                           // p(B) y_{k-1}
            double *out;
            if (k == 1) {
                out = yb;
                EVSL_TRY(gen_step<0>(c, A, sv, cur, nullptr, out, scr, cc, 1.0 / dd, 0.0, 0.0));
            } else {
                out = const_cast<double *>(prev);  // y_{k-2}'s buffer, read before it is written
                EVSL_TRY(gen_step<1>(c, A, sv, cur, prev, out, scr, cc, 2.0 / dd, 0.0, 0.0));
            }
            prev = cur;
            cur = out;
            EVSL_TRY(coldot(c, n, 1, u, n, cur, n, row + k));
        }
    }
    std::vector<double> h(rows);
    cudaError_t e = cudaMemcpyAsync(h.data(), mud, sizeof(double) * rows, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "kpm_dos_gen readback");
    for (int k = 0; k <= M; k++) {
        double sum = 0.0;
        for (int l = 0; l < nvec; l++) sum += h[(size_t)l * (M + 1) + k];
        mu[k] = sum / nvec;
    }
    return EVSL_OK;
}

// ------------------------------------------------------------------------------------------
// Thick-restart filtered Lanczos with locking for the pencil (Algorithm 2 in the B-inner
// product).  Vectors come in pairs (w, z = B w) with W^T Z = I; locked eigenvectors U are
// B-orthonormal and BU = B U is kept beside them, so deflating a z-vector is z -= BU (U^T z)
// (the paper's (I - B U U^T) scheme, Sec. 2.5).
namespace {

struct TrGen {
    evsl_ctx *c;
    int64_t n;
    double *W, *Z, *U, *BU, *trw, *trz, *sc;
    Vecs v;
    uint64_t seed, fresh_index = 0;
    int nlock = 0;

    // one classical Gram-Schmidt pass of x against [P1 (k1 columns), P2 (k2)] with update
    // columns [Q1, Q2]: x -= [Q1 Q2] ([P1 P2]^T x)
    int pass(double *x, const double *P1, const double *Q1, int k1, const double *P2, const double *Q2, int k2)
    {
        if (k1 + k2 == 0) return EVSL_OK;
        EVSL_TRY(gemv_t2(c, n, k1 ? P1 : P2, k1 ? k1 : k2, k1 ? P2 : nullptr, k1 ? k2 : 0, x, sc + S_H));
        return gemv_n2(c, n, k1 ? Q1 : Q2, k1 ? k1 : k2, k1 ? Q2 : nullptr, k1 ? k2 : 0, sc + S_H, x, sc + S_TMP);
    }

    // two passes of z -= BU (U^T z) and z -= Z (W^T z) over the first k basis pairs
    int reorth(double *z, int k)
    {
        for (int p = 0; p < 2; p++) EVSL_TRY(pass(z, U, BU, nlock, W, Z, k));
        return EVSL_OK;
    }

    // fresh pair into (w, z): w uniform(-1, 1) (Lanczos stream, next index), made B-orthogonal to
    // U and the first k basis vectors (w -= U (BU^T w), w -= W (Z^T w), twice), z = B w, w^T z = 1
    int fresh(double *w, double *z, int k)
    {
        EVSL_TRY(fill_uniform_f64(c, n, seed, SM_STREAM_LANCZOS, fresh_index++, w));
        for (int p = 0; p < 2; p++) EVSL_TRY(pass(w, BU, U, nlock, Z, W, k));
        EVSL_TRY(gen_step<2>(c, c->B, w, nullptr, nullptr, z, nullptr, 0.0, 0.0, 0.0, 0.0));
        EVSL_TRY(coldot(c, n, 1, w, n, z, n, sc + S_NB2));
        double s2 = 0.0;
        EVSL_TRY(d2h(c, &s2, sc + S_NB2, sizeof(double)));
        if (!(s2 > 0.0)) return ctx_fail(c, EVSL_ERR_ARG, "chebLanTr_gen: (w, B w) = %g; B is not positive definite", s2);
        const double inv = 1.0 / std::sqrt(s2);
        EVSL_TRY(scale_vec(c, n, w, inv, nullptr));
        return scale_vec(c, n, z, inv, nullptr);
    }

    // close a step on z (= v.z, reorthogonalised): w = p(B) z, beta = (w^T z)^{1/2}; the next pair
    // is (w, z) / beta, or a fresh pair after a breakdown (beta <= 1e-13 ||y|| / sqrt(bmax), ||y||^2
    // in sc[S_YN2]); returns beta (0 after a breakdown) and alpha from sc[S_ALPHA]
    int close(int next, double *alpha, double *beta)
    {
        EVSL_TRY(solve_b(c, v.z, v.wt, v.t1, v.t2));
        EVSL_TRY(coldot(c, n, 1, v.wt, n, v.z, n, sc + S_BETA2));
        double hs[S_YN2 + 1];
        EVSL_TRY(d2h(c, hs, sc, sizeof(hs)));
        *alpha = hs[S_ALPHA];
        const double b = std::sqrt(std::max(0.0, hs[S_BETA2]));
        double *wn = W + (int64_t)next * n, *zn = Z + (int64_t)next * n;
        if (b > 1e-13 * std::sqrt(std::max(0.0, hs[S_YN2])) / std::sqrt(c->b_max)) {
            EVSL_TRY(scale_vec(c, n, v.wt, 1.0 / b, wn));
            EVSL_TRY(scale_vec(c, n, v.z, 1.0 / b, zn));
            *beta = b;
        } else {
            EVSL_TRY(fresh(wn, zn, next));
            *beta = 0.0;
        }
        return EVSL_OK;
    }
};

}  // namespace

// Filtered thick-restart Lanczos with locking for A x = lambda B x.  The control flow of the
// standard solver's Algorithm 2 (special TR step with the arrow matrix, early restart on the sum
// of Ritz values >= bar every ncycle steps, candidates largest first, at most m/2 TR pairs
// (W s, Z s), fresh pairs after breakdown or a cycle without candidates, stop after two such
// cycles); locking when ||A x - lambda B x|| <= tol bmax max(|lmin|, |lmax|) with x = W s
// B-normalised and lambda = x^T A x.  No refinement of stalled candidates.  FP64.
int drv_chebLanTr_gen(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *o, int cap,
                      int *nev, double *lam, double *Y, double *res, evsl_stats *stats)
{
    EVSL_TRY(check_pencil(c, "chebLanTr_gen"));
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t n = c->A.n;
    int m = o->m;
    if (m > n) m = (int)n;
    const int maxit = o->maxit > 0 ? o->maxit : 20 * m;
    const int ncycle = o->ncycle > 0 ? o->ncycle : 10;
    const int trcap = m / 2 + 1;
    const double bar = pol->bar;
    const double scale = c->b_max * std::max(std::fabs(pol->lmin), std::fabs(pol->lmax));
    TrGen g;
    g.c = c;
    g.n = n;
    g.seed = o->seed;
    double *X = nullptr;
    EVSL_TRY(get_basis(c, m, 2 * cap + 2 * trcap, &g.W, &g.Z, &X, &g.sc, cap + m + 2));
    g.U = X;
    g.BU = X + (int64_t)cap * n;
    g.trw = X + 2 * (int64_t)cap * n;
    g.trz = g.trw + (int64_t)trcap * n;
    EVSL_TRY(get_vecs(c, g.v));
    const Vecs &v = g.v;
    double *W = g.W, *Z = g.Z, *sc = g.sc;
    const int ldt = m + 1;
    std::vector<double> T((size_t)ldt * ldt), w, trtheta(trcap), trs(trcap), lam_c(cap), res_c(cap);
    int64_t nmv = 0, nrestart = 0;
    int its = 0, l = 0, nocand = 0, status = EVSL_OK;

    EVSL_TRY(g.fresh(W, Z, 0));
    while (its <= maxit) {
        int k;
        std::fill(T.begin(), T.end(), 0.0);
        if (l > 0) {
            for (int j = 0; j < l; j++) {
                T[(size_t)j * ldt + j] = trtheta[j];
                T[(size_t)l * ldt + j] = trs[j];
                T[(size_t)j * ldt + l] = trs[j];
            }
            const double *zl = Z + (int64_t)l * n, *wl = W + (int64_t)l * n;
            EVSL_TRY(filter_gen_run(c, pol, zl, v, &nmv));
            its++;
            EVSL_TRY(coldot(c, n, 1, v.z, n, v.z, n, sc + S_YN2));
            EVSL_TRY(coldot(c, n, 1, wl, n, v.z, n, sc + S_ALPHA));     // alpha = w_l^T y
            cudaError_t e = cudaMemcpyAsync(sc + S_H, trs.data(), sizeof(double) * l, cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanTr_gen arrow upload");
            EVSL_TRY(gemv_n2(c, n, Z, l, nullptr, 0, sc + S_H, v.z, sc + S_TMP));   // z -= sum_j s_j z_j
            EVSL_TRY(lan_sub_alpha(c, n, v.z, zl, sc + S_ALPHA, sc + S_TMP));
            EVSL_TRY(g.reorth(v.z, l + 1));
            double alpha = 0.0, beta = 0.0;
            EVSL_TRY(g.close(l + 1, &alpha, &beta));
            T[(size_t)l * ldt + l] = alpha;
            T[(size_t)(l + 1) * ldt + l] = beta;
            T[(size_t)l * ldt + l + 1] = beta;
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
            const double *zi = Z + (int64_t)i * n, *wi = W + (int64_t)i * n;
            EVSL_TRY(filter_gen_run(c, pol, zi, v, &nmv));
            EVSL_TRY(coldot(c, n, 1, v.z, n, v.z, n, sc + S_YN2));
            const double bi = i > 0 ? T[(size_t)i * ldt + i - 1] : 0.0;
            EVSL_TRY(lan_three_term(c, n, v.z, i > 0 ? Z + (int64_t)(i - 1) * n : nullptr, bi, wi, v.z, sc + S_ALPHA));
            EVSL_TRY(lan_sub_alpha(c, n, v.z, zi, sc + S_ALPHA, sc + S_TMP));
            EVSL_TRY(g.reorth(v.z, i + 1));
            double alpha = 0.0, beta = 0.0;
            EVSL_TRY(g.close(i + 1, &alpha, &beta));
            T[(size_t)i * ldt + i] = alpha;
            T[(size_t)(i + 1) * ldt + i] = beta;
            T[(size_t)i * ldt + i + 1] = beta;
            k = i + 1;
            if ((k - lstart) % ncycle == 0) {
                double *V = nullptr;
                int ldv = 0;
                EVSL_TRY(tri_eig(c, k, T, ldt, w, &V, &ldv));
                double t_new = 0.0;
                int nabove = 0;
                for (double th : w)
                    if (th >= bar) {
                        t_new += th;
                        nabove++;
                    }
                if (have_old && nabove > 0 && std::fabs(t_new - t_old) < o->tau1 * std::max(1.0, std::fabs(t_new))) break;
                const int min_empty = std::max(2 * ncycle, m / 4);
                if (have_old && nabove == 0 && prev_nabove == 0 && k - lstart >= min_empty) break;
                t_old = t_new;
                prev_nabove = nabove;
                have_old = true;
            }
            if (its > maxit) break;
        }
        // restart: Ritz pairs of T_k
        nrestart++;
        double *V = nullptr;
        int ldv = 0;
        EVSL_TRY(tri_eig(c, k, T, ldt, w, &V, &ldv));
        const double betak = T[(size_t)(k - 1) * ldt + k];
        std::vector<int> order(k);
        for (int j = 0; j < k; j++) order[j] = j;
        std::sort(order.begin(), order.end(), [&](int p, int q) { return w[p] > w[q]; });
        int ncand = 0, ntr = 0;
        for (int jj : order) {
            if (w[jj] < bar) break;
            const double *s = V + (int64_t)jj * ldv;
            EVSL_TRY(gemm_nn(c, n, 1, k, W, n, s, ldv, v.x, n));     // x = W s
            EVSL_TRY(gemm_nn(c, n, 1, k, Z, n, s, ldv, v.f1, n));    // B x = Z s (the z-side of the pair)
            EVSL_TRY(gen_step<2>(c, c->B, v.x, nullptr, nullptr, v.bx, nullptr, 0.0, 0.0, 0.0, 0.0));
            EVSL_TRY(coldot(c, n, 1, v.x, n, v.bx, n, sc + S_NB2));
            double sh[2];  // (x, B x), s_k (last component of the Ritz vector)
            EVSL_TRY(d2h(c, sh, sc + S_NB2, sizeof(double)));
            EVSL_TRY(d2h(c, sh + 1, s + (k - 1), sizeof(double)));
            if (!(sh[0] > 0.0)) return ctx_fail(c, EVSL_ERR_ARG, "chebLanTr_gen: (x, B x) = %g; B is not positive definite", sh[0]);
            const double inv = 1.0 / std::sqrt(sh[0]);
            EVSL_TRY(scale_vec(c, n, v.x, inv, v.f2));               // u = x / ||x||_B
            EVSL_TRY(scale_vec(c, n, v.bx, inv, nullptr));
            EVSL_TRY(gen_step<2>(c, c->A, v.f2, nullptr, nullptr, v.ax, nullptr, 0.0, 0.0, 0.0, 0.0));
            EVSL_TRY(coldot(c, n, 1, v.f2, n, v.ax, n, sc + S_LAM));
            EVSL_TRY(colres2(c, n, 1, v.ax, v.bx, n, sc + S_LAM, sc + S_RES2));
            double lr[2];
            EVSL_TRY(d2h(c, lr, sc + S_LAM, sizeof(lr)));
            const double lamj = lr[0];
            const bool inside = lamj >= a && (o->right_closed ? lamj <= b : lamj < b);
            if (!inside) continue;
            ncand++;
            const double rj = std::sqrt(std::max(0.0, lr[1])) / scale;
            if (rj <= o->tol) {
                if (g.nlock >= cap) {
                    status = EVSL_ERR_CAPACITY;
                    break;
                }
                cudaError_t e = cudaMemcpyAsync(g.U + (int64_t)g.nlock * n, v.f2, sizeof(double) * n,
                                                cudaMemcpyDeviceToDevice, c->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(g.BU + (int64_t)g.nlock * n, v.bx, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                        c->stream);
                if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanTr_gen lock");
                lam_c[g.nlock] = lamj;
                res_c[g.nlock] = rj;
                g.nlock++;
            } else if (ntr < m / 2) {
                cudaError_t e = cudaMemcpyAsync(g.trw + (int64_t)ntr * n, v.x, sizeof(double) * n,
                                                cudaMemcpyDeviceToDevice, c->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(g.trz + (int64_t)ntr * n, v.f1, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                        c->stream);
                if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanTr_gen TR copy");
                trtheta[ntr] = w[jj];
                trs[ntr] = betak * sh[1];
                ntr++;
            }
        }
        if (status == EVSL_ERR_CAPACITY) break;
        nocand = (ncand == 0) ? nocand + 1 : 0;
        if (nocand >= 2) break;
        if (its > maxit) {
            status = EVSL_ERR_NOCONV;
            break;
        }
        if (ncand == 0) {
            l = 0;
            EVSL_TRY(g.fresh(W, Z, 0));
        } else {
            cudaError_t e = cudaSuccess;
            if (ntr != k) {
                e = cudaMemcpyAsync(W + (int64_t)ntr * n, W + (int64_t)k * n, sizeof(double) * n,
                                    cudaMemcpyDeviceToDevice, c->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(Z + (int64_t)ntr * n, Z + (int64_t)k * n, sizeof(double) * n,
                                        cudaMemcpyDeviceToDevice, c->stream);
            }
            if (e == cudaSuccess && ntr > 0)
                e = cudaMemcpyAsync(W, g.trw, sizeof(double) * n * ntr, cudaMemcpyDeviceToDevice, c->stream);
            if (e == cudaSuccess && ntr > 0)
                e = cudaMemcpyAsync(Z, g.trz, sizeof(double) * n * ntr, cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanTr_gen restart copy");
            l = ntr;
            if (l == 0) {
                // continue from z_{k+1}, deflated against the new locked pairs
                for (int p = 0; p < 2; p++) EVSL_TRY(g.pass(Z, g.U, g.BU, g.nlock, nullptr, nullptr, 0));
                EVSL_TRY(solve_b(c, Z, W, v.t1, v.t2));
                EVSL_TRY(coldot(c, n, 1, W, n, Z, n, sc + S_NB2));
                double s2 = 0.0;
                EVSL_TRY(d2h(c, &s2, sc + S_NB2, sizeof(double)));
                if (!(s2 > 0.0)) return ctx_fail(c, EVSL_ERR_ARG, "chebLanTr_gen: (w, z) = %g after deflation", s2);
                const double inv = 1.0 / std::sqrt(s2);
                EVSL_TRY(scale_vec(c, n, W, inv, nullptr));
                EVSL_TRY(scale_vec(c, n, Z, inv, nullptr));
            }
        }
    }
    const int found = g.nlock;
    std::vector<int> perm(found);
    for (int i = 0; i < found; i++) perm[i] = i;
    std::sort(perm.begin(), perm.end(), [&](int p, int q) { return lam_c[p] < lam_c[q]; });
    for (int i = 0; i < found; i++) {
        lam[i] = lam_c[perm[i]];
        res[i] = res_c[perm[i]];
        if (Y) {
            cudaError_t e = cudaMemcpyAsync(Y + (int64_t)i * n, g.U + (int64_t)perm[i] * n, sizeof(double) * n,
                                            cudaMemcpyDefault, c->stream);
            if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanTr_gen eigenvector readback");
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "chebLanTr_gen outputs");
    *nev = found;
    if (stats) {
        *stats = evsl_stats();
        stats->niter = its;
        stats->nmv = nmv;
        stats->nrestart = nrestart;
        stats->t_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

// Lanczos quadrature density of the pencil (the density of S = B^{-1/2} A B^{-1/2}): for each of
// nvec unit vectors v_l (uniform(-1, 1), the standard density's stream and indexing, normalised),
// the pair w_1 = q(B) v_l, z_1 = B w_1 scaled to w_1^T z_1 = 1 starts m steps of Algorithm 3 on
// B^{-1} A (as drv_bounds_gen).  T_m = S diag(theta) S^T gives the Gauss quadrature of
// v_l^T f(S) v_l: nodes theta_j (ascending), weights S_{1j}^2.  A breakdown
// (beta <= 1e-13 ||A w_i|| / sqrt(bmax)) ends that vector's run.  Outputs as drv_landos.
int drv_landos_gen(evsl_ctx *c, int m, int nvec, uint64_t seed, double *nodes, double *weights, int *mused)
{
    EVSL_TRY(check_pencil(c, "landos_gen"));
    if (c->b_coef_isqrt.empty()) return ctx_fail(c, EVSL_ERR_STATE, "landos_gen: no B^{-1/2} polynomial");
    const int64_t n = c->A.n;
    const int mm = (int)std::min<int64_t>(m, n);
    double *W, *Z, *sc;
    EVSL_TRY(get_basis(c, mm, 0, &W, &Z, nullptr, &sc, mm + 1));
    Vecs v;
    EVSL_TRY(get_vecs(c, v));
    const double sqrt_bmax = std::sqrt(c->b_max);
    for (int l = 0; l < nvec; l++) {
        EVSL_TRY(fill_uniform_f64(c, n, seed, SM_STREAM_LANDOS, (uint64_t)l, v.x));
        EVSL_TRY(coldot(c, n, 1, v.x, n, v.x, n, sc + S_NB2));
        double nv2 = 0.0;
        EVSL_TRY(d2h(c, &nv2, sc + S_NB2, sizeof(double)));
        EVSL_TRY(scale_vec(c, n, v.x, 1.0 / std::sqrt(nv2), nullptr));
        EVSL_TRY(apply_poly_b(c, c->b_coef_isqrt, v.x, W, v.t1, v.t2));                       // w_1 = q(B) v
        EVSL_TRY(gen_step<2>(c, c->B, W, nullptr, nullptr, Z, nullptr, 0.0, 0.0, 0.0, 0.0));  // z_1 = B w_1
        EVSL_TRY(coldot(c, n, 1, W, n, Z, n, sc + S_NB2));
        double s2 = 0.0;
        EVSL_TRY(d2h(c, &s2, sc + S_NB2, sizeof(double)));
        if (!(s2 > 0.0)) return ctx_fail(c, EVSL_ERR_ARG, "landos_gen: (w, B w) = %g; B is not positive definite", s2);
        EVSL_TRY(scale_vec(c, n, W, 1.0 / std::sqrt(s2), nullptr));
        EVSL_TRY(scale_vec(c, n, Z, 1.0 / std::sqrt(s2), nullptr));
        std::vector<double> T((size_t)mm * mm, 0.0);
        double beta = 0.0;
        int k = 0;
        for (int j = 0; j < mm; j++) {
            EVSL_TRY(gen_step<2>(c, c->A, W + (int64_t)j * n, nullptr, nullptr, v.z, nullptr, 0.0, 0.0, 0.0, 0.0));
            EVSL_TRY(coldot(c, n, 1, v.z, n, v.z, n, sc + S_YN2));
            double alpha = 0.0, bn = 0.0, nz2 = 0.0;
            EVSL_TRY(lanab_step(c, j, W, Z, v.z, beta, v, sc, &alpha, &bn));
            EVSL_TRY(d2h(c, &nz2, sc + S_YN2, sizeof(double)));
            T[(size_t)j * mm + j] = alpha;
            k = j + 1;
            beta = bn;
            if (j + 1 == mm || beta <= 1e-13 * std::sqrt(std::max(0.0, nz2)) / sqrt_bmax) break;
            T[(size_t)(j + 1) * mm + j] = beta;
            T[(size_t)j * mm + j + 1] = beta;
        }
        std::vector<double> w;
        double *V = nullptr;
        int ldv = 0;
        EVSL_TRY(tri_eig(c, k, T, mm, w, &V, &ldv));
        std::vector<double> s0(k);
        cudaError_t e = cudaMemcpy2DAsync(s0.data(), sizeof(double), V, sizeof(double) * ldv, sizeof(double), k,
                                          cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "landos_gen first row");
        std::vector<int> order(k);
        for (int j = 0; j < k; j++) order[j] = j;
        std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] < w[y]; });
        for (int j = 0; j < m; j++) {
            nodes[(size_t)l * m + j] = j < k ? w[order[j]] : 0.0;
            weights[(size_t)l * m + j] = j < k ? s0[order[j]] * s0[order[j]] : 0.0;
        }
        mused[l] = k;
    }
    return EVSL_OK;
}
