/*
 * evsl_oracle.c -- plain, slow, FP64 CPU oracle for polynomial-filtered spectrum slicing
 * (Li, Xi, Erlandson, Saad, "The Eigenvalues Slicing Library (EVSL)", arXiv:1802.05215).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this code.  It shares nothing with the CUDA path: no headers, no helpers, no
 * tables.  Every loop is written in the order the paper states the method, without blocking,
 * fusion or reordering, so that it can be read against the paper.  Built with
 * -ffp-contract=off (no fused multiply-add).  The `omp parallel for` pragmas mark loops
 * without reductions (SpMV rows, elementwise updates, independent dot products); a build with
 * -fopenmp runs them on several host threads with bitwise the same results, for the
 * multi-core CPU baseline, and a build without it ignores them.
 *
 * Contents (paper passage in brackets):
 *   SplitMix64 counter-based draws  [seeded inputs; Steele-Lea-Flood 2014]
 *   CSR SpMV                         [Sec. 3.1, CSR storage]
 *   dense symmetric eigensolver      [Householder tridiagonalisation + implicit symmetric QR
 *                                     with Wilkinson shift, Golub & Van Loan Sec. 8.3]
 *   spectral bounds by Lanczos       [Sec. 2.2.1 text after Eq. (2.3); LanTrbounds Sec. 3.1]
 *   KPM moments (and per-probe sums), Jackson damping, cumulative DOS, slicer
 *                                    [Sec. 2.1, Eqs. (2.1)-(2.2)]
 *   Chebyshev filter build           [Sec. 2.2.1, Eqs. (2.3)-(2.6)]
 *   filter application               [Eq. (2.4) with the mapping of Eq. (2.3)]
 *   filtered thick-restart Lanczos with locking  [Sec. 2.3, Eqs. (2.10)-(2.11); Algorithm 2]
 *   non-restart filtered Lanczos (ChebLanNr)     [Sec. 2.3; Algorithm 2 without restarts]
 *   polynomial filtered subspace iteration        [Sec. 2.6]
 *   Lanczos quadrature density and its slicer     [Sec. 2.1]
 *   KPM moment doubling                           [Sec. 2.1; T_2k = 2 T_k^2 - T_0]
 *   generalized problems A x = lambda B x         [Sec. 2.4-2.5, Algorithm 3; lsPol of Sec. 4.3]:
 *     polynomial B^{-1} and B^{-1/2}, the pencil's bounds, KPM density, non-restart and
 *     thick-restart filtered Lanczos in the B-inner product
 *
 * Readings of passages that the paper leaves open are marked READING in the comments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* SplitMix64, used counter-based: draw(s,t,k) = (k+1)-th output of SplitMix64 seeded with
 * key(s,t) = first output of SplitMix64 seeded with s ^ (t * 0xD1B54A32D192ED03).         */
static uint64_t orc_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_next(uint64_t *state)
{
    *state += 0x9E3779B97F4A7C15ULL;
    return orc_mix(*state);
}

uint64_t orc_draw(uint64_t seed, uint64_t stream, uint64_t k)
{
    uint64_t s = seed ^ (stream * 0xD1B54A32D192ED03ULL);
    uint64_t key = orc_splitmix64_next(&s);
    uint64_t st = key + k * 0x9E3779B97F4A7C15ULL;
    return orc_splitmix64_next(&st);
}

static double orc_unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }
static double orc_sign(uint64_t x) { return (x >> 63) ? -1.0 : 1.0; }

enum { ORC_STREAM_ANDERSON = 1, ORC_STREAM_KPM = 2, ORC_STREAM_LANCZOS = 3, ORC_STREAM_BOUNDS = 4,
       ORC_STREAM_LANDOS = 5 };

/* ------------------------------------------------------------------------------------ */
/* Sparse matrix in CSR form (Sec. 3.1): y = A x.                                          */
typedef struct {
    int64_t n;
    const int64_t *rp;
    const int32_t *ci;
    const double *v;
} orc_csr;

static void orc_matvec(const orc_csr *A, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->n; i++) {
        double s = 0.0;
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++)
            s += A->v[p] * x[A->ci[p]];
        y[i] = s;
    }
}

void orc_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
              const double *x, double *y)
{
    orc_csr A = {n, rp, ci, v};
    orc_matvec(&A, x, y);
}

static double orc_dot(int64_t n, const double *x, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += x[i] * y[i];
    return s;
}

static double orc_nrm2(int64_t n, const double *x) { return sqrt(orc_dot(n, x, x)); }

/* Mapped operator of Eq. (2.3): y = (A x - c x) / d.                                      */
static void orc_mapped_matvec(const orc_csr *A, double c, double d, const double *x, double *y)
{
    orc_matvec(A, x, y);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->n; i++) y[i] = (y[i] - c * x[i]) / d;
}

/* ------------------------------------------------------------------------------------ */
/* Dense symmetric eigensolver (Golub & Van Loan, Matrix Computations, Sec. 8.3):
 * Householder tridiagonalisation (Alg. 8.3.1) with the orthogonal factor accumulated,
 * then the implicit symmetric QR algorithm with Wilkinson shift (Algs. 8.3.2-8.3.3),
 * every Givens rotation accumulated into the eigenvector matrix.
 * A: n x n column-major symmetric (read only).  w: eigenvalues ascending.  Z: n x n
 * column-major eigenvectors (may be NULL).  Returns 0, or -1 if QR did not converge.    */
#define AT(M, i, j, ld) (M)[(size_t)(j) * (ld) + (i)]

int orc_syev(int n, const double *Ain, double *w, double *Zout)
{
    if (n <= 0) return 0;
    double *A = malloc(sizeof(double) * n * n);
    double *Q = malloc(sizeof(double) * n * n);
    double *vv = malloc(sizeof(double) * n);
    double *pp = malloc(sizeof(double) * n);
    double *d = malloc(sizeof(double) * n);
    double *e = malloc(sizeof(double) * n);
    memcpy(A, Ain, sizeof(double) * n * n);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) AT(Q, i, j, n) = (i == j) ? 1.0 : 0.0;

    /* Householder tridiagonalisation: at step k reflect x = A[k+1:n, k] onto alpha e_1.  */
    for (int k = 0; k + 2 < n; k++) {
        int m = n - k - 1;
        double xn = 0.0;
        for (int i = 0; i < m; i++) xn += AT(A, k + 1 + i, k, n) * AT(A, k + 1 + i, k, n);
        xn = sqrt(xn);
        if (xn == 0.0) continue;
        double alpha = (AT(A, k + 1, k, n) > 0.0) ? -xn : xn;
        for (int i = 0; i < m; i++) vv[i] = AT(A, k + 1 + i, k, n);
        vv[0] -= alpha;
        double vn2 = 0.0;
        for (int i = 0; i < m; i++) vn2 += vv[i] * vv[i];
        if (vn2 == 0.0) continue;
        double beta = 2.0 / vn2;
        /* p = beta * A22 v ; w = p - (beta/2)(p.v) v ; A22 -= v w^T + w v^T              */
        for (int i = 0; i < m; i++) {
            double s = 0.0;
            for (int j = 0; j < m; j++) s += AT(A, k + 1 + i, k + 1 + j, n) * vv[j];
            pp[i] = beta * s;
        }
        double pv = 0.0;
        for (int i = 0; i < m; i++) pv += pp[i] * vv[i];
        double K = 0.5 * beta * pv;
        for (int i = 0; i < m; i++) pp[i] -= K * vv[i];
        for (int j = 0; j < m; j++)
            for (int i = 0; i < m; i++)
                AT(A, k + 1 + i, k + 1 + j, n) -= vv[i] * pp[j] + pp[i] * vv[j];
        AT(A, k + 1, k, n) = alpha;
        AT(A, k, k + 1, n) = alpha;
        for (int i = 1; i < m; i++) {
            AT(A, k + 1 + i, k, n) = 0.0;
            AT(A, k, k + 1 + i, n) = 0.0;
        }
        /* Q = Q (I - beta v v^T) on columns k+1..n-1                                      */
        for (int r = 0; r < n; r++) {
            double s = 0.0;
            for (int j = 0; j < m; j++) s += AT(Q, r, k + 1 + j, n) * vv[j];
            s *= beta;
            for (int j = 0; j < m; j++) AT(Q, r, k + 1 + j, n) -= s * vv[j];
        }
    }
    for (int i = 0; i < n; i++) d[i] = AT(A, i, i, n);
    for (int i = 0; i + 1 < n; i++) e[i] = AT(A, i + 1, i, n);
    e[n - 1] = 0.0;

    /* Implicit symmetric QR.  Rotation on (k,k+1): rows' = [c -s; s c] rows, and the same
     * on columns; the accumulated eigenvector matrix gets col_k' = c col_k - s col_{k+1},
     * col_{k+1}' = s col_k + c col_{k+1}.                                                 */
    const double eps = 2.220446049250313e-16;
    int status = 0;
    long iter = 0, maxiter = 60L * n + 100;
    int hi = n - 1;
    while (hi > 0) {
        if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            hi--;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) lo--;
        if (lo > 0) e[lo - 1] = 0.0;
        if (++iter > maxiter) { status = -1; break; }
        /* Wilkinson shift from the trailing 2x2 of the block                               */
        double del = 0.5 * (d[hi - 1] - d[hi]);
        double eb = e[hi - 1];
        double sg = (del >= 0.0) ? 1.0 : -1.0;
        double mu = d[hi] - eb * eb / (del + sg * sqrt(del * del + eb * eb));
        double x = d[lo] - mu, z = e[lo];
        double bulge = 0.0;
        for (int k = lo; k < hi; k++) {
            double r = sqrt(x * x + z * z);
            double c = (r == 0.0) ? 1.0 : x / r;
            double s = (r == 0.0) ? 0.0 : -z / r;
            if (k > lo) {
                /* rotate column k-1: [e[k-1]; bulge] -> [r; 0]                              */
                e[k - 1] = c * e[k - 1] - s * bulge;
            }
            double a = d[k], b = e[k], cc = d[k + 1];
            d[k] = c * c * a - 2.0 * c * s * b + s * s * cc;
            d[k + 1] = s * s * a + 2.0 * c * s * b + c * c * cc;
            e[k] = c * s * (a - cc) + (c * c - s * s) * b;
            if (k + 1 < hi) {
                bulge = -s * e[k + 1];
                e[k + 1] = c * e[k + 1];
                x = e[k];
                z = bulge;
            }
            for (int rr = 0; rr < n; rr++) {
                double qk = AT(Q, rr, k, n), qk1 = AT(Q, rr, k + 1, n);
                AT(Q, rr, k, n) = c * qk - s * qk1;
                AT(Q, rr, k + 1, n) = s * qk + c * qk1;
            }
        }
    }
    /* sort ascending (selection sort keeps it obvious)                                     */
    for (int i = 0; i < n; i++) {
        int best = i;
        for (int j = i + 1; j < n; j++)
            if (d[j] < d[best]) best = j;
        if (best != i) {
            double t = d[i]; d[i] = d[best]; d[best] = t;
            for (int rr = 0; rr < n; rr++) {
                double q = AT(Q, rr, i, n);
                AT(Q, rr, i, n) = AT(Q, rr, best, n);
                AT(Q, rr, best, n) = q;
            }
        }
    }
    for (int i = 0; i < n; i++) w[i] = d[i];
    if (Zout) memcpy(Zout, Q, sizeof(double) * n * n);
    free(A); free(Q); free(vv); free(pp); free(d); free(e);
    return status;
}

/* ------------------------------------------------------------------------------------ */
/* Full reorthogonalisation (Sec. 2.3): at most two passes of classical Gram-Schmidt
 * against the columns of the blocks, the second pass taken only when the DGKS test
 * ||z_after|| < eta ||z_before|| (eta = 1/sqrt(2)) says that the first one lost too much.
 * READING: eta = 1/sqrt(2), the classical Daniel-Gragg-Kaufman-Stewart choice.
 * Blocks are column-major n x ncol with leading dimension n.  Returns the number of passes. */
static int orc_reorth(int64_t n, double *z, const double *B1, int nc1, const double *B2, int nc2)
{
    double *h = malloc(sizeof(double) * (size_t)(nc1 + nc2 + 1));
    int passes = 0;
    for (int pass = 0; pass < 2; pass++) {
        double before = orc_nrm2(n, z);
#pragma omp parallel for schedule(dynamic, 4)
        for (int j = 0; j < nc1; j++) h[j] = orc_dot(n, B1 + (size_t)j * n, z);
#pragma omp parallel for schedule(dynamic, 4)
        for (int j = 0; j < nc2; j++) h[nc1 + j] = orc_dot(n, B2 + (size_t)j * n, z);
        for (int j = 0; j < nc1; j++) {
            const double *b = B1 + (size_t)j * n;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; i++) z[i] -= h[j] * b[i];
        }
        for (int j = 0; j < nc2; j++) {
            const double *b = B2 + (size_t)j * n;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; i++) z[i] -= h[nc1 + j] * b[i];
        }
        passes++;
        double after = orc_nrm2(n, z);
        if (after >= 0.7071067811865476 * before) break;
    }
    free(h);
    return passes;
}

/* Public form of one full reorthogonalisation of z against the ncol columns of B.           */
int orc_reorth_cgs(int64_t n, double *z, const double *B, int ncol)
{
    return orc_reorth(n, z, B, ncol, NULL, 0);
}

/* ------------------------------------------------------------------------------------ */
/* Spectral bounds (Sec. 2.2.1: "a few steps of the Lanczos algorithm"; LanTrbounds).
 * READING: `steps` Lanczos steps with full reorthogonalisation from the seeded start vector
 * (stream 4); the bounds are the extreme Ritz values widened by their residual bounds,
 * lmin = theta_1 - |beta_{m+1} s_{m,1}|, lmax = theta_m + |beta_{m+1} s_{m,m}|.            */
int orc_bounds(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
               int steps, uint64_t seed, double *lmin, double *lmax)
{
    orc_csr A = {n, rp, ci, v};
    if (steps > n) steps = (int)n;
    if (steps < 1) return -1;
    double *Q = calloc((size_t)n * (steps + 1), sizeof(double));
    double *T = calloc((size_t)steps * steps, sizeof(double));
    double *z = malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; i++)
        Q[i] = 2.0 * orc_unit(orc_draw(seed, ORC_STREAM_BOUNDS, (uint64_t)i)) - 1.0;
    double nq = orc_nrm2(n, Q);
    for (int64_t i = 0; i < n; i++) Q[i] /= nq;
    double beta = 0.0;
    int m = 0;
    for (int j = 0; j < steps; j++) {
        double *qj = Q + (size_t)j * n;
        orc_matvec(&A, qj, z);
        if (j > 0) {
            double *qp = Q + (size_t)(j - 1) * n;
            for (int64_t i = 0; i < n; i++) z[i] -= beta * qp[i];
        }
        double alpha = orc_dot(n, qj, z);
        for (int64_t i = 0; i < n; i++) z[i] -= alpha * qj[i];
        orc_reorth(n, z, Q, j + 1, NULL, 0);
        AT(T, j, j, steps) = alpha;
        beta = orc_nrm2(n, z);
        m = j + 1;
        if (j + 1 < steps) {
            AT(T, j, j + 1, steps) = beta;
            AT(T, j + 1, j, steps) = beta;
        }
        if (beta == 0.0) break;
        double *qn = Q + (size_t)(j + 1) * n;
        for (int64_t i = 0; i < n; i++) qn[i] = z[i] / beta;
    }
    double *Tm = malloc(sizeof(double) * m * m), *w = malloc(sizeof(double) * m),
           *S = malloc(sizeof(double) * m * m);
    for (int j = 0; j < m; j++)
        for (int i = 0; i < m; i++) AT(Tm, i, j, m) = AT(T, i, j, steps);
    int st = orc_syev(m, Tm, w, S);
    *lmin = w[0] - fabs(beta * AT(S, m - 1, 0, m));
    *lmax = w[m - 1] + fabs(beta * AT(S, m - 1, m - 1, m));
    free(Q); free(T); free(z); free(Tm); free(w); free(S);
    return st;
}

/* ------------------------------------------------------------------------------------ */
/* Kernel polynomial method (Sec. 2.1; the paper cites Lin, Saad and Yang for the formulas).
 * With Ahat = (A - cI)/d of Eq. (2.3) and nvec Rademacher probes v_l (stream 2, k = l*n+i):
 *   mu_k = (1/nvec) sum_l v_l^T T_k(Ahat) v_l ,  k = 0..M   (so mu_0 = n exactly),
 * by the three-term recurrence w_0 = v, w_1 = Ahat v, w_{k+1} = 2 Ahat w_k - w_{k-1}.      */
int orc_kpm_moments(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                    int M, int nvec, uint64_t seed, double lmin, double lmax, double *mu)
{
    orc_csr A = {n, rp, ci, v};
    double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    double *vl = malloc(sizeof(double) * n), *w0 = malloc(sizeof(double) * n),
           *w1 = malloc(sizeof(double) * n), *w2 = malloc(sizeof(double) * n);
    for (int k = 0; k <= M; k++) mu[k] = 0.0;
    for (int l = 0; l < nvec; l++) {
        for (int64_t i = 0; i < n; i++)
            vl[i] = orc_sign(orc_draw(seed, ORC_STREAM_KPM, (uint64_t)l * (uint64_t)n + (uint64_t)i));
        memcpy(w0, vl, sizeof(double) * n);
        mu[0] += orc_dot(n, vl, w0);
        if (M >= 1) {
            orc_mapped_matvec(&A, c, d, w0, w1);
            mu[1] += orc_dot(n, vl, w1);
        }
        for (int k = 1; k < M; k++) {
            orc_mapped_matvec(&A, c, d, w1, w2);
            for (int64_t i = 0; i < n; i++) w2[i] = 2.0 * w2[i] - w0[i];
            mu[k + 1] += orc_dot(n, vl, w2);
            double *t = w0; w0 = w1; w1 = w2; w2 = t;
        }
    }
    for (int k = 0; k <= M; k++) mu[k] /= nvec;
    free(vl); free(w0); free(w1); free(w2);
    return 0;
}

/* Per-probe KPM sums (Sec. 2.1, the terms of the estimator above before the average):
 *   out[l*(M+1) + k] = v_{first+l}^T T_k(Ahat) v_{first+l},  l = 0..nprobe-1, k = 0..M,
 * for the same Rademacher probes as orc_kpm_moments (probe index first+l draws its signs at
 * counter (first+l)*n + i).  Summing rows 0..nvec-1 in order and dividing by nvec reproduces
 * orc_kpm_moments exactly; a split of the probes over processes therefore only has to gather
 * these rows.                                                                              */
int orc_kpm_probe_moments(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                          int M, int64_t first, int nprobe, uint64_t seed, double lmin, double lmax,
                          double *out)
{
    orc_csr A = {n, rp, ci, v};
    double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    double *vl = malloc(sizeof(double) * n), *w0 = malloc(sizeof(double) * n),
           *w1 = malloc(sizeof(double) * n), *w2 = malloc(sizeof(double) * n);
    for (int l = 0; l < nprobe; l++) {
        double *o = out + (int64_t)l * (M + 1);
        const uint64_t probe = (uint64_t)(first + l);
        for (int64_t i = 0; i < n; i++)
            vl[i] = orc_sign(orc_draw(seed, ORC_STREAM_KPM, probe * (uint64_t)n + (uint64_t)i));
        memcpy(w0, vl, sizeof(double) * n);
        o[0] = orc_dot(n, vl, w0);
        if (M >= 1) {
            orc_mapped_matvec(&A, c, d, w0, w1);
            o[1] = orc_dot(n, vl, w1);
        }
        for (int k = 1; k < M; k++) {
            orc_mapped_matvec(&A, c, d, w1, w2);
            for (int64_t i = 0; i < n; i++) w2[i] = 2.0 * w2[i] - w0[i];
            o[k + 1] = orc_dot(n, vl, w2);
            double *t = w0; w0 = w1; w1 = w2; w2 = t;
        }
    }
    free(vl); free(w0); free(w1); free(w2);
    return 0;
}

/* Jackson damping factors for a degree-M expansion (standard KPM kernel, Weisse et al.,
 * Rev. Mod. Phys. 78 (2006)); READING: the variant with M+2 in the denominator.
 *   g_k = [(M-k+2) cos(k a) + sin(k a) cot(a)] / (M+2),  a = pi/(M+2),  k = 0..M.         */
void orc_jackson(int M, double *g)
{
    double a = M_PI / (M + 2);
    for (int k = 0; k <= M; k++)
        g[k] = ((M - k + 2) * cos(k * a) + sin(k * a) * (cos(a) / sin(a))) / (M + 2);
}

/* Cumulative DOS count on [lmin, t] from Jackson-damped moments (Eq. (2.1) integrated):
 * with th = arccos(that), that = (t-c)/d clamped to [-1,1],
 *   N(t) = (1/pi) [ g_0 mu_0 (pi - th) - 2 sum_{k>=1} g_k mu_k sin(k th)/k ].              */
double orc_dos_count(const double *mu, int M, double lmin, double lmax, double t)
{
    double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    double th = (t - c) / d;
    if (th < -1.0) th = -1.0;
    if (th > 1.0) th = 1.0;
    th = acos(th);
    double *g = malloc(sizeof(double) * (M + 1));
    orc_jackson(M, g);
    double s = g[0] * mu[0] * (M_PI - th);
    for (int k = 1; k <= M; k++) s -= 2.0 * g[k] * mu[k] * sin(k * th) / k;
    free(g);
    return s / M_PI;
}

/* Slicer of Eq. (2.2) (spslicer): npts evenly spaced x_j on [xi, eta]; C_j = N(x_j);
 * t_i = the first x_j with C_j - C_0 >= (i/ns)(C_{N-1} - C_0), refined by linear
 * interpolation between x_{j-1} and x_j.  READING: first crossing + linear interpolation.
 * est[i] = N(t_{i+1}) - N(t_i) from the same DOS.                                         */
int orc_slicer(const double *mu, int M, double lmin, double lmax, double xi, double eta,
               int ns, int npts, double *sli, double *est)
{
    if (ns < 1 || npts < 2 || !(eta > xi)) return -1;
    double *x = malloc(sizeof(double) * npts), *C = malloc(sizeof(double) * npts);
    for (int j = 0; j < npts; j++) {
        x[j] = xi + (eta - xi) * j / (npts - 1);
        C[j] = orc_dos_count(mu, M, lmin, lmax, x[j]);
    }
    double total = C[npts - 1] - C[0];
    sli[0] = xi;
    sli[ns] = eta;
    int j = 1;
    for (int i = 1; i < ns; i++) {
        double target = total * i / ns;
        while (j < npts - 1 && C[j] - C[0] < target) j++;
        double c0 = C[j - 1] - C[0], c1 = C[j] - C[0];
        double f = (c1 > c0) ? (target - c0) / (c1 - c0) : 1.0;
        if (f < 0.0) f = 0.0;
        if (f > 1.0) f = 1.0;
        sli[i] = x[j - 1] + f * (x[j] - x[j - 1]);
    }
    for (int i = 0; i < ns; i++)
        est[i] = orc_dos_count(mu, M, lmin, lmax, sli[i + 1]) - orc_dos_count(mu, M, lmin, lmax, sli[i]);
    free(x); free(C);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Chebyshev delta filter (Sec. 2.2.1).  rho(t) = sum_j g_j mu_j T_j(t) / sum_j g_j mu_j T_j(gamma)
 * with mu_0 = 1/2, mu_j = cos(j arccos gamma) (Eqs. (2.4)-(2.5)) and damping g_j (Eq. (2.6)).
 * T_j is evaluated from its definition cos(j arccos t) (cosh form outside [-1,1]).        */
enum { ORC_DAMP_NONE = 0, ORC_DAMP_JACKSON = 1, ORC_DAMP_SIGMA = 2 };

static double orc_chebT(int j, double t)
{
    if (t >= -1.0 && t <= 1.0) return cos(j * acos(t));
    double s = (t < 0.0 && (j & 1)) ? -1.0 : 1.0;
    return s * cosh(j * acosh(fabs(t)));
}

static void orc_damping(int type, int k, double *g)
{
    g[0] = 1.0;
    for (int j = 1; j <= k; j++) {
        if (type == ORC_DAMP_SIGMA) {              /* Lanczos sigma factors, Eq. (2.6)    */
            double th = M_PI / (k + 1);
            g[j] = sin(j * th) / (j * th);
        } else if (type == ORC_DAMP_JACKSON) {     /* Jackson factors for degree k        */
            double a = M_PI / (k + 2);
            g[j] = ((k - j + 2) * cos(j * a) + sin(j * a) * (cos(a) / sin(a))) / (k + 2);
        } else {
            g[j] = 1.0;
        }
    }
}

/* Unnormalised filter value P(t) = sum_j g_j mu_j(gamma) T_j(t), gamma = cos(th).         */
static double orc_P(int k, const double *g, double th, double t)
{
    double s = 0.5 * g[0];
    for (int j = 1; j <= k; j++) s += g[j] * cos(j * th) * orc_chebT(j, t);
    return s;
}

/* Balance equation of Eq. (2.7): rho(ta) - rho(tb) = 0 in the unknown gamma = cos(th).
 * READING: the garbled index in Eq. (2.7) is read as the two ends of the same interval.
 * Since both sides share the denominator, solve f(th) = P(ta) - P(tb) = 0 for th in
 * [acos(tb), acos(ta)] by Newton's method safeguarded with bisection.                     */
static double orc_balance(int k, const double *g, double ta, double tb)
{
    double lo = acos(tb), hi = acos(ta);    /* acos decreasing: lo < hi                    */
    double flo = orc_P(k, g, lo, ta) - orc_P(k, g, lo, tb);
    double fhi = orc_P(k, g, hi, ta) - orc_P(k, g, hi, tb);
    if (flo * fhi > 0.0) return 0.5 * (lo + hi);   /* no sign change: centre of interval  */
    double th = 0.5 * (lo + hi);
    for (int it = 0; it < 200; it++) {
        double f = 0.0, fp = 0.0;
        for (int j = 1; j <= k; j++) {
            double dT = orc_chebT(j, ta) - orc_chebT(j, tb);
            f += g[j] * cos(j * th) * dT;
            fp -= g[j] * j * sin(j * th) * dT;
        }
        if ((f < 0.0) == (flo < 0.0)) { lo = th; flo = f; } else { hi = th; }
        double nt = (fp != 0.0) ? th - f / fp : 0.5 * (lo + hi);
        if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
        double step = fabs(nt - th);
        th = nt;
        if (step < 1e-14) break;
    }
    return th;
}

/* Filter construction (find_pol, Sec. 2.2.1): for k = 2, 3, ... balance gamma, and stop at
 * the first k whose end value bar = rho(ta) = rho(tb) is <= tau (default 0.8).
 * Boundary slices (READING; the paper only says that a special, lower-degree filter is
 * used for them, Sec. 4.2): when ta <= -1 the filter is centred at gamma = -1 (the left end
 * of the spectrum) with the same damping, and k grows until rho(tb) <= tau_ext (default
 * 0.4); bar = rho(tb).  Mirrored (gamma = 1, rho(ta) <= tau_ext) when tb >= 1.  With Lanczos
 * sigma damping this reproduces the boundary-slice degrees 5, 6, 7, 8, 8, 9 of Table 4.
 * An interval covering the whole spectrum (ta <= -1 and tb >= 1), or lying outside it
 * (tb <= -1 or ta >= 1), is rejected.
 * Output coef[j] = g_j mu_j / P(gamma), j = 0..deg.  Returns 0, -1 on bad input, -2 if
 * maxdeg was reached, -5 if cap < deg+1 (deg then holds the needed degree).              */
int orc_filter_build(double a, double b, double lmin, double lmax, double tau, double tau_ext,
                     int damping, int maxdeg, int *deg, double *gamma, double *bar,
                     double *coef, int cap, int *boundary)
{
    if (!(b > a) || !(lmax > lmin) || maxdeg < 2) return -1;
    double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    double ta = (a - c) / d, tb = (b - c) / d;
    int left = (ta <= -1.0), right = (tb >= 1.0);
    if (left && right) return -1;
    if (tb <= -1.0 || ta >= 1.0) return -1;   /* slice outside the spectral interval */
    double *g = malloc(sizeof(double) * (maxdeg + 1));
    *boundary = left ? -1 : (right ? 1 : 0);
    int status = -2, k;
    double th = 0.0, bv = 0.0, Pg = 1.0;
    for (k = 2; k <= maxdeg; k++) {
        if (left || right) {
            orc_damping(damping, k, g);
            th = left ? M_PI : 0.0;
            Pg = orc_P(k, g, th, cos(th));
            bv = orc_P(k, g, th, left ? tb : ta) / Pg;
            if (bv <= tau_ext) { status = 0; break; }
        } else {
            orc_damping(damping, k, g);
            th = orc_balance(k, g, ta, tb);
            Pg = orc_P(k, g, th, cos(th));
            bv = orc_P(k, g, th, ta) / Pg;
            if (bv <= tau) { status = 0; break; }
        }
    }
    if (status != 0) k = maxdeg;
    *deg = k;
    *gamma = cos(th);
    *bar = bv;
    if (k + 1 > cap) { free(g); return status ? status : -5; }
    coef[0] = 0.5 * g[0] / Pg;
    for (int j = 1; j <= k; j++) coef[j] = g[j] * cos(j * th) / Pg;
    free(g);
    return status;
}

/* Filter application y = rho(Ahat) x = sum_j coef_j T_j(Ahat) x with the three-term
 * recurrence of the Chebyshev polynomials and Ahat of Eq. (2.3).                          */
static void orc_filter_apply_csr(const orc_csr *A, double c, double d, int deg,
                                 const double *coef, const double *x, double *y,
                                 double *w0, double *w1, double *w2)
{
    int64_t n = A->n;
    memcpy(w0, x, sizeof(double) * n);
    for (int64_t i = 0; i < n; i++) y[i] = coef[0] * w0[i];
    if (deg < 1) return;
    orc_mapped_matvec(A, c, d, w0, w1);
    for (int64_t i = 0; i < n; i++) y[i] += coef[1] * w1[i];
    for (int j = 1; j < deg; j++) {
        orc_mapped_matvec(A, c, d, w1, w2);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            w2[i] = 2.0 * w2[i] - w0[i];
            y[i] += coef[j + 1] * w2[i];
        }
        double *t = w0; w0 = w1; w1 = w2; w2 = t;
    }
}

void orc_filter_apply(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                      double lmin, double lmax, int deg, const double *coef, int nvec,
                      const double *X, double *Y)
{
    orc_csr A = {n, rp, ci, v};
    double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    double *w0 = malloc(sizeof(double) * n), *w1 = malloc(sizeof(double) * n),
           *w2 = malloc(sizeof(double) * n);
    for (int l = 0; l < nvec; l++)
        orc_filter_apply_csr(&A, c, d, deg, coef, X + (size_t)l * n, Y + (size_t)l * n, w0, w1, w2);
    free(w0); free(w1); free(w2);
}

/* ------------------------------------------------------------------------------------ */
/* Filtered thick-restart Lanczos with locking (Algorithm 2, Sec. 2.5) for A x = lambda x.
 *
 * Operator: (I - U U^T) rho(A) with rho the filter above; the deflation by the locked set U
 * is applied through the full reorthogonalisation against [U, Q] (U has orthonormal columns
 * orthogonal to Q, so the Rayleigh quotients q^T (I-UU^T) rho(A) q equal q^T rho(A) q).
 * Lanczos step (Eq. (2.10)): y = rho(A) q_i; z = y - beta_i q_{i-1}; alpha_i = q_i^T z;
 * z -= alpha_i q_i; full reorthogonalisation of z against [U, Q_i]; beta_{i+1} = ||z||.
 * Special TR step: with TR vectors u_1..u_l (Ritz values theta_j, couplings s_j) and
 * q_{l+1}: y = rho(A) q_{l+1}; alpha = q_{l+1}^T y; z = y - sum_j s_j u_j - alpha q_{l+1};
 * reorthogonalise; the projected matrix is the arrowhead diag(theta) bordered by s, followed
 * by the tridiagonal of the ordinary steps (thick restart of Wu and Simon).
 * Early-restart test every Ncycle steps: t = sum of the Ritz values >= bar; restart when it
 * changed by less than tau1 * max(1, |t|) since the previous test of the same cycle
 * (READING: and at least one Ritz value is >= bar, so that a cycle is never cut short
 * before anything has emerged above the threshold).
 * At restart every Ritz pair with theta >= bar is a candidate: u = Q s normalised,
 * lambda = u^T A u; pairs with lambda outside the slice are ignored; pairs with
 * ||A u - lambda u|| <= tol * ||A|| are locked; the others form the next TR set.
 *
 * READINGS (the paper leaves these open):
 *   - the candidate threshold is bar = rho(t_i) = rho(t_{i+1}) of the built filter (the
 *     paper writes tau, but eigenvalues just inside the slice map to [bar, tau) when bar<tau);
 *   - ||A|| = max(|lmin|, |lmax|);
 *   - slice membership is [a, b) when right_closed == 0 and [a, b] otherwise;
 *   - a restart that yields no candidate in the slice makes the next cycle start from a fresh
 *     seeded random vector orthogonalised against U (stream 3, index = restart count); the
 *     run stops after two consecutive restarts without candidates (the paper's "extra
 *     restart"), or when Its exceeds maxit;
 *   - a Lanczos breakdown (beta <= 1e-13 * ||y||) continues with a fresh seeded vector
 *     orthogonalised against [U, Q] and a zero coupling;
 *   - the TR set keeps at most m/2 vectors (those with the largest Ritz values), so that every
 *     cycle adds at least m/2 - 1 Lanczos steps and the basis never exceeds m+1 vectors;
 *   - a check at which no Ritz value is >= bar counts as stable only if the previous check of
 *     the cycle had none either and the cycle has taken max(2 Ncycle, m/4) steps (so a cycle
 *     that finds nothing ends early, but not before a missed eigenvalue could emerge);
 *   - stagnation: when two consecutive restarts lock nothing although candidates in the slice
 *     remain, the locked set and those candidates are refined together by a Rayleigh-Ritz
 *     projection with A (orc_refine), which separates Ritz vectors that mix nearly equal
 *     eigenvalues on both sides of a slice end; the next cycle then starts from a fresh vector
 *     as after a restart without candidates.  At most two refinements per call.
 * Y: n x cap column-major, lam/res: cap.  stats[0..3] = iterations, matvecs, restarts,
 * reorth passes.  Returns 0, -4 if maxit was exceeded, -5 if more than cap converged
 * (nev then holds the number found so far).                                               */
typedef struct {
    const orc_csr *A;
    double c, d;
    int deg;
    const double *coef;
    double *w0, *w1, *w2;
    long nmv;
} orc_filt;

static void orc_apply_filter(orc_filt *F, const double *x, double *y)
{
    orc_filter_apply_csr(F->A, F->c, F->d, F->deg, F->coef, x, y, F->w0, F->w1, F->w2);
    F->nmv += F->deg;
}

static void orc_fresh_vector(int64_t n, uint64_t seed, uint64_t index, double *q,
                             const double *U, int nlock, const double *Q, int nq)
{
    for (int64_t i = 0; i < n; i++)
        q[i] = 2.0 * orc_unit(orc_draw(seed, ORC_STREAM_LANCZOS, index * (uint64_t)n + (uint64_t)i)) - 1.0;
    orc_reorth(n, q, U, nlock, Q, nq);
    orc_reorth(n, q, U, nlock, Q, nq);
    double nr = orc_nrm2(n, q);
    for (int64_t i = 0; i < n; i++) q[i] /= nr;
}

/* Rayleigh-Ritz refinement with A (READING, see orc_cheblantr): W = [U(:, :nlock), C] has
 * orthonormal columns; G = W^T A W is eigendecomposed, G = Z diag(theta) Z^T, and the columns of
 * W Z whose theta lies in the slice and whose residual ||A w - theta w|| <= tol ||A|| become the
 * new locked set (in the order of Z's columns, i.e. ascending theta).  Returns the new count. */
static int orc_refine(const orc_csr *A, double a, double b, int right_closed, double normA,
                      double tol, double *U, int nlock, const double *C, int nc, int cap,
                      double *lam, double *res)
{
    int64_t n = A->n;
    int p = nlock + nc;
    double *W = malloc(sizeof(double) * (size_t)n * p), *AW = malloc(sizeof(double) * (size_t)n * p);
    double *G = malloc(sizeof(double) * (size_t)p * p), *th = malloc(sizeof(double) * p);
    double *Z = malloc(sizeof(double) * (size_t)p * p);
    double *w = malloc(sizeof(double) * n), *aw = malloc(sizeof(double) * n);
    memcpy(W, U, sizeof(double) * (size_t)n * nlock);
    memcpy(W + (size_t)n * nlock, C, sizeof(double) * (size_t)n * nc);
    for (int j = 0; j < p; j++) orc_matvec(A, W + (size_t)j * n, AW + (size_t)j * n);
    for (int j = 0; j < p; j++)
        for (int i = 0; i < p; i++) AT(G, i, j, p) = orc_dot(n, W + (size_t)i * n, AW + (size_t)j * n);
    for (int j = 0; j < p; j++)
        for (int i = 0; i < j; i++) {
            double s = 0.5 * (AT(G, i, j, p) + AT(G, j, i, p));
            AT(G, i, j, p) = s;
            AT(G, j, i, p) = s;
        }
    orc_syev(p, G, th, Z);
    int kept = 0;
    double *Unew = malloc(sizeof(double) * (size_t)n * (cap > 0 ? cap : 1));
    for (int j = 0; j < p; j++) {
        int inside = (th[j] >= a) && (right_closed ? (th[j] <= b) : (th[j] < b));
        if (!inside) continue;
        for (int64_t r = 0; r < n; r++) {
            double s1 = 0.0, s2 = 0.0;
            for (int q = 0; q < p; q++) {
                s1 += W[(size_t)q * n + r] * AT(Z, q, j, p);
                s2 += AW[(size_t)q * n + r] * AT(Z, q, j, p);
            }
            w[r] = s1;
            aw[r] = s2;
        }
        for (int64_t r = 0; r < n; r++) aw[r] -= th[j] * w[r];
        double rj = orc_nrm2(n, aw) / normA;
        if (rj <= tol && kept < cap) {
            memcpy(Unew + (size_t)kept * n, w, sizeof(double) * n);
            lam[kept] = th[j];
            res[kept] = rj;
            kept++;
        }
    }
    memcpy(U, Unew, sizeof(double) * (size_t)n * kept);
    free(W); free(AW); free(G); free(th); free(Z); free(w); free(aw); free(Unew);
    return kept;
}

int orc_cheblantr(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                  double a, double b, int right_closed, double lmin, double lmax,
                  int deg, const double *coef, double bar,
                  int m, int maxit, int ncycle, double tol, double tau1, uint64_t seed,
                  int cap, int *nev, double *lam, double *Y, double *res, long *stats)
{
    orc_csr A = {n, rp, ci, v};
    orc_filt F = {&A, 0.5 * (lmax + lmin), 0.5 * (lmax - lmin), deg, coef, NULL, NULL, NULL, 0};
    F.w0 = malloc(sizeof(double) * n);
    F.w1 = malloc(sizeof(double) * n);
    F.w2 = malloc(sizeof(double) * n);
    double normA = fmax(fabs(lmin), fabs(lmax));
    if (m > n) m = (int)n;
    double *U = calloc((size_t)n * (cap > 0 ? cap : 1), sizeof(double));
    double *Q = calloc((size_t)n * (m + 1), sizeof(double));
    double *T = calloc((size_t)(m + 1) * (m + 1), sizeof(double));
    double *y = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *u = malloc(sizeof(double) * n), *Au = malloc(sizeof(double) * n);
    double *theta = malloc(sizeof(double) * (m + 1)), *S = malloc(sizeof(double) * (m + 1) * (m + 1));
    double *Tk = malloc(sizeof(double) * (m + 1) * (m + 1));
    double *trv = malloc(sizeof(double) * (size_t)n * (m + 1));
    double *trtheta = malloc(sizeof(double) * (m + 1)), *trs = malloc(sizeof(double) * (m + 1));
    int nlock = 0, l = 0, its = 0, nrestart = 0, nocand = 0, status = 0, stall = 0, nrefine = 0;
    long npass = 0;
    uint64_t fresh_index = 0;

    orc_fresh_vector(n, seed, fresh_index++, Q, U, 0, NULL, 0);
    while (its <= maxit) {
        int k;                        /* number of basis vectors whose T-columns are complete */
        memset(T, 0, sizeof(double) * (m + 1) * (m + 1));
        if (l > 0) {
            /* special TR step on q_{l+1} = Q[:, l]                                           */
            for (int j = 0; j < l; j++) {
                AT(T, j, j, m + 1) = trtheta[j];
                AT(T, j, l, m + 1) = trs[j];
                AT(T, l, j, m + 1) = trs[j];
            }
            double *ql = Q + (size_t)l * n;
            orc_apply_filter(&F, ql, y);
            its++;
            double alpha = orc_dot(n, ql, y);
            for (int64_t i = 0; i < n; i++) z[i] = y[i];
            for (int j = 0; j < l; j++) {
                const double *uj = Q + (size_t)j * n;
                for (int64_t i = 0; i < n; i++) z[i] -= trs[j] * uj[i];
            }
            for (int64_t i = 0; i < n; i++) z[i] -= alpha * ql[i];
            npass += orc_reorth(n, z, U, nlock, Q, l + 1);
            AT(T, l, l, m + 1) = alpha;
            double beta = orc_nrm2(n, z);
            double *qn = Q + (size_t)(l + 1) * n;
            if (beta <= 1e-13 * orc_nrm2(n, y)) {
                orc_fresh_vector(n, seed, fresh_index++, qn, U, nlock, Q, l + 1);
                beta = 0.0;
            } else {
                for (int64_t i = 0; i < n; i++) qn[i] = z[i] / beta;
            }
            AT(T, l, l + 1, m + 1) = beta;
            AT(T, l + 1, l, m + 1) = beta;
            k = l + 1;
        } else {
            k = 0;
        }
        int lstart = k;
        double t_old = 0.0;
        int have_old = 0, prev_nabove = 0;
        for (int i = k; i < m; i++) {
            its++;
            double *qi = Q + (size_t)i * n;
            orc_apply_filter(&F, qi, y);
            for (int64_t r = 0; r < n; r++) z[r] = y[r];
            if (i > 0) {
                double bi = AT(T, i - 1, i, m + 1);
                const double *qp = Q + (size_t)(i - 1) * n;
                for (int64_t r = 0; r < n; r++) z[r] -= bi * qp[r];
            }
            double alpha = orc_dot(n, qi, z);
            for (int64_t r = 0; r < n; r++) z[r] -= alpha * qi[r];
            npass += orc_reorth(n, z, U, nlock, Q, i + 1);
            AT(T, i, i, m + 1) = alpha;
            double beta = orc_nrm2(n, z);
            double *qn = Q + (size_t)(i + 1) * n;
            if (beta <= 1e-13 * orc_nrm2(n, y)) {
                orc_fresh_vector(n, seed, fresh_index++, qn, U, nlock, Q, i + 1);
                beta = 0.0;
            } else {
                for (int64_t r = 0; r < n; r++) qn[r] = z[r] / beta;
            }
            AT(T, i, i + 1, m + 1) = beta;
            AT(T, i + 1, i, m + 1) = beta;
            k = i + 1;
            if ((k - lstart) % ncycle == 0) {
                for (int jj = 0; jj < k; jj++)
                    for (int ii = 0; ii < k; ii++) AT(Tk, ii, jj, k) = AT(T, ii, jj, m + 1);
                orc_syev(k, Tk, theta, NULL);
                double t_new = 0.0;
                int nabove = 0;
                for (int jj = 0; jj < k; jj++)
                    if (theta[jj] >= bar) { t_new += theta[jj]; nabove++; }
                if (have_old && nabove > 0 && fabs(t_new - t_old) < tau1 * fmax(1.0, fabs(t_new)))
                    break;
                int min_empty = (2 * ncycle > m / 4) ? 2 * ncycle : m / 4;
                if (have_old && nabove == 0 && prev_nabove == 0 && k - lstart >= min_empty) break;
                t_old = t_new;
                prev_nabove = nabove;
                have_old = 1;
            }
            if (its > maxit) break;
        }
        /* restart: Ritz pairs of T_k                                                         */
        nrestart++;
        for (int jj = 0; jj < k; jj++)
            for (int ii = 0; ii < k; ii++) AT(Tk, ii, jj, k) = AT(T, ii, jj, m + 1);
        orc_syev(k, Tk, theta, S);
        double betak = AT(T, k - 1, k, m + 1);
        int ncand = 0, ntr = 0, nlock_before = nlock;
        for (int jj = k - 1; jj >= 0; jj--) {          /* candidates, largest theta first     */
            if (theta[jj] < bar) break;
            const double *s = S + (size_t)jj * k;
            for (int64_t r = 0; r < n; r++) {
                double acc = 0.0;
                for (int p = 0; p < k; p++) acc += Q[(size_t)p * n + r] * s[p];
                u[r] = acc;
            }
            double nu = orc_nrm2(n, u);
            for (int64_t r = 0; r < n; r++) u[r] /= nu;
            orc_matvec(&A, u, Au);
            double lamj = orc_dot(n, u, Au);
            int inside = (lamj >= a) && (right_closed ? (lamj <= b) : (lamj < b));
            if (!inside) continue;
            ncand++;
            for (int64_t r = 0; r < n; r++) Au[r] -= lamj * u[r];
            double rj = orc_nrm2(n, Au) / normA;
            if (rj <= tol) {
                if (nlock >= cap) { status = -5; goto done; }
                memcpy(U + (size_t)nlock * n, u, sizeof(double) * n);
                lam[nlock] = lamj;
                res[nlock] = rj;
                nlock++;
            } else if (ntr < m / 2) {
                memcpy(trv + (size_t)ntr * n, u, sizeof(double) * n);
                trtheta[ntr] = theta[jj];
                trs[ntr] = betak * s[k - 1];
                ntr++;
            }
        }
        if (ncand == 0) nocand++; else nocand = 0;
        if (ncand > 0 && nlock == nlock_before) stall++; else stall = 0;
        int refined = 0;
        if (stall >= 2 && nrefine < 2 && ntr > 0 && nlock + ntr <= cap) {
            nlock = orc_refine(&A, a, b, right_closed, normA, tol, U, nlock, trv, ntr, cap, lam, res);
            nrefine++;
            stall = 0;
            nocand = 1;
            refined = 1;
        }
        if (nocand >= 2) break;
        if (its > maxit) { status = -4; break; }
        if (ncand == 0 || refined) {
            l = 0;
            orc_fresh_vector(n, seed, fresh_index++, Q, U, nlock, NULL, 0);
        } else {
            /* next cycle: TR vectors, then the residual direction q_{k+1}                      */
            memcpy(Q + (size_t)ntr * n, Q + (size_t)k * n, sizeof(double) * n);
            memcpy(Q, trv, sizeof(double) * (size_t)n * ntr);
            l = ntr;
            if (l == 0) {
                /* continue from q_{k+1}, re-orthogonalised against the new locked vectors */
                npass += orc_reorth(n, Q, U, nlock, NULL, 0);
                double nr = orc_nrm2(n, Q);
                for (int64_t r = 0; r < n; r++) Q[r] /= nr;
            }
        }
    }
done:
    /* sort the locked pairs by eigenvalue, ascending (selection sort)                      */
    for (int i = 0; i < nlock; i++) {
        int best = i;
        for (int j = i + 1; j < nlock; j++)
            if (lam[j] < lam[best]) best = j;
        if (best != i) {
            double t = lam[i]; lam[i] = lam[best]; lam[best] = t;
            t = res[i]; res[i] = res[best]; res[best] = t;
            for (int64_t r = 0; r < n; r++) {
                t = U[(size_t)i * n + r];
                U[(size_t)i * n + r] = U[(size_t)best * n + r];
                U[(size_t)best * n + r] = t;
            }
        }
    }
    if (Y) memcpy(Y, U, sizeof(double) * (size_t)n * nlock);
    *nev = nlock;
    if (stats) {
        stats[0] = its;
        stats[1] = F.nmv;
        stats[2] = nrestart;
        stats[3] = npass;
    }
    free(F.w0); free(F.w1); free(F.w2); free(U); free(Q); free(T); free(y); free(z);
    free(u); free(Au); free(theta); free(S); free(Tk); free(trv); free(trtheta); free(trs);
    return status;
}

/* Filtered non-restart Lanczos (ChebLanNr; the paper names a "simple non-restart Lanczos
 * algorithm", Sec. 2.3, and times it in Tables 2 and 4, but prints no listing).  READING:
 * Algorithm 2 without restarts and without locking.  One Krylov basis of rho(Ahat) is built
 * with full reorthogonalisation (CGS, DGKS second pass), up to m vectors, from the seeded start
 * vector.  Every Ncycle steps the sum t of the Ritz values >= bar is formed (the same test as
 * Algorithm 2's early restart).  When it is stable (|t - t_old| < tau1 max(1, |t|) with at least
 * one value >= bar) the candidate Ritz pairs (theta >= bar) are extracted: u = Q y normalised,
 * lambda = u^T A u, pairs outside the slice dropped.  If every remaining pair has
 * ||A u - lambda u|| <= tol ||A|| the run stops with them.  Otherwise the same basis is extended
 * and tested again (t_old is reset).  A test with no Ritz value >= bar after one without any,
 * once max(2 Ncycle, m/4) steps are done, ends the run with an empty result.  After m steps the
 * converged in-slice pairs are returned, with status -4 if some in-slice candidate did not
 * converge.  A breakdown (beta <= 1e-13 ||y||) continues with a fresh seeded vector orthogonal
 * to the basis and a zero coupling, as in orc_cheblantr.  stats: its, nmv, extractions, passes. */
int orc_cheblannr(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                  double a, double b, int right_closed, double lmin, double lmax,
                  int deg, const double *coef, double bar,
                  int m, int ncycle, double tol, double tau1, uint64_t seed,
                  int cap, int *nev, double *lam, double *Y, double *res, long *stats)
{
    orc_csr A = {n, rp, ci, v};
    orc_filt F = {&A, 0.5 * (lmax + lmin), 0.5 * (lmax - lmin), deg, coef, NULL, NULL, NULL, 0};
    F.w0 = malloc(sizeof(double) * n);
    F.w1 = malloc(sizeof(double) * n);
    F.w2 = malloc(sizeof(double) * n);
    double normA = fmax(fabs(lmin), fabs(lmax));
    if (m > n) m = (int)n;
    double *Q = calloc((size_t)n * (m + 1), sizeof(double));
    double *T = calloc((size_t)(m + 1) * (m + 1), sizeof(double));
    double *Tk = malloc(sizeof(double) * (size_t)(m + 1) * (m + 1));
    double *S = malloc(sizeof(double) * (size_t)(m + 1) * (m + 1));
    double *theta = malloc(sizeof(double) * (m + 1));
    double *y = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *u = malloc(sizeof(double) * n), *Au = malloc(sizeof(double) * n);
    int its = 0, status = 0, found = 0, extractions = 0, done = 0;
    long npass = 0;
    uint64_t fresh_index = 0;
    double t_old = 0.0;
    int have_old = 0, prev_nabove = 0;

    orc_fresh_vector(n, seed, fresh_index++, Q, NULL, 0, NULL, 0);
    for (int i = 0; i < m && !done; i++) {
        its++;
        double *qi = Q + (size_t)i * n;
        orc_apply_filter(&F, qi, y);
        for (int64_t r = 0; r < n; r++) z[r] = y[r];
        if (i > 0) {
            double bi = AT(T, i - 1, i, m + 1);
            const double *qp = Q + (size_t)(i - 1) * n;
            for (int64_t r = 0; r < n; r++) z[r] -= bi * qp[r];
        }
        double alpha = orc_dot(n, qi, z);
        for (int64_t r = 0; r < n; r++) z[r] -= alpha * qi[r];
        npass += orc_reorth(n, z, NULL, 0, Q, i + 1);
        AT(T, i, i, m + 1) = alpha;
        double beta = orc_nrm2(n, z);
        double *qn = Q + (size_t)(i + 1) * n;
        if (beta <= 1e-13 * orc_nrm2(n, y)) {
            orc_fresh_vector(n, seed, fresh_index++, qn, NULL, 0, Q, i + 1);
            beta = 0.0;
        } else {
            for (int64_t r = 0; r < n; r++) qn[r] = z[r] / beta;
        }
        AT(T, i, i + 1, m + 1) = beta;
        AT(T, i + 1, i, m + 1) = beta;
        int k = i + 1;
        int extract = (k == m);
        if (k % ncycle == 0 && k < m) {
            for (int jj = 0; jj < k; jj++)
                for (int ii = 0; ii < k; ii++) AT(Tk, ii, jj, k) = AT(T, ii, jj, m + 1);
            orc_syev(k, Tk, theta, NULL);
            double t_new = 0.0;
            int nabove = 0;
            for (int jj = 0; jj < k; jj++)
                if (theta[jj] >= bar) { t_new += theta[jj]; nabove++; }
            int min_empty = (2 * ncycle > m / 4) ? 2 * ncycle : m / 4;
            if (have_old && nabove == 0 && prev_nabove == 0 && k >= min_empty) {
                done = 1;                                    /* empty slice */
                break;
            }
            if (have_old && nabove > 0 && fabs(t_new - t_old) < tau1 * fmax(1.0, fabs(t_new))) extract = 1;
            t_old = t_new;
            prev_nabove = nabove;
            have_old = 1;
        }
        if (!extract) continue;
        /* candidate Ritz pairs of T_k, largest theta first */
        extractions++;
        for (int jj = 0; jj < k; jj++)
            for (int ii = 0; ii < k; ii++) AT(Tk, ii, jj, k) = AT(T, ii, jj, m + 1);
        orc_syev(k, Tk, theta, S);
        int nconv = 0, nunconv = 0;
        for (int jj = k - 1; jj >= 0; jj--) {
            if (theta[jj] < bar) break;
            const double *s = S + (size_t)jj * k;
            for (int64_t r = 0; r < n; r++) {
                double acc = 0.0;
                for (int p = 0; p < k; p++) acc += Q[(size_t)p * n + r] * s[p];
                u[r] = acc;
            }
            double nu = orc_nrm2(n, u);
            for (int64_t r = 0; r < n; r++) u[r] /= nu;
            orc_matvec(&A, u, Au);
            double lamj = orc_dot(n, u, Au);
            int inside = (lamj >= a) && (right_closed ? (lamj <= b) : (lamj < b));
            if (!inside) continue;
            for (int64_t r = 0; r < n; r++) Au[r] -= lamj * u[r];
            double rj = orc_nrm2(n, Au) / normA;
            if (rj > tol) { nunconv++; continue; }
            if (nconv >= cap) { status = -5; break; }
            if (Y) memcpy(Y + (size_t)nconv * n, u, sizeof(double) * n);
            lam[nconv] = lamj;
            res[nconv] = rj;
            nconv++;
        }
        found = nconv;
        if (status == -5) break;
        if (nunconv == 0 || k == m) {
            if (nunconv > 0) status = -4;
            done = 1;
            break;
        }
        have_old = 0;                                        /* extend the same basis */
    }
    /* sort ascending (selection sort), eigenvectors along */
    for (int i = 0; i < found; i++) {
        int best = i;
        for (int j = i + 1; j < found; j++)
            if (lam[j] < lam[best]) best = j;
        if (best != i) {
            double t = lam[i]; lam[i] = lam[best]; lam[best] = t;
            t = res[i]; res[i] = res[best]; res[best] = t;
            if (Y)
                for (int64_t r = 0; r < n; r++) {
                    t = Y[(size_t)i * n + r];
                    Y[(size_t)i * n + r] = Y[(size_t)best * n + r];
                    Y[(size_t)best * n + r] = t;
                }
        }
    }
    *nev = found;
    if (stats) {
        stats[0] = its;
        stats[1] = F.nmv;
        stats[2] = extractions;
        stats[3] = npass;
    }
    free(F.w0); free(F.w1); free(F.w2); free(Q); free(T); free(Tk); free(S); free(theta);
    free(y); free(z); free(u); free(Au);
    return status;
}

/* Polynomial filtered subspace iteration (ChebSI; the paper lists it among EVSL's projection
 * methods, Sec. 2.6 and Sec. 3, and notes that the subspace dimension comes from the DOS count,
 * but prints no listing).  READING: V (n x nv) starts as nv seeded random vectors (stream 3,
 * indices 0..nv-1), orthonormalised.  Each pass forms W = rho(Ahat) V; when V holds the Ritz
 * vectors of the previous pass, mu_j = v_j^T w_j is the filter's Rayleigh quotient of v_j.  A
 * vector made only of eigenvectors outside the slice has mu < bar (rho < bar outside the slice),
 * an eigenvector inside has mu >= bar, so the in-slice Ritz pairs with mu >= bar are the wanted
 * ones: when all of them have ||A v - theta v|| <= tol ||A||, the run stops and returns the
 * converged in-slice pairs.  Otherwise W is orthonormalised (CGS with the DGKS second pass,
 * column by column; a column that vanishes is replaced by the next seeded vector) and
 * Rayleigh-Ritz with A gives the next V = W S (W^T A W = S diag(theta) S^T, theta ascending).
 * After maxit passes the converged in-slice pairs are returned with status -4.
 * stats: passes, nmv, 0, CGS passes. */
int orc_chebsi(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
               double a, double b, int right_closed, double lmin, double lmax,
               int deg, const double *coef, double bar, int nv, int maxit, double tol, uint64_t seed,
               int cap, int *nev, double *lam, double *Y, double *res, long *stats)
{
    orc_csr A = {n, rp, ci, v};
    orc_filt F = {&A, 0.5 * (lmax + lmin), 0.5 * (lmax - lmin), deg, coef, NULL, NULL, NULL, 0};
    F.w0 = malloc(sizeof(double) * n);
    F.w1 = malloc(sizeof(double) * n);
    F.w2 = malloc(sizeof(double) * n);
    double normA = fmax(fabs(lmin), fabs(lmax));
    if (nv > n) nv = (int)n;
    double *V = malloc(sizeof(double) * (size_t)n * nv), *W = malloc(sizeof(double) * (size_t)n * nv);
    double *AW = malloc(sizeof(double) * (size_t)n * nv);
    double *G = malloc(sizeof(double) * (size_t)nv * nv), *S = malloc(sizeof(double) * (size_t)nv * nv);
    double *th = malloc(sizeof(double) * nv), *rr = malloc(sizeof(double) * nv), *r = malloc(sizeof(double) * n);
    uint64_t fresh_index = 0;
    long npass = 0;
    int it = 0, status = -4, found = 0, ritz = 0;
    for (int j = 0; j < nv; j++)
        orc_fresh_vector(n, seed, fresh_index++, V + (size_t)j * n, NULL, 0, V, j);
    for (it = 1; it <= maxit + 1; it++) {
        for (int j = 0; j < nv; j++) orc_apply_filter(&F, V + (size_t)j * n, W + (size_t)j * n);
        if (ritz) {
            /* the previous pass's Ritz pairs: stop if every wanted one has converged */
            int all = 1;
            for (int j = 0; j < nv; j++) {
                int inside = (th[j] >= a) && (right_closed ? (th[j] <= b) : (th[j] < b));
                double mu = orc_dot(n, V + (size_t)j * n, W + (size_t)j * n);
                if (inside && mu >= bar && rr[j] > tol) all = 0;
            }
            if (all || it == maxit + 1) {
                found = 0;
                status = all ? 0 : -4;
                for (int j = 0; j < nv; j++) {
                    int inside = (th[j] >= a) && (right_closed ? (th[j] <= b) : (th[j] < b));
                    if (!inside || rr[j] > tol) continue;
                    if (found >= cap) { status = -5; break; }
                    lam[found] = th[j];
                    res[found] = rr[j];
                    if (Y) memcpy(Y + (size_t)found * n, V + (size_t)j * n, sizeof(double) * n);
                    found++;
                }
                it--;                   /* this filter pass only served the test */
                break;
            }
        }
        for (int j = 0; j < nv; j++) {
            double *w = W + (size_t)j * n;
            double before = orc_nrm2(n, w);
            npass += orc_reorth(n, w, W, j, NULL, 0);
            double nw = orc_nrm2(n, w);
            if (!(nw > 1e-12 * before)) {                    /* dependent: a fresh direction */
                orc_fresh_vector(n, seed, fresh_index++, w, W, j, NULL, 0);
                continue;
            }
            for (int64_t i = 0; i < n; i++) w[i] /= nw;
        }
        for (int j = 0; j < nv; j++) orc_matvec(&A, W + (size_t)j * n, AW + (size_t)j * n);
        for (int j = 0; j < nv; j++)
            for (int i = 0; i <= j; i++) {
                double g = 0.5 * (orc_dot(n, W + (size_t)i * n, AW + (size_t)j * n) +
                                  orc_dot(n, W + (size_t)j * n, AW + (size_t)i * n));
                AT(G, i, j, nv) = g;
                AT(G, j, i, nv) = g;
            }
        orc_syev(nv, G, th, S);
        for (int64_t i = 0; i < n; i++)
            for (int j = 0; j < nv; j++) {
                double acc = 0.0;
                for (int p = 0; p < nv; p++) acc += W[(size_t)p * n + i] * AT(S, p, j, nv);
                V[(size_t)j * n + i] = acc;
            }
        for (int j = 0; j < nv; j++) {
            const double *vj = V + (size_t)j * n;
            orc_matvec(&A, vj, r);
            for (int64_t i = 0; i < n; i++) r[i] -= th[j] * vj[i];
            rr[j] = orc_nrm2(n, r) / normA;
        }
        ritz = 1;
    }
    *nev = found;
    if (stats) {
        stats[0] = it;
        stats[1] = F.nmv;
        stats[2] = 0;
        stats[3] = npass;
    }
    free(F.w0); free(F.w1); free(F.w2); free(V); free(W); free(AW); free(G); free(S); free(th);
    free(rr); free(r);
    return status;
}

/* Lanczos spectral density (landos; Sec. 2.1 names the Lanczos / Gaussian-quadrature DOS of
 * Lin, Saad and Yang as the second DOS method, with no formulas).  READING: for each of nvec unit
 * vectors v_l (uniform(-1, 1) entries from stream 5, index l n + i, normalised) an m-step Lanczos
 * run on A with full reorthogonalisation (CGS, DGKS second pass) gives T = S diag(theta) S^T;
 * the Gaussian quadrature of v_l^T f(A) v_l has nodes theta_j and weights tau_j = S_{1j}^2.  The
 * density is (n / nvec) sum_l sum_j tau_lj delta(t - theta_lj).  A breakdown (beta <= 1e-13 ||Av||)
 * ends the run of that vector (mused[l] < m: the quadrature is then exact for v_l).
 * Outputs (nvec x m, row l = vector l): nodes, weights, mused. */
int orc_landos(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int m, int nvec,
               uint64_t seed, double *nodes, double *weights, int *mused)
{
    orc_csr A = {n, rp, ci, v};
    if (m > n) m = (int)n;
    double *Q = calloc((size_t)n * (m + 1), sizeof(double));
    double *T = calloc((size_t)m * m, sizeof(double)), *S = malloc(sizeof(double) * (size_t)m * m);
    double *th = malloc(sizeof(double) * m), *z = malloc(sizeof(double) * n);
    for (int l = 0; l < nvec; l++) {
        double *q0 = Q;
        for (int64_t i = 0; i < n; i++)
            q0[i] = 2.0 * orc_unit(orc_draw(seed, ORC_STREAM_LANDOS, (uint64_t)l * (uint64_t)n + (uint64_t)i)) - 1.0;
        double nq = orc_nrm2(n, q0);
        for (int64_t i = 0; i < n; i++) q0[i] /= nq;
        memset(T, 0, sizeof(double) * (size_t)m * m);
        int k = 0;
        double beta = 0.0;
        for (int j = 0; j < m; j++) {
            double *qj = Q + (size_t)j * n;
            orc_matvec(&A, qj, z);
            double nz = orc_nrm2(n, z);
            if (j > 0)
                for (int64_t i = 0; i < n; i++) z[i] -= beta * Q[(size_t)(j - 1) * n + i];
            double alpha = orc_dot(n, qj, z);
            for (int64_t i = 0; i < n; i++) z[i] -= alpha * qj[i];
            orc_reorth(n, z, NULL, 0, Q, j + 1);
            AT(T, j, j, m) = alpha;
            k = j + 1;
            beta = orc_nrm2(n, z);
            if (j + 1 == m || beta <= 1e-13 * nz) break;
            AT(T, j, j + 1, m) = beta;
            AT(T, j + 1, j, m) = beta;
            for (int64_t i = 0; i < n; i++) Q[(size_t)(j + 1) * n + i] = z[i] / beta;
        }
        double *Tk = malloc(sizeof(double) * (size_t)k * k), *Sk = malloc(sizeof(double) * (size_t)k * k);
        for (int c = 0; c < k; c++)
            for (int r = 0; r < k; r++) AT(Tk, r, c, k) = AT(T, r, c, m);
        orc_syev(k, Tk, th, Sk);
        for (int j = 0; j < m; j++) {
            nodes[(size_t)l * m + j] = j < k ? th[j] : 0.0;
            weights[(size_t)l * m + j] = j < k ? AT(Sk, 0, j, k) * AT(Sk, 0, j, k) : 0.0;
        }
        mused[l] = k;
        free(Tk);
        free(Sk);
    }
    free(Q); free(T); free(S); free(th); free(z);
    return 0;
}

/* Slicer on the Lanczos density (spslicer2; the paper names it with no definition).  READING: the
 * cumulative count N(t) = (n / nvec) sum of the weights of the nodes <= t is a step function.
 * With C0 = N just below xi and C1 = N(eta), boundary t_i (0 < i < ns) is placed midway between
 * the first node in [xi, eta] at which N reaches C0 + (i / ns)(C1 - C0) and the node before it
 * (xi if there is none); t_0 = xi, t_ns = eta; est[i] = N(t_{i+1}) - N(t_i) (with N just below
 * xi for i = 0).  Returns 0, or -1 if no node lies in [xi, eta]. */
int orc_slicer_landos(const double *nodes, const double *weights, const int *mused, int m, int nvec,
                      int64_t n, double xi, double eta, int ns, double *sli, double *est)
{
    int tot = 0;
    for (int l = 0; l < nvec; l++) tot += mused[l];
    double *t = malloc(sizeof(double) * (tot > 0 ? tot : 1)), *w = malloc(sizeof(double) * (tot > 0 ? tot : 1));
    int q = 0;
    for (int l = 0; l < nvec; l++)
        for (int j = 0; j < mused[l]; j++) {
            t[q] = nodes[(size_t)l * m + j];
            w[q] = weights[(size_t)l * m + j] * (double)n / (double)nvec;
            q++;
        }
    /* insertion sort by node (stable) */
    for (int i = 1; i < tot; i++) {
        double ti = t[i], wi = w[i];
        int j = i - 1;
        while (j >= 0 && t[j] > ti) { t[j + 1] = t[j]; w[j + 1] = w[j]; j--; }
        t[j + 1] = ti;
        w[j + 1] = wi;
    }
    double c0 = 0.0, c1 = 0.0;
    int first = -1, last = -1;
    for (int i = 0; i < tot; i++) {
        if (t[i] < xi) c0 += w[i];
        if (t[i] <= eta) c1 += w[i];
        if (t[i] >= xi && t[i] <= eta) { if (first < 0) first = i; last = i; }
    }
    if (first < 0) { free(t); free(w); return -1; }
    sli[0] = xi;
    sli[ns] = eta;
    double cum = c0;
    int p = first;
    for (int s = 1; s < ns; s++) {
        double target = c0 + (double)s / ns * (c1 - c0);
        while (p <= last && cum + w[p] < target) { cum += w[p]; p++; }
        if (p > last) p = last;
        double prev = (p > first) ? t[p - 1] : xi;
        sli[s] = 0.5 * (prev + t[p]);
    }
    for (int s = 0; s < ns; s++) {
        double lo = 0.0, hi = 0.0;
        for (int i = 0; i < tot; i++) {
            if (t[i] < sli[s]) lo += w[i];
            if (s + 1 == ns ? t[i] <= sli[s + 1] : t[i] < sli[s + 1]) hi += w[i];
        }
        est[s] = hi - lo;
    }
    free(t);
    free(w);
    return 0;
}

/* KPM moments with the doubling identities (the moment-doubling variant of the KPM density,
 * listed beside kpmdos; Chebyshev identities T_{2k} = 2 T_k^2 - T_0 and
 * T_{2k+1} = 2 T_{k+1} T_k - T_1): with w_k = T_k(Ahat) v_l,
 *   mu_{2k} = (1/nvec) sum_l (2 w_k^T w_k - v_l^T v_l),
 *   mu_{2k+1} = (1/nvec) sum_l (2 w_{k+1}^T w_k - v_l^T w_1),
 * so moments up to M need only ceil(M/2) recurrence steps.  Same probes as orc_kpm_moments. */
int orc_kpm_moments_doubling(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                             int M, int nvec, uint64_t seed, double lmin, double lmax, double *mu)
{
    orc_csr A = {n, rp, ci, v};
    double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    double *w0 = malloc(sizeof(double) * n), *w1 = malloc(sizeof(double) * n), *w2 = malloc(sizeof(double) * n);
    for (int k = 0; k <= M; k++) mu[k] = 0.0;
    const int K = (M + 1) / 2;   /* w_0 .. w_K are formed; 2K >= M */
    for (int l = 0; l < nvec; l++) {
        for (int64_t i = 0; i < n; i++)
            w0[i] = orc_sign(orc_draw(seed, ORC_STREAM_KPM, (uint64_t)l * (uint64_t)n + (uint64_t)i));
        const double m0 = orc_dot(n, w0, w0);
        mu[0] += m0;
        if (M == 0) continue;
        orc_mapped_matvec(&A, c, d, w0, w1);
        const double m1 = orc_dot(n, w0, w1);
        mu[1] += m1;
        /* k = 1: mu_2 = 2 w1.w1 - m0, mu_3 = 2 w2.w1 - m1, ... */
        for (int k = 1; k <= K; k++) {
            if (2 * k <= M) mu[2 * k] += 2.0 * orc_dot(n, w1, w1) - m0;
            if (2 * k + 1 > M) break;
            orc_mapped_matvec(&A, c, d, w1, w2);
            for (int64_t i = 0; i < n; i++) w2[i] = 2.0 * w2[i] - w0[i];
            mu[2 * k + 1] += 2.0 * orc_dot(n, w2, w1) - m1;
            double *t = w0; w0 = w1; w1 = w2; w2 = t;
        }
    }
    for (int k = 0; k <= M; k++) mu[k] /= nvec;
    free(w0); free(w1); free(w2);
    return 0;
}

/* ---- Generalized problems A x = lambda B x with B SPD (Sec. 2.4) and the polynomial B^{-1}
 * of Sec. 4.3 (lsPol: "Chebyshev polynomial expansion" for the solves with a well-conditioned
 * mass matrix B).  READING: p(t) ~ 1/t on [bmin, bmax] is the Chebyshev interpolant at the
 * Chebyshev-Gauss points of degree k, k the smallest degree (up to maxdeg) whose relative error
 * max |t p(t) - 1| on 2001 equispaced points is <= eps. */
int orc_lspol(double bmin, double bmax, double eps, int maxdeg, int *deg, double *coef)
{
    const double c = 0.5 * (bmax + bmin), h = 0.5 * (bmax - bmin);
    for (int k = 1; k <= maxdeg; k++) {
        const int N = k + 1;
        for (int j = 0; j <= k; j++) {
            double s = 0.0;
            for (int q = 0; q < N; q++) {
                const double th = M_PI * (q + 0.5) / N;
                s += cos(j * th) / (c + h * cos(th));
            }
            coef[j] = (j == 0 ? 1.0 : 2.0) * s / N;
        }
        double err = 0.0;
        for (int q = 0; q <= 2000; q++) {
            const double t = bmin + (bmax - bmin) * q / 2000.0, u = (t - c) / h;
            double p = 0.0;
            for (int j = 0; j <= k; j++) p += coef[j] * orc_chebT(j, u);
            err = fmax(err, fabs(t * p - 1.0));
        }
        if (err <= eps) { *deg = k; return 0; }
    }
    *deg = maxdeg;
    return -4;
}

/* lsPol for B^{-1/2} (Sec. 2.1: the DOS of a pencil needs starting vectors built with B^{1/2}
 * or the Cholesky factor; for a well-conditioned mass matrix a polynomial replaces the
 * factorisation).  READING: as orc_lspol with f(t) = t^{-1/2}: the Chebyshev interpolant at the
 * Chebyshev-Gauss points, of the smallest degree k (up to maxdeg) whose relative error
 * max |sqrt(t) p(t) - 1| on 2001 equispaced points is <= eps. */
int orc_lspol_isqrt(double bmin, double bmax, double eps, int maxdeg, int *deg, double *coef)
{
    const double c = 0.5 * (bmax + bmin), h = 0.5 * (bmax - bmin);
    for (int k = 1; k <= maxdeg; k++) {
        const int N = k + 1;
        for (int j = 0; j <= k; j++) {
            double s = 0.0;
            for (int q = 0; q < N; q++) {
                const double th = M_PI * (q + 0.5) / N;
                s += cos(j * th) / sqrt(c + h * cos(th));
            }
            coef[j] = (j == 0 ? 1.0 : 2.0) * s / N;
        }
        double err = 0.0;
        for (int q = 0; q <= 2000; q++) {
            const double t = bmin + (bmax - bmin) * q / 2000.0, u = (t - c) / h;
            double p = 0.0;
            for (int j = 0; j <= k; j++) p += coef[j] * orc_chebT(j, u);
            err = fmax(err, fabs(sqrt(t) * p - 1.0));
        }
        if (err <= eps) { *deg = k; return 0; }
    }
    *deg = maxdeg;
    return -4;
}

/* y = p(B) x with the Chebyshev recurrence on Bhat = (B - c I) / h */
static void orc_polyB(const orc_csr *B, double c, double h, int deg, const double *coef,
                      const double *x, double *y, double *w0, double *w1, double *w2)
{
    int64_t n = B->n;
    memcpy(w0, x, sizeof(double) * n);
    for (int64_t i = 0; i < n; i++) y[i] = coef[0] * x[i];
    if (deg == 0) return;
    orc_mapped_matvec(B, c, h, w0, w1);
    for (int64_t i = 0; i < n; i++) y[i] += coef[1] * w1[i];
    for (int j = 2; j <= deg; j++) {
        orc_mapped_matvec(B, c, h, w1, w2);
        for (int64_t i = 0; i < n; i++) w2[i] = 2.0 * w2[i] - w0[i];
        for (int64_t i = 0; i < n; i++) y[i] += coef[j] * w2[i];
        double *t = w0; w0 = w1; w1 = w2; w2 = t;
    }
}

/* Public form: y = p(B) x (the approximate solve of Sec. 4.3). */
void orc_polyB_apply(int64_t n, const int64_t *brp, const int32_t *bci, const double *bv, double bmin,
                     double bmax, int deg, const double *coef, const double *x, double *y)
{
    orc_csr B = {n, brp, bci, bv};
    double *w = malloc(sizeof(double) * 3 * n);
    orc_polyB(&B, 0.5 * (bmax + bmin), 0.5 * (bmax - bmin), deg, coef, x, y, w, w + n, w + 2 * n);
    free(w);
}

typedef struct {
    const orc_csr *A, *B;
    double bc, bh;        /* mapping of B for the polynomial inverse */
    int bdeg;
    const double *bcoef;
    double *t0, *t1, *t2; /* scratch of the polynomial solve */
} orc_pencil;

static void orc_solveB(orc_pencil *P, const double *x, double *y)
{
    orc_polyB(P->B, P->bc, P->bh, P->bdeg, P->bcoef, x, y, P->t0, P->t1, P->t2);
}

/* One step of the B-inner-product Lanczos (Algorithm 3, "Lanczos algorithm for Ax = lambda Bx"),
 * with the operator applied to z_i already in `z`: z -= beta_i z_{i-1}; alpha = (z, w_i);
 * z -= alpha z_i; full reorthogonalisation z -= sum_j (z, w_j) z_j (two passes); w = B^{-1} z;
 * beta = (w, z)^{1/2}; w_{i+1} = w / beta, z_{i+1} = z / beta.  Returns alpha, *beta_out. */
static double orc_lanab_step(orc_pencil *P, int i, double *W, double *Z, double *z, double beta_i,
                             double *wtmp, double *beta_out)
{
    const int64_t n = P->A->n;
    double *zi = Z + (size_t)i * n, *wi = W + (size_t)i * n;
    if (i > 0)
        for (int64_t r = 0; r < n; r++) z[r] -= beta_i * Z[(size_t)(i - 1) * n + r];
    const double alpha = orc_dot(n, z, wi);
    for (int64_t r = 0; r < n; r++) z[r] -= alpha * zi[r];
    for (int pass = 0; pass < 2; pass++)
        for (int j = 0; j <= i; j++) {
            const double h = orc_dot(n, z, W + (size_t)j * n);
            const double *zj = Z + (size_t)j * n;
            for (int64_t r = 0; r < n; r++) z[r] -= h * zj[r];
        }
    orc_solveB(P, z, wtmp);
    const double beta = sqrt(fmax(0.0, orc_dot(n, wtmp, z)));
    if (beta > 0.0) {
        for (int64_t r = 0; r < n; r++) W[(size_t)(i + 1) * n + r] = wtmp[r] / beta;
        for (int64_t r = 0; r < n; r++) Z[(size_t)(i + 1) * n + r] = z[r] / beta;
    }
    *beta_out = beta;
    return alpha;
}

/* seeded start: w_1 uniform(-1,1) (stream 3, index 0), z_1 = B w_1, both scaled to (w_1, z_1) = 1 */
static void orc_lanab_start(orc_pencil *P, uint64_t seed, double *W, double *Z)
{
    const int64_t n = P->A->n;
    for (int64_t i = 0; i < n; i++) W[i] = 2.0 * orc_unit(orc_draw(seed, ORC_STREAM_LANCZOS, (uint64_t)i)) - 1.0;
    orc_matvec(P->B, W, Z);
    const double s = sqrt(orc_dot(n, W, Z));
    for (int64_t i = 0; i < n; i++) { W[i] /= s; Z[i] /= s; }
}

/* Bounds of the pencil's spectrum: `steps` B-Lanczos steps on B^{-1} A (unfiltered),
 * lmin = theta_1 - |beta s_{m,1}|, lmax = theta_m + |beta s_{m,m}| (as orc_bounds). */
int orc_bounds_gen(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                   const int64_t *brp, const int32_t *bci, const double *bv, double bmin, double bmax,
                   int bdeg, const double *bcoef, int steps, uint64_t seed, double *lmin, double *lmax)
{
    orc_csr A = {n, rp, ci, v}, B = {n, brp, bci, bv};
    double *t = malloc(sizeof(double) * 3 * n);
    orc_pencil P = {&A, &B, 0.5 * (bmax + bmin), 0.5 * (bmax - bmin), bdeg, bcoef, t, t + n, t + 2 * n};
    if (steps > n) steps = (int)n;
    double *W = calloc((size_t)n * (steps + 1), sizeof(double)), *Z = calloc((size_t)n * (steps + 1), sizeof(double));
    double *z = malloc(sizeof(double) * n), *wt = malloc(sizeof(double) * n);
    double *T = calloc((size_t)steps * steps, sizeof(double)), *S = malloc(sizeof(double) * (size_t)steps * steps);
    double *th = malloc(sizeof(double) * steps);
    orc_lanab_start(&P, seed, W, Z);
    double beta = 0.0;
    int m = 0;
    for (int i = 0; i < steps; i++) {
        orc_matvec(&A, W + (size_t)i * n, z);
        double bn = 0.0;
        const double alpha = orc_lanab_step(&P, i, W, Z, z, beta, wt, &bn);
        AT(T, i, i, steps) = alpha;
        m = i + 1;
        beta = bn;
        if (i + 1 < steps) { AT(T, i, i + 1, steps) = beta; AT(T, i + 1, i, steps) = beta; }
        if (!(beta > 0.0)) break;
    }
    double *Tm = malloc(sizeof(double) * (size_t)m * m);
    for (int j = 0; j < m; j++)
        for (int i = 0; i < m; i++) AT(Tm, i, j, m) = AT(T, i, j, steps);
    orc_syev(m, Tm, th, S);
    *lmin = th[0] - fabs(beta * AT(S, m - 1, 0, m));
    *lmax = th[m - 1] + fabs(beta * AT(S, m - 1, m - 1, m));
    free(t); free(W); free(Z); free(z); free(wt); free(T); free(S); free(th); free(Tm);
    return 0;
}

/* Filtered non-restart Lanczos for A x = lambda B x (ChebLanNr with Algorithm 3 on the pencil
 * (K, B), K = B rho(B^{-1} Ahat), Sec. 2.5): the operator applied to z_i is
 * rho(Ahat B^{-1}) z_i, a Chebyshev recurrence on Mhat = (A B^{-1} - c I) / d (B^{-1} the
 * polynomial solve).  Reorthogonalisation and the sum test as orc_cheblannr (two passes,
 * reading of Algorithm 3's single pass).  Candidates: Ritz values >= bar; x = W y (B-orthonormal),
 * lambda = x^T A x / x^T B x, dropped outside the slice, converged if
 * ||A x - lambda B x|| <= tol ||B|| max(|lmin|, |lmax|) (||B|| by bmax).  stats: its, nmv (A), 0, 0.
 */
int orc_cheblannr_gen(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                      const int64_t *brp, const int32_t *bci, const double *bv, double bmin, double bmax,
                      int bdeg, const double *bcoef, double a, double b, int right_closed, double lmin,
                      double lmax, int deg, const double *coef, double bar, int m, int ncycle, double tol,
                      double tau1, uint64_t seed, int cap, int *nev, double *lam, double *X, double *res,
                      long *stats)
{
    orc_csr A = {n, rp, ci, v}, B = {n, brp, bci, bv};
    double *t = malloc(sizeof(double) * 3 * n);
    orc_pencil P = {&A, &B, 0.5 * (bmax + bmin), 0.5 * (bmax - bmin), bdeg, bcoef, t, t + n, t + 2 * n};
    const double cc = 0.5 * (lmax + lmin), dd = 0.5 * (lmax - lmin);
    const double scale = bmax * fmax(fabs(lmin), fabs(lmax));
    if (m > n) m = (int)n;
    double *W = calloc((size_t)n * (m + 1), sizeof(double)), *Z = calloc((size_t)n * (m + 1), sizeof(double));
    double *T = calloc((size_t)(m + 1) * (m + 1), sizeof(double)), *Tk = malloc(sizeof(double) * (size_t)m * m);
    double *S = malloc(sizeof(double) * (size_t)m * m), *th = malloc(sizeof(double) * m);
    double *z = malloc(sizeof(double) * n), *wt = malloc(sizeof(double) * n);
    double *f0 = malloc(sizeof(double) * n), *f1 = malloc(sizeof(double) * n), *f2 = malloc(sizeof(double) * n);
    double *u = malloc(sizeof(double) * n), *Au = malloc(sizeof(double) * n), *Bu = malloc(sizeof(double) * n);
    long nmv = 0;
    int its = 0, status = 0, found = 0, done = 0, have_old = 0, prev_nabove = 0;
    double t_old = 0.0, beta = 0.0;
    orc_lanab_start(&P, seed, W, Z);
    for (int i = 0; i < m && !done; i++) {
        its++;
        /* z = rho(Mhat) z_i: f0 = z_i, f1 = Mhat f0, f_{j+1} = 2 Mhat f_j - f_{j-1} */
        const double *zi = Z + (size_t)i * n;
        double *p0 = f0, *p1 = f1, *p2 = f2;
        memcpy(p0, zi, sizeof(double) * n);
        for (int64_t r = 0; r < n; r++) z[r] = coef[0] * p0[r];
        for (int j = 1; j <= deg; j++) {
            const double *src = (j == 1) ? p0 : p1;                 /* f_{j-1} */
            double *dst = (j == 1) ? p1 : p2;                       /* f_j */
            orc_solveB(&P, src, u);                                 /* u = B^{-1} f_{j-1} */
            orc_matvec(&A, u, Au);
            nmv++;
            for (int64_t r = 0; r < n; r++) {
                const double mf = (Au[r] - cc * src[r]) / dd;
                dst[r] = (j == 1) ? mf : 2.0 * mf - p0[r];
            }
            for (int64_t r = 0; r < n; r++) z[r] += coef[j] * dst[r];
            if (j >= 2) { double *tmp = p0; p0 = p1; p1 = p2; p2 = tmp; }
        }
        double bn = 0.0;
        const double alpha = orc_lanab_step(&P, i, W, Z, z, beta, wt, &bn);
        AT(T, i, i, m + 1) = alpha;
        beta = bn;
        AT(T, i, i + 1, m + 1) = beta;
        AT(T, i + 1, i, m + 1) = beta;
        const int k = i + 1;
        int extract = (k == m) || !(beta > 0.0);
        if (!extract && k % ncycle == 0) {
            for (int jj = 0; jj < k; jj++)
                for (int ii = 0; ii < k; ii++) AT(Tk, ii, jj, k) = AT(T, ii, jj, m + 1);
            orc_syev(k, Tk, th, NULL);
            double t_new = 0.0;
            int nabove = 0;
            for (int jj = 0; jj < k; jj++)
                if (th[jj] >= bar) { t_new += th[jj]; nabove++; }
            int min_empty = (2 * ncycle > m / 4) ? 2 * ncycle : m / 4;
            if (have_old && nabove == 0 && prev_nabove == 0 && k >= min_empty) { done = 1; break; }
            if (have_old && nabove > 0 && fabs(t_new - t_old) < tau1 * fmax(1.0, fabs(t_new))) extract = 1;
            t_old = t_new;
            prev_nabove = nabove;
            have_old = 1;
        }
        if (!extract) continue;
        for (int jj = 0; jj < k; jj++)
            for (int ii = 0; ii < k; ii++) AT(Tk, ii, jj, k) = AT(T, ii, jj, m + 1);
        orc_syev(k, Tk, th, S);
        int nconv = 0, nunconv = 0;
        for (int jj = k - 1; jj >= 0; jj--) {
            if (th[jj] < bar) break;
            for (int64_t r = 0; r < n; r++) {
                double acc = 0.0;
                for (int p = 0; p < k; p++) acc += W[(size_t)p * n + r] * AT(S, p, jj, k);
                u[r] = acc;
            }
            orc_matvec(&B, u, Bu);
            const double nb = sqrt(orc_dot(n, u, Bu));
            for (int64_t r = 0; r < n; r++) { u[r] /= nb; Bu[r] /= nb; }
            orc_matvec(&A, u, Au);
            const double lamj = orc_dot(n, u, Au);
            int inside = (lamj >= a) && (right_closed ? (lamj <= b) : (lamj < b));
            if (!inside) continue;
            for (int64_t r = 0; r < n; r++) Au[r] -= lamj * Bu[r];
            const double rj = orc_nrm2(n, Au) / scale;
            if (rj > tol) { nunconv++; continue; }
            if (nconv >= cap) { status = -5; break; }
            if (X) memcpy(X + (size_t)nconv * n, u, sizeof(double) * n);
            lam[nconv] = lamj;
            res[nconv] = rj;
            nconv++;
        }
        found = nconv;
        if (status == -5) break;
        if (nunconv == 0 || k == m || !(beta > 0.0)) {
            if (nunconv > 0) status = -4;
            break;
        }
        have_old = 0;
    }
    for (int i = 0; i < found; i++) {                  /* ascending */
        int best = i;
        for (int j = i + 1; j < found; j++)
            if (lam[j] < lam[best]) best = j;
        if (best != i) {
            double tt = lam[i]; lam[i] = lam[best]; lam[best] = tt;
            tt = res[i]; res[i] = res[best]; res[best] = tt;
            if (X)
                for (int64_t r = 0; r < n; r++) {
                    tt = X[(size_t)i * n + r];
                    X[(size_t)i * n + r] = X[(size_t)best * n + r];
                    X[(size_t)best * n + r] = tt;
                }
        }
    }
    *nev = found;
    if (stats) { stats[0] = its; stats[1] = nmv; stats[2] = 0; stats[3] = 0; }
    free(t); free(W); free(Z); free(T); free(Tk); free(S); free(th); free(z); free(wt);
    free(f0); free(f1); free(f2); free(u); free(Au); free(Bu);
    return status;
}

/* KPM moments of the pencil (A, B) (Sec. 2.1's DOS extended to A x = lambda B x): the moments of
 * the DOS of S = B^{-1/2} A B^{-1/2}, whose eigenvalues are the pencil's.  With
 * Shat = (S - cI)/d, Rademacher probes v_l (stream 2, k = l*n+i, as orc_kpm_moments),
 * u_l = q(B) v_l ~ B^{-1/2} v_l (q: orc_lspol_isqrt) and y_0 = B u_l (~ B^{1/2} v_l):
 *   mu_k = (1/nvec) sum_l v_l^T T_k(Shat) v_l = (1/nvec) sum_l u_l^T T_k(Mhat) y_0,
 * with Mhat = (A B^{-1} - cI)/d and B^{-1} by p(B) (orc_lspol): T_k(Shat) = B^{1/2} T_k((B^{-1}A - cI)/d)
 * B^{-1/2} and B T_k((B^{-1}A - cI)/d) = T_k(Mhat) B.  Recurrence y_1 = Mhat y_0,
 * y_{k+1} = 2 Mhat y_k - y_{k-1}, each Mhat y = (A p(B) y - c y)/d. */
int orc_kpm_moments_gen(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                        const int64_t *brp, const int32_t *bci, const double *bv, double bmin, double bmax,
                        int bdeg, const double *bcoef, int sdeg, const double *scoef, int M, int nvec,
                        uint64_t seed, double lmin, double lmax, double *mu)
{
    orc_csr A = {n, rp, ci, v}, B = {n, brp, bci, bv};
    double *t = malloc(sizeof(double) * 3 * n);
    orc_pencil P = {&A, &B, 0.5 * (bmax + bmin), 0.5 * (bmax - bmin), bdeg, bcoef, t, t + n, t + 2 * n};
    const double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    double *vl = malloc(sizeof(double) * n), *u = malloc(sizeof(double) * n);
    double *y0 = malloc(sizeof(double) * n), *y1 = malloc(sizeof(double) * n), *y2 = malloc(sizeof(double) * n);
    double *s = malloc(sizeof(double) * n), *As = malloc(sizeof(double) * n);
    for (int k = 0; k <= M; k++) mu[k] = 0.0;
    for (int l = 0; l < nvec; l++) {
        for (int64_t i = 0; i < n; i++)
            vl[i] = orc_sign(orc_draw(seed, ORC_STREAM_KPM, (uint64_t)l * (uint64_t)n + (uint64_t)i));
        orc_polyB(&B, P.bc, P.bh, sdeg, scoef, vl, u, t, t + n, t + 2 * n);      /* u = q(B) v */
        orc_matvec(&B, u, y0);                                                   /* y_0 = B u */
        mu[0] += orc_dot(n, u, y0);
        double *p0 = y0, *p1 = y1, *p2 = y2;
        for (int k = 1; k <= M; k++) {
            const double *src = (k == 1) ? p0 : p1;                              /* y_{k-1} */
            double *dst = (k == 1) ? p1 : p2;                                    /* y_k */
            orc_solveB(&P, src, s);
            orc_matvec(&A, s, As);
            for (int64_t i = 0; i < n; i++) {
                const double mf = (As[i] - c * src[i]) / d;
                dst[i] = (k == 1) ? mf : 2.0 * mf - p0[i];
            }
            mu[k] += orc_dot(n, u, dst);
            if (k >= 2) { double *tmp = p0; p0 = p1; p1 = p2; p2 = tmp; }
        }
    }
    for (int k = 0; k <= M; k++) mu[k] /= nvec;
    free(t); free(vl); free(u); free(y0); free(y1); free(y2); free(s); free(As);
    return 0;
}

/* ---- Thick-restart filtered Lanczos with locking for A x = lambda B x ------------------ */
/* Vectors come in pairs (w, z = B w); the inner product of two z-vectors is (z, z')_{B^{-1}} =
 * w^T z', so a pair basis (W, Z) has W^T Z = I.  Locked eigenvectors U are B-orthonormal and
 * BU = B U is kept beside them: deflating z against them is z -= BU (U^T z), the (I - B U U^T)
 * of the paper's generalized TR scheme (Sec. 2.5). */

/* z = rho(Mhat) zi, Mhat = (A B^{-1} - cI)/d, the recurrence of orc_cheblannr_gen */
static void orc_gen_filter(orc_pencil *P, double cc, double dd, int deg, const double *coef, const double *zi,
                           double *z, double *f0, double *f1, double *f2, double *u, double *Au, long *nmv)
{
    const int64_t n = P->A->n;
    double *p0 = f0, *p1 = f1, *p2 = f2;
    memcpy(p0, zi, sizeof(double) * n);
    for (int64_t r = 0; r < n; r++) z[r] = coef[0] * p0[r];
    for (int j = 1; j <= deg; j++) {
        const double *src = (j == 1) ? p0 : p1;
        double *dst = (j == 1) ? p1 : p2;
        orc_solveB(P, src, u);
        orc_matvec(P->A, u, Au);
        (*nmv)++;
        for (int64_t r = 0; r < n; r++) {
            const double mf = (Au[r] - cc * src[r]) / dd;
            dst[r] = (j == 1) ? mf : 2.0 * mf - p0[r];
        }
        for (int64_t r = 0; r < n; r++) z[r] += coef[j] * dst[r];
        if (j >= 2) { double *tmp = p0; p0 = p1; p1 = p2; p2 = tmp; }
    }
}

/* two passes of z -= BU (U^T z) (locked, nlock columns) and z -= Z (W^T z) (basis, k columns) */
static void orc_gen_reorth(int64_t n, double *z, const double *U, const double *BU, int nlock, const double *W,
                           const double *Z, int k)
{
    for (int pass = 0; pass < 2; pass++) {
        for (int j = 0; j < nlock; j++) {
            const double h = orc_dot(n, z, U + (size_t)j * n);
            for (int64_t r = 0; r < n; r++) z[r] -= h * BU[(size_t)j * n + r];
        }
        for (int j = 0; j < k; j++) {
            const double h = orc_dot(n, z, W + (size_t)j * n);
            for (int64_t r = 0; r < n; r++) z[r] -= h * Z[(size_t)j * n + r];
        }
    }
}

/* fresh pair: w uniform(-1, 1) (stream 3, k = index*n + i), made B-orthogonal to U and W by two
 * passes of w -= U (BU^T w) and w -= W (Z^T w), z = B w, both scaled to w^T z = 1 */
static void orc_gen_fresh(orc_pencil *P, uint64_t seed, uint64_t index, double *w, double *z, const double *U,
                          const double *BU, int nlock, const double *W, const double *Z, int k)
{
    const int64_t n = P->A->n;
    for (int64_t i = 0; i < n; i++)
        w[i] = 2.0 * orc_unit(orc_draw(seed, ORC_STREAM_LANCZOS, index * (uint64_t)n + (uint64_t)i)) - 1.0;
    /* the roles of the pairs swap: B-orthogonality of w to u_j is (BU_j)^T w */
    orc_gen_reorth(n, w, BU, U, nlock, Z, W, k);
    orc_matvec(P->B, w, z);
    const double s = sqrt(orc_dot(n, w, z));
    for (int64_t i = 0; i < n; i++) { w[i] /= s; z[i] /= s; }
}

/* w = p(B) z; beta = (w^T z)^{1/2}; breakdown (returns 0) if beta <= 1e-13 ||y|| / sqrt(bmax)
 * (||y|| / sqrt(bmax) bounds the B^{-1}-norm of the filtered vector y from below) */
static int orc_gen_close(orc_pencil *P, double bmax, const double *y, double *z, double *w, double *beta)
{
    const int64_t n = P->A->n;
    orc_solveB(P, z, w);
    const double b = sqrt(fmax(0.0, orc_dot(n, w, z)));
    *beta = b;
    return b > 1e-13 * orc_nrm2(n, y) / sqrt(bmax);
}

/* Filtered thick-restart Lanczos with locking (Algorithm 2) for the pencil, in the pair basis
 * above: the operator rho(Mhat) (orc_cheblannr_gen) applied to z-vectors, Lanczos coefficients
 * alpha = w_i^T y, beta = (w^T z)^{1/2}, two reorthogonalisation passes against locked and basis
 * pairs.  READINGS: the control flow of orc_cheblantr (special TR step with the arrow matrix,
 * early restart on the sum of Ritz values >= bar, candidates largest first, lock when
 * ||A x - lambda B x|| <= tol bmax max(|lmin|, |lmax|) with x = W s B-normalised and
 * lambda = x^T A x, at most m/2 TR pairs (W s, Z s), fresh pairs after breakdown or a cycle
 * without candidates, stop after two such cycles); the refinement of stalled candidates of the
 * standard solver is not used.  stats: its, nmv, nrestart, 0. */
int orc_cheblantr_gen(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                      const int64_t *brp, const int32_t *bci, const double *bv, double bmin, double bmax,
                      int bdeg, const double *bcoef, double a, double b, int right_closed, double lmin,
                      double lmax, int deg, const double *coef, double bar, int m, int maxit, int ncycle,
                      double tol, double tau1, uint64_t seed, int cap, int *nev, double *lam, double *X,
                      double *res, long *stats)
{
    orc_csr A = {n, rp, ci, v}, B = {n, brp, bci, bv};
    double *t = malloc(sizeof(double) * 3 * n);
    orc_pencil P = {&A, &B, 0.5 * (bmax + bmin), 0.5 * (bmax - bmin), bdeg, bcoef, t, t + n, t + 2 * n};
    const double cc = 0.5 * (lmax + lmin), dd = 0.5 * (lmax - lmin);
    const double scale = bmax * fmax(fabs(lmin), fabs(lmax));
    if (m > n) m = (int)n;
    const int capc = cap > 0 ? cap : 1;
    double *U = calloc((size_t)n * capc, sizeof(double)), *BU = calloc((size_t)n * capc, sizeof(double));
    double *W = calloc((size_t)n * (m + 1), sizeof(double)), *Z = calloc((size_t)n * (m + 1), sizeof(double));
    double *T = calloc((size_t)(m + 1) * (m + 1), sizeof(double)), *Tk = malloc(sizeof(double) * (size_t)(m + 1) * (m + 1));
    double *S = malloc(sizeof(double) * (size_t)(m + 1) * (m + 1)), *theta = malloc(sizeof(double) * (m + 1));
    double *y = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n), *wt = malloc(sizeof(double) * n);
    double *f0 = malloc(sizeof(double) * n), *f1 = malloc(sizeof(double) * n), *f2 = malloc(sizeof(double) * n);
    double *u = malloc(sizeof(double) * n), *Au = malloc(sizeof(double) * n);
    double *x = malloc(sizeof(double) * n), *xz = malloc(sizeof(double) * n), *Bx = malloc(sizeof(double) * n);
    double *trw = malloc(sizeof(double) * (size_t)n * (m / 2 + 1)), *trz = malloc(sizeof(double) * (size_t)n * (m / 2 + 1));
    double *trtheta = malloc(sizeof(double) * (m + 1)), *trs = malloc(sizeof(double) * (m + 1));
    long nmv = 0;
    int nlock = 0, l = 0, its = 0, nrestart = 0, nocand = 0, status = 0;
    uint64_t fresh_index = 0;

    orc_gen_fresh(&P, seed, fresh_index++, W, Z, U, BU, 0, NULL, NULL, 0);
    while (its <= maxit) {
        int k;
        memset(T, 0, sizeof(double) * (size_t)(m + 1) * (m + 1));
        if (l > 0) {
            for (int j = 0; j < l; j++) {
                AT(T, j, j, m + 1) = trtheta[j];
                AT(T, j, l, m + 1) = trs[j];
                AT(T, l, j, m + 1) = trs[j];
            }
            const double *zl = Z + (size_t)l * n, *wl = W + (size_t)l * n;
            orc_gen_filter(&P, cc, dd, deg, coef, zl, y, f0, f1, f2, u, Au, &nmv);
            its++;
            const double alpha = orc_dot(n, wl, y);
            memcpy(z, y, sizeof(double) * n);
            for (int j = 0; j < l; j++)
                for (int64_t r = 0; r < n; r++) z[r] -= trs[j] * Z[(size_t)j * n + r];
            for (int64_t r = 0; r < n; r++) z[r] -= alpha * zl[r];
            orc_gen_reorth(n, z, U, BU, nlock, W, Z, l + 1);
            AT(T, l, l, m + 1) = alpha;
            double beta = 0.0;
            double *wn = W + (size_t)(l + 1) * n, *zn = Z + (size_t)(l + 1) * n;
            if (orc_gen_close(&P, bmax, y, z, wt, &beta)) {
                for (int64_t r = 0; r < n; r++) { wn[r] = wt[r] / beta; zn[r] = z[r] / beta; }
            } else {
                orc_gen_fresh(&P, seed, fresh_index++, wn, zn, U, BU, nlock, W, Z, l + 1);
                beta = 0.0;
            }
            AT(T, l, l + 1, m + 1) = beta;
            AT(T, l + 1, l, m + 1) = beta;
            k = l + 1;
        } else {
            k = 0;
        }
        const int lstart = k;
        double t_old = 0.0;
        int have_old = 0, prev_nabove = 0;
        for (int i = k; i < m; i++) {
            its++;
            const double *zi = Z + (size_t)i * n, *wi = W + (size_t)i * n;
            orc_gen_filter(&P, cc, dd, deg, coef, zi, y, f0, f1, f2, u, Au, &nmv);
            memcpy(z, y, sizeof(double) * n);
            if (i > 0) {
                const double bi = AT(T, i - 1, i, m + 1);
                for (int64_t r = 0; r < n; r++) z[r] -= bi * Z[(size_t)(i - 1) * n + r];
            }
            const double alpha = orc_dot(n, wi, z);
            for (int64_t r = 0; r < n; r++) z[r] -= alpha * zi[r];
            orc_gen_reorth(n, z, U, BU, nlock, W, Z, i + 1);
            AT(T, i, i, m + 1) = alpha;
            double beta = 0.0;
            double *wn = W + (size_t)(i + 1) * n, *zn = Z + (size_t)(i + 1) * n;
            if (orc_gen_close(&P, bmax, y, z, wt, &beta)) {
                for (int64_t r = 0; r < n; r++) { wn[r] = wt[r] / beta; zn[r] = z[r] / beta; }
            } else {
                orc_gen_fresh(&P, seed, fresh_index++, wn, zn, U, BU, nlock, W, Z, i + 1);
                beta = 0.0;
            }
            AT(T, i, i + 1, m + 1) = beta;
            AT(T, i + 1, i, m + 1) = beta;
            k = i + 1;
            if ((k - lstart) % ncycle == 0) {
                for (int jj = 0; jj < k; jj++)
                    for (int ii = 0; ii < k; ii++) AT(Tk, ii, jj, k) = AT(T, ii, jj, m + 1);
                orc_syev(k, Tk, theta, NULL);
                double t_new = 0.0;
                int nabove = 0;
                for (int jj = 0; jj < k; jj++)
                    if (theta[jj] >= bar) { t_new += theta[jj]; nabove++; }
                if (have_old && nabove > 0 && fabs(t_new - t_old) < tau1 * fmax(1.0, fabs(t_new))) break;
                const int min_empty = (2 * ncycle > m / 4) ? 2 * ncycle : m / 4;
                if (have_old && nabove == 0 && prev_nabove == 0 && k - lstart >= min_empty) break;
                t_old = t_new;
                prev_nabove = nabove;
                have_old = 1;
            }
            if (its > maxit) break;
        }
        nrestart++;
        for (int jj = 0; jj < k; jj++)
            for (int ii = 0; ii < k; ii++) AT(Tk, ii, jj, k) = AT(T, ii, jj, m + 1);
        orc_syev(k, Tk, theta, S);
        const double betak = AT(T, k - 1, k, m + 1);
        int ncand = 0, ntr = 0;
        for (int jj = k - 1; jj >= 0; jj--) {
            if (theta[jj] < bar) break;
            const double *s = S + (size_t)jj * k;
            for (int64_t r = 0; r < n; r++) {
                double aw = 0.0, az = 0.0;
                for (int p = 0; p < k; p++) {
                    aw += W[(size_t)p * n + r] * s[p];
                    az += Z[(size_t)p * n + r] * s[p];
                }
                x[r] = aw;
                xz[r] = az;
            }
            orc_matvec(&B, x, Bx);
            const double nb = sqrt(orc_dot(n, x, Bx));
            for (int64_t r = 0; r < n; r++) { u[r] = x[r] / nb; Bx[r] /= nb; }
            orc_matvec(&A, u, Au);
            const double lamj = orc_dot(n, u, Au);
            const int inside = (lamj >= a) && (right_closed ? (lamj <= b) : (lamj < b));
            if (!inside) continue;
            ncand++;
            for (int64_t r = 0; r < n; r++) Au[r] -= lamj * Bx[r];
            const double rj = orc_nrm2(n, Au) / scale;
            if (rj <= tol) {
                if (nlock >= cap) { status = -5; goto done; }
                memcpy(U + (size_t)nlock * n, u, sizeof(double) * n);
                memcpy(BU + (size_t)nlock * n, Bx, sizeof(double) * n);
                lam[nlock] = lamj;
                res[nlock] = rj;
                nlock++;
            } else if (ntr < m / 2) {
                memcpy(trw + (size_t)ntr * n, x, sizeof(double) * n);
                memcpy(trz + (size_t)ntr * n, xz, sizeof(double) * n);
                trtheta[ntr] = theta[jj];
                trs[ntr] = betak * s[k - 1];
                ntr++;
            }
        }
        if (ncand == 0) nocand++; else nocand = 0;
        if (nocand >= 2) break;
        if (its > maxit) { status = -4; break; }
        if (ncand == 0) {
            l = 0;
            orc_gen_fresh(&P, seed, fresh_index++, W, Z, U, BU, nlock, NULL, NULL, 0);
        } else {
            if (ntr != k) {
                memcpy(W + (size_t)ntr * n, W + (size_t)k * n, sizeof(double) * n);
                memcpy(Z + (size_t)ntr * n, Z + (size_t)k * n, sizeof(double) * n);
            }
            memcpy(W, trw, sizeof(double) * (size_t)n * ntr);
            memcpy(Z, trz, sizeof(double) * (size_t)n * ntr);
            l = ntr;
            if (l == 0) {
                /* continue from z_{k+1}, deflated against the new locked pairs */
                orc_gen_reorth(n, Z, U, BU, nlock, NULL, NULL, 0);
                orc_solveB(&P, Z, W);
                const double s = sqrt(orc_dot(n, W, Z));
                for (int64_t r = 0; r < n; r++) { W[r] /= s; Z[r] /= s; }
            }
        }
    }
done:
    for (int i = 0; i < nlock; i++) {
        int best = i;
        for (int j = i + 1; j < nlock; j++)
            if (lam[j] < lam[best]) best = j;
        if (best != i) {
            double tt = lam[i]; lam[i] = lam[best]; lam[best] = tt;
            tt = res[i]; res[i] = res[best]; res[best] = tt;
            for (int64_t r = 0; r < n; r++) {
                tt = U[(size_t)i * n + r];
                U[(size_t)i * n + r] = U[(size_t)best * n + r];
                U[(size_t)best * n + r] = tt;
            }
        }
    }
    if (X) memcpy(X, U, sizeof(double) * (size_t)n * nlock);
    *nev = nlock;
    if (stats) { stats[0] = its; stats[1] = nmv; stats[2] = nrestart; stats[3] = 0; }
    free(t); free(U); free(BU); free(W); free(Z); free(T); free(Tk); free(S); free(theta); free(y); free(z);
    free(wt); free(f0); free(f1); free(f2); free(u); free(Au); free(x); free(xz); free(Bx); free(trw); free(trz);
    free(trtheta); free(trs);
    return status;
}

/* Lanczos density of a pencil (Sec. 2.1: the DOS methods extend to A x = lambda B x with solves
 * with B and starting vectors built with B^{1/2} or the Cholesky factor; Example 1 of Sec. 3 runs
 * lanDos and spslicer2 on a pencil).  READING: the density of S = B^{-1/2} A B^{-1/2}, whose
 * eigenvalues are the pencil's.  For each of nvec unit vectors v_l (as orc_landos: uniform(-1, 1)
 * entries from stream 5, index l n + i, normalised), the pair w_1 = q(B) v_l (~ B^{-1/2} v_l,
 * q from orc_lspol_isqrt), z_1 = B w_1, scaled to w_1^T z_1 = 1, starts m steps of the
 * B-inner-product Lanczos on B^{-1} A (Algorithm 3 as in orc_bounds_gen, B^{-1} by p(B)).
 * Since B^{1/2} f(B^{-1} A) B^{-1/2} = f(S), T_m = S diag(theta) S^T gives the Gaussian
 * quadrature of v_l^T f(S) v_l: nodes theta_j, weights S_{1j}^2.  A breakdown
 * (beta <= 1e-13 ||A w_i|| / sqrt(bmax), that norm a lower bound of ||A w_i||_{B^{-1}}) ends the
 * run of that vector.  Outputs as orc_landos (nvec x m rows: nodes, weights; mused). */
int orc_landos_gen(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                   const int64_t *brp, const int32_t *bci, const double *bv, double bmin, double bmax,
                   int bdeg, const double *bcoef, int sdeg, const double *scoef, int m, int nvec,
                   uint64_t seed, double *nodes, double *weights, int *mused)
{
    orc_csr A = {n, rp, ci, v}, B = {n, brp, bci, bv};
    double *t = malloc(sizeof(double) * 3 * n);
    orc_pencil P = {&A, &B, 0.5 * (bmax + bmin), 0.5 * (bmax - bmin), bdeg, bcoef, t, t + n, t + 2 * n};
    if (m > n) m = (int)n;
    double *W = calloc((size_t)n * (m + 1), sizeof(double)), *Z = calloc((size_t)n * (m + 1), sizeof(double));
    double *T = calloc((size_t)m * m, sizeof(double)), *th = malloc(sizeof(double) * m);
    double *z = malloc(sizeof(double) * n), *wt = malloc(sizeof(double) * n), *vl = malloc(sizeof(double) * n);
    for (int l = 0; l < nvec; l++) {
        for (int64_t i = 0; i < n; i++)
            vl[i] = 2.0 * orc_unit(orc_draw(seed, ORC_STREAM_LANDOS, (uint64_t)l * (uint64_t)n + (uint64_t)i)) - 1.0;
        const double nv = orc_nrm2(n, vl);
        for (int64_t i = 0; i < n; i++) vl[i] /= nv;
        orc_polyB(&B, P.bc, P.bh, sdeg, scoef, vl, W, t, t + n, t + 2 * n);     /* w_1 = q(B) v */
        orc_matvec(&B, W, Z);                                                   /* z_1 = B w_1 */
        const double s = sqrt(orc_dot(n, W, Z));
        for (int64_t i = 0; i < n; i++) { W[i] /= s; Z[i] /= s; }
        memset(T, 0, sizeof(double) * (size_t)m * m);
        int k = 0;
        double beta = 0.0;
        for (int j = 0; j < m; j++) {
            orc_matvec(&A, W + (size_t)j * n, z);
            const double nz = orc_nrm2(n, z);
            double bn = 0.0;
            const double alpha = orc_lanab_step(&P, j, W, Z, z, beta, wt, &bn);
            AT(T, j, j, m) = alpha;
            k = j + 1;
            beta = bn;
            if (j + 1 == m || beta <= 1e-13 * nz / sqrt(bmax)) break;
            AT(T, j, j + 1, m) = beta;
            AT(T, j + 1, j, m) = beta;
        }
        double *Tk = malloc(sizeof(double) * (size_t)k * k), *Sk = malloc(sizeof(double) * (size_t)k * k);
        for (int c = 0; c < k; c++)
            for (int r = 0; r < k; r++) AT(Tk, r, c, k) = AT(T, r, c, m);
        orc_syev(k, Tk, th, Sk);
        for (int j = 0; j < m; j++) {
            nodes[(size_t)l * m + j] = j < k ? th[j] : 0.0;
            weights[(size_t)l * m + j] = j < k ? AT(Sk, 0, j, k) * AT(Sk, 0, j, k) : 0.0;
        }
        mused[l] = k;
        free(Tk);
        free(Sk);
    }
    free(t); free(W); free(Z); free(T); free(th); free(z); free(wt); free(vl);
    return 0;
}
