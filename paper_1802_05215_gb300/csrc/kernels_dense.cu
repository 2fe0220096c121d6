// Dense kernels for sm_103a used by the filtered Lanczos driver:
//  - deterministic two-phase reductions (per-chunk partials, then a fixed-order sum),
//  - the classical Gram-Schmidt projections of the full reorthogonalisation (Sec. 2.3):
//    h = [U Q]^T z (GEMV-T) and z -= [U Q] h (GEMV-N), HBM-streaming kernels,
//  - Ritz vectors Y = Q S (FP64 GEMM, Algorithm 2 "compute candidate Ritz pairs"),
//  - the eigensolves of the projected matrix: cyclic two-sided Jacobi (round-robin pairs,
//    Golub & Van Loan Sec. 8.5) for the restart, and Sturm-count bisection on the
//    arrowhead-plus-tridiagonal matrix for the early-restart test.
#include <algorithm>
#include <cmath>
#include <vector>

#include "evsl_internal.h"

namespace {

constexpr int RT = 256;       // threads per block of the row-streaming kernels
constexpr int RPT = 8;        // rows per thread in a reduction chunk
constexpr int64_t CHUNK = RT * RPT;

inline unsigned nblk(int64_t threads, int tpb) { return (unsigned)((threads + tpb - 1) / tpb); }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// block-wide sum of one value per thread (blockDim.x == RT); result valid in thread 0
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[RT / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < RT / 32; i++) t += red[i];
    return t;
}

// out[j] = sum_c part[j * nch + c], one warp per output, fixed order
__global__ void k_reduce(int k, int64_t nch, const double *__restrict__ part, double *__restrict__ out)
{
    int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (j >= k) return;
    double s = 0.0;
    for (int64_t c = lane; c < nch; c += 32) s += part[(int64_t)j * nch + c];
    s = warp_sum(s);
    if (lane == 0) out[j] = s;
}

__global__ void __launch_bounds__(RT)
k_coldot(int64_t n, int64_t nch, const double *__restrict__ X, int64_t ldx,
         const double *__restrict__ Y, int64_t ldy, double *__restrict__ part)
{
    int64_t c = blockIdx.x;
    int j = blockIdx.y;
    const double *x = X + (int64_t)j * ldx;
    const double *y = Y + (int64_t)j * ldy;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < RPT; i++) {
        int64_t r = c * CHUNK + i * RT + threadIdx.x;
        if (r < n) s += x[r] * y[r];
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[(int64_t)j * nch + c] = s;
}

__global__ void __launch_bounds__(RT)
k_colres2(int64_t n, int64_t nch, const double *__restrict__ Z, const double *__restrict__ Y,
          int64_t ld, const double *__restrict__ lam, double *__restrict__ part)
{
    int64_t c = blockIdx.x;
    int j = blockIdx.y;
    const double *z = Z + (int64_t)j * ld;
    const double *y = Y + (int64_t)j * ld;
    double l = lam[j];
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < RPT; i++) {
        int64_t r = c * CHUNK + i * RT + threadIdx.x;
        if (r < n) {
            double t = z[r] - l * y[r];
            s += t * t;
        }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[(int64_t)j * nch + c] = s;
}

// z = y - beta qprev ; partial of q . z
__global__ void __launch_bounds__(RT)
k_three_term(int64_t n, const double *y, const double *__restrict__ qprev, double beta,
             const double *__restrict__ q, double *z, double *__restrict__ part)
{
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < RPT; i++) {
        int64_t r = blockIdx.x * CHUNK + i * RT + threadIdx.x;
        if (r < n) {
            double v = y[r];
            if (qprev) v -= beta * qprev[r];
            z[r] = v;
            s += q[r] * v;
        }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// z -= alpha q ; partial of ||z||^2
__global__ void __launch_bounds__(RT)
k_sub_alpha(int64_t n, double *__restrict__ z, const double *__restrict__ q,
            const double *__restrict__ alpha, double *__restrict__ part)
{
    double a = *alpha;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < RPT; i++) {
        int64_t r = blockIdx.x * CHUNK + i * RT + threadIdx.x;
        if (r < n) {
            double v = z[r] - a * q[r];
            z[r] = v;
            s += v * v;
        }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// GEMV-T over two column blocks.  Block (chunk c, column group g) computes, for the 32
// columns of the group, the partial dot products with z over the chunk's rows.  Each warp
// keeps 32 accumulators and reduces them with a transposing butterfly (31 shuffles) so that
// lane j ends with column j's warp sum; the 8 warp sums are then added in a fixed order.
constexpr int GT_COLS = 32;

__global__ void __launch_bounds__(RT)
k_gemv_t2(int64_t n, int64_t nch, const double *__restrict__ B1, int k1,
          const double *__restrict__ B2, int k2, const double *__restrict__ z,
          double *__restrict__ part)
{
    __shared__ double red[RT / 32][GT_COLS];
    int64_t c = blockIdx.x;
    int j0 = blockIdx.y * GT_COLS;
    int k = k1 + k2;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[GT_COLS];
#pragma unroll
    for (int j = 0; j < GT_COLS; j++) acc[j] = 0.0;
#pragma unroll 1
    for (int i = 0; i < RPT; i++) {
        int64_t r = c * CHUNK + i * RT + threadIdx.x;
        if (r >= n) break;
        double zr = z[r];
#pragma unroll
        for (int j = 0; j < GT_COLS; j++) {
            int jj = j0 + j;
            if (jj < k) {
                const double *col = (jj < k1) ? (B1 + (int64_t)jj * n) : (B2 + (int64_t)(jj - k1) * n);
                acc[j] += col[r] * zr;
            }
        }
    }
    // transposing butterfly: after the loop lane L holds the warp sum of column L
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; i++) {
            double send = upper ? acc[i] : acc[i + s];
            double keep = upper ? acc[i + s] : acc[i];
            acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    red[warp][lane] = acc[0];
    __syncthreads();
    if (threadIdx.x < GT_COLS) {
        int jj = j0 + threadIdx.x;
        double t = 0.0;
        for (int w = 0; w < RT / 32; w++) t += red[w][threadIdx.x];
        if (jj < k) part[(int64_t)jj * nch + c] = t;
    }
}

// GEMV-N over two column blocks: z -= [B1 B2] h, h staged in shared memory; partial ||z||^2
constexpr int GN_RPT = 4;

__global__ void __launch_bounds__(RT)
k_gemv_n2(int64_t n, const double *__restrict__ B1, int k1, const double *__restrict__ B2,
          int k2, const double *__restrict__ h, double *__restrict__ z, double *__restrict__ part)
{
    extern __shared__ double hs[];
    int k = k1 + k2;
    for (int j = threadIdx.x; j < k; j += RT) hs[j] = h[j];
    __syncthreads();
    int64_t r0 = (int64_t)blockIdx.x * RT * GN_RPT + threadIdx.x;
    double acc[GN_RPT];
#pragma unroll
    for (int i = 0; i < GN_RPT; i++) acc[i] = 0.0;
    for (int j = 0; j < k; j++) {
        const double *col = (j < k1) ? (B1 + (int64_t)j * n) : (B2 + (int64_t)(j - k1) * n);
        double hj = hs[j];
#pragma unroll
        for (int i = 0; i < GN_RPT; i++) {
            int64_t r = r0 + (int64_t)i * RT;
            if (r < n) acc[i] += col[r] * hj;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < GN_RPT; i++) {
        int64_t r = r0 + (int64_t)i * RT;
        if (r < n) {
            double v = z[r] - acc[i];
            z[r] = v;
            s += v * v;
        }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_scale(int64_t n, const double *x, double s, double *y)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = s * x[i];
}

__global__ void k_colscale(int64_t n, int k, double *__restrict__ Y, const double *__restrict__ nrm2)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i < n && j < k) Y[(int64_t)j * n + i] *= 1.0 / sqrt(nrm2[j]);
}

// Y[:, j] *= scale[j] (columns of length rows)
__global__ void k_colscale_by(int64_t rows, double *__restrict__ Y, const double *__restrict__ scale)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i < rows) Y[(int64_t)j * rows + i] *= scale[j];
}

__global__ void k_gather(int64_t rows, int k, const double *__restrict__ src, int64_t lds,
                         const int *__restrict__ idx, double *__restrict__ dst, int64_t ldd)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int t = blockIdx.y;
    if (i < rows) dst[(int64_t)t * ldd + i] = src[(int64_t)idx[t] * lds + i];
}

// C = A B, FP64, 64 x 64 tiles, 16-deep k panels, 4 x 4 outputs per thread.
constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

// SUB = true: C -= A B instead of C = A B
template <bool SUB>
__global__ void __launch_bounds__(256)
k_gemm_nn(int64_t n, int l, int k, const double *__restrict__ A, int64_t lda,
          const double *__restrict__ B, int64_t ldb, double *__restrict__ C, int64_t ldc)
{
    __shared__ double As[GB_K][GB_M + 1];
    __shared__ double Bs[GB_K][GB_N + 1];
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int64_t row0 = (int64_t)blockIdx.x * GB_M;
    int col0 = blockIdx.y * GB_N;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < k; k0 += GB_K) {
#pragma unroll
        for (int t = 0; t < 4; t++) {
            int e = threadIdx.x + 256 * t;      // 0..1023
            int rr = e & 63, kk = e >> 6;       // A tile: 64 rows x 16
            int64_t gr = row0 + rr;
            int gk = k0 + kk;
            As[kk][rr] = (gr < n && gk < k) ? A[(int64_t)gk * lda + gr] : 0.0;
            int bk = e & 15, bc = e >> 4;       // B tile: 16 x 64
            int gbk = k0 + bk, gbc = col0 + bc;
            Bs[bk][bc] = (gbk < k && gbc < l) ? B[(int64_t)gbc * ldb + gbk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int64_t gr = row0 + tx + 16 * i;
        if (gr >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int gc = col0 + ty + 16 * j;
            if (gc < l) {
                if (SUB)
                    C[(int64_t)gc * ldc + gr] -= acc[i][j];
                else
                    C[(int64_t)gc * ldc + gr] = acc[i][j];
            }
        }
    }
}

// C = A^T B (A: n x p, B: n x q, column-major), split over row ranges: block (i, j, z)
// accumulates the 64 x 64 tile (i, j) over rows [z*rows, (z+1)*rows) into part[z].
__global__ void __launch_bounds__(256)
k_gemm_tn(int64_t n, int p, int q, const double *__restrict__ A, int64_t lda,
          const double *__restrict__ B, int64_t ldb, int64_t rows, double *__restrict__ part)
{
    __shared__ double As[GB_K][GB_M + 1];
    __shared__ double Bs[GB_K][GB_N + 1];
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int i0 = blockIdx.x * GB_M, j0 = blockIdx.y * GB_N;
    int64_t r_begin = (int64_t)blockIdx.z * rows, r_end = min(n, r_begin + rows);
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    for (int64_t r0 = r_begin; r0 < r_end; r0 += GB_K) {
#pragma unroll
        for (int t = 0; t < 4; t++) {
            int e = threadIdx.x + 256 * t;  // 0..1023: 16 rows x 64 columns
            int rr = e & 15, cc = e >> 4;
            int64_t gr = r0 + rr;
            As[rr][cc] = (gr < r_end && i0 + cc < p) ? A[(int64_t)(i0 + cc) * lda + gr] : 0.0;
            Bs[rr][cc] = (gr < r_end && j0 + cc < q) ? B[(int64_t)(j0 + cc) * ldb + gr] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
    double *out = part + (int64_t)blockIdx.z * p * q;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int gi = i0 + tx + 16 * i;
        if (gi >= p) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int gj = j0 + ty + 16 * j;
            if (gj < q) out[(int64_t)gj * p + gi] = acc[i][j];
        }
    }
}

// C[i + j*ldc] = sum_z part[z][i + j*p], fixed order
__global__ void k_sum_splits(int p, int q, int nsplit, const double *__restrict__ part,
                             double *__restrict__ C, int64_t ldc)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)p * q) return;
    int i = (int)(t % p), j = (int)(t / p);
    double s = 0.0;
    for (int z = 0; z < nsplit; z++) s += part[(int64_t)z * p * q + t];
    C[(int64_t)j * ldc + i] = s;
}

// ---------------------------------------------------------------- Jacobi eigensolver
// Round-robin ("chess tournament") pairing of M (even) indices: round r in [0, M-1),
// pair i in [0, M/2).  Every unordered pair occurs once per sweep of M-1 rounds.
__device__ __forceinline__ void rr_pair(int M, int r, int i, int *p, int *q)
{
    if (i == 0) {
        *p = M - 1;
        *q = r;
    } else {
        *p = (r + i) % (M - 1);
        *q = (r - i + (M - 1)) % (M - 1);
    }
}

// rotation for pair i: J = [c s; -s c] on (p, q) annihilates a_pq (Golub-Van Loan sym.schur2)
__global__ void k_jac_params(int M, int m, int r, const double *__restrict__ Amat, double *__restrict__ cs,
                             int *__restrict__ nrot)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M / 2) return;
    int p, q;
    rr_pair(M, r, i, &p, &q);
    double c = 1.0, s = 0.0;
    if (p < m && q < m) {
        double apq = Amat[(int64_t)q * M + p];
        double app = Amat[(int64_t)p * M + p], aqq = Amat[(int64_t)q * M + q];
        if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            double tau = (aqq - app) / (2.0 * apq);
            double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            atomicAdd(nrot, 1);
        }
    }
    cs[2 * i] = c;
    cs[2 * i + 1] = s;
}

// A <- J^T A J on all 2 x 2 blocks (rows of pair i, columns of pair j), V <- V J
__global__ void k_jac_apply(int M, int r, double *__restrict__ Amat, double *__restrict__ V,
                            const double *__restrict__ cs)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t H = M / 2;
    if (t < H * H) {
        int i = (int)(t % H), j = (int)(t / H);
        int pi, qi, pj, qj;
        rr_pair(M, r, i, &pi, &qi);
        rr_pair(M, r, j, &pj, &qj);
        double ci = cs[2 * i], si = cs[2 * i + 1], cj = cs[2 * j], sj = cs[2 * j + 1];
        if (si == 0.0 && sj == 0.0) return;
        double b00 = Amat[(int64_t)pj * M + pi], b01 = Amat[(int64_t)qj * M + pi];
        double b10 = Amat[(int64_t)pj * M + qi], b11 = Amat[(int64_t)qj * M + qi];
        double t00 = ci * b00 - si * b10, t01 = ci * b01 - si * b11;
        double t10 = si * b00 + ci * b10, t11 = si * b01 + ci * b11;
        double n00 = cj * t00 - sj * t01, n01 = sj * t00 + cj * t01;
        double n10 = cj * t10 - sj * t11, n11 = sj * t10 + cj * t11;
        if (i == j) {
            n01 = 0.0;
            n10 = 0.0;
        }
        Amat[(int64_t)pj * M + pi] = n00;
        Amat[(int64_t)qj * M + pi] = n01;
        Amat[(int64_t)pj * M + qi] = n10;
        Amat[(int64_t)qj * M + qi] = n11;
    } else {
        int64_t u = t - H * H;
        if (u >= (int64_t)M * H) return;
        int row = (int)(u % M), j = (int)(u / M);
        double cj = cs[2 * j], sj = cs[2 * j + 1];
        if (sj == 0.0) return;
        int pj, qj;
        rr_pair(M, r, j, &pj, &qj);
        double vp = V[(int64_t)pj * M + row], vq = V[(int64_t)qj * M + row];
        V[(int64_t)pj * M + row] = cj * vp - sj * vq;
        V[(int64_t)qj * M + row] = sj * vp + cj * vq;
    }
}

__global__ void k_init_eye(int M, int m, double *__restrict__ V)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < (int64_t)M * M) {
        int i = (int)(t % M), j = (int)(t / M);
        V[t] = (i == j) ? 1.0 : 0.0;
    }
}

// partials: [0] off-diagonal sum of squares, [1] total sum of squares, per block
__global__ void __launch_bounds__(RT)
k_jac_norms(int M, const double *__restrict__ Amat, double *__restrict__ part)
{
    int64_t total = (int64_t)M * M;
    double off = 0.0, all = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)RT + threadIdx.x; t < total; t += (int64_t)gridDim.x * RT) {
        double v = Amat[t];
        int i = (int)(t % M), j = (int)(t / M);
        all += v * v;
        if (i != j) off += v * v;
    }
    double so = block_sum(off);
    __syncthreads();
    double sa = block_sum(all);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = so;
        part[gridDim.x + blockIdx.x] = sa;
    }
}

__global__ void k_diag(int m, int M, const double *__restrict__ Amat, double *__restrict__ w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) w[i] = Amat[(int64_t)i * M + i];
}

// ---------------------------------------------------------------- bisection
// Number of eigenvalues < sigma of the arrow + tridiagonal matrix (Sylvester's law of inertia).
// Arrow rows i < l: pivots d_i - sigma (independent, so their divisions pipeline) and their
// Schur complement sum_i e_i^2 / (d_i - sigma) folded into row l.  Rows i >= l: the leading
// minors p_i = (d_i - sigma) p_{i-1} - e_{i-1}^2 p_{i-2} (p_{l-1} = 1, p_l = pivot of row l)
// without divisions; a sign change between consecutive minors is a negative pivot.  The pair
// (p_{i-1}, p_i) is rescaled by 2^-600 / 2^600 when it grows or shrinks too far (exact scaling,
// signs unchanged); a zero minor becomes -pmin times the previous one (a negative pivot).
__device__ int dev_count_below(int k, int l, const double *__restrict__ d, const double *__restrict__ e,
                               double sigma, double pmin)
{
    int cnt = 0;
    double sum = 0.0;
    for (int i = 0; i < l; i++) {
        double piv = d[i] - sigma;
        if (fabs(piv) < pmin) piv = -pmin;
        cnt += piv < 0.0;
        sum += e[i] * e[i] / piv;
    }
    if (l >= k) return cnt;
    double pm = 1.0;                      // p_{i-1}
    double p = d[l] - sigma - sum;        // p_l (pivot of row l times p_{l-1} = 1)
    if (fabs(p) < pmin) p = -pmin;
    cnt += p < 0.0;
    for (int i = l + 1; i < k; i++) {
        double e2 = e[i - 1] * e[i - 1];
        double pn = (d[i] - sigma) * p - e2 * pm;
        if (pn == 0.0) pn = -pmin * p;  // a zero pivot counts as negative
        cnt += (pn < 0.0) != (p < 0.0);
        pm = p;
        p = pn;
        double ap = fabs(p);
        if (ap > 0x1p+600) {
            p *= 0x1p-600;
            pm *= 0x1p-600;
        } else if (ap < 0x1p-600) {
            p *= 0x1p+600;
            pm *= 0x1p+600;
        }
    }
    return cnt;
}

// one eigenvalue per thread, few threads per block so that the work spreads over all SMs
__global__ void k_bisect(int k, int l, const double *__restrict__ d, const double *__restrict__ e,
                         int k0, int k1, double lo0, double hi0, double pmin, double *__restrict__ w)
{
    int j = k0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k1) return;
    double lo = lo0, hi = hi0;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (hi - lo <= 4.5e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300 || mid <= lo || mid >= hi) break;
        if (dev_count_below(k, l, d, e, mid, pmin) > j)
            hi = mid;
        else
            lo = mid;
    }
    w[j - k0] = 0.5 * (lo + hi);
}

// Multisection: one warp per eigenvalue j (ascending index); each round the 32 lanes count
// the eigenvalues below 32 interior points of [lo, hi] (33 equal parts) at once and the
// bracket shrinks to the part where the count passes j, so a round does the work of five
// bisection steps with the same sequential depth as one.  d and e are staged in shared memory.
// Same stopping rule as k_bisect.
__global__ void k_multisect(int k, int l, const double *__restrict__ dg, const double *__restrict__ eg,
                            int k0, int k1, double lo0, double hi0, double pmin, double *__restrict__ w)
{
    extern __shared__ double sh[];
    double *d = sh, *e = sh + k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        d[i] = dg[i];
        e[i] = eg[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int j = k0 + (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (j >= k1) return;  // whole warps leave together
    double lo = lo0, hi = hi0;
    for (int it = 0; it < 64; it++) {
        if (hi - lo <= 4.5e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
        const double h = (hi - lo) * (1.0 / 33.0);
        const double x = lo + h * (double)(lane + 1);
        const bool above = dev_count_below(k, l, d, e, x, pmin) > j;  // lambda_j < x
        const unsigned b = __ballot_sync(0xffffffffu, above);
        const double nlo = (b == 0u) ? lo + h * 32.0 : (__ffs(b) == 1 ? lo : lo + h * (double)(__ffs(b) - 1));
        const double nhi = (b == 0u) ? hi : lo + h * (double)__ffs(b);
        if (!(nlo > lo) && !(nhi < hi)) break;  // the points no longer split the bracket
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) w[j - k0] = 0.5 * (lo + hi);
}

}  // namespace

// ------------------------------------------------------------------------------------------
int64_t red_nchunks(int64_t n) { return (n + CHUNK - 1) / CHUNK; }

static double *partials(evsl_ctx *c, int64_t count, int *st)
{
    return (double *)ctx_ws(c, WS_PARTIAL, sizeof(double) * std::max<int64_t>(count, 1), st);
}

static int reduce_to(evsl_ctx *c, int k, int64_t nch, const double *part, double *out)
{
    k_reduce<<<nblk((int64_t)k * 32, 256), 256, 0, c->stream>>>(k, nch, part, out);
    c->launches++;
    return check_launch(c, "reduce");
}

int reduce_rows(evsl_ctx *c, int k, int64_t nch, const double *part, double *out)
{
    return reduce_to(c, k, nch, part, out);
}

int coldot(evsl_ctx *c, int64_t n, int k, const double *X, int64_t ldx, const double *Y,
           int64_t ldy, double *out)
{
    if (k <= 0) return EVSL_OK;
    int64_t nch = red_nchunks(n);
    int st = EVSL_OK;
    double *part = partials(c, nch * k, &st);
    if (st) return st;
    k_coldot<<<dim3((unsigned)nch, k), RT, 0, c->stream>>>(n, nch, X, ldx, Y, ldy, part);
    c->launches++;
    EVSL_TRY(check_launch(c, "coldot"));
    return reduce_to(c, k, nch, part, out);
}

int colres2(evsl_ctx *c, int64_t n, int k, const double *Z, const double *Y, int64_t ld,
            const double *lam, double *out)
{
    if (k <= 0) return EVSL_OK;
    int64_t nch = red_nchunks(n);
    int st = EVSL_OK;
    double *part = partials(c, nch * k, &st);
    if (st) return st;
    k_colres2<<<dim3((unsigned)nch, k), RT, 0, c->stream>>>(n, nch, Z, Y, ld, lam, part);
    c->launches++;
    EVSL_TRY(check_launch(c, "colres2"));
    return reduce_to(c, k, nch, part, out);
}

int lan_three_term(evsl_ctx *c, int64_t n, const double *y, const double *qprev, double beta,
                   const double *q, double *z, double *out_dot)
{
    int64_t nch = red_nchunks(n);
    int st = EVSL_OK;
    double *part = partials(c, nch, &st);
    if (st) return st;
    k_three_term<<<(unsigned)nch, RT, 0, c->stream>>>(n, y, qprev, beta, q, z, part);
    c->launches++;
    EVSL_TRY(check_launch(c, "three_term"));
    return reduce_to(c, 1, nch, part, out_dot);
}

int lan_sub_alpha(evsl_ctx *c, int64_t n, double *z, const double *q, const double *alpha,
                  double *out_nrm2)
{
    int64_t nch = red_nchunks(n);
    int st = EVSL_OK;
    double *part = partials(c, nch, &st);
    if (st) return st;
    k_sub_alpha<<<(unsigned)nch, RT, 0, c->stream>>>(n, z, q, alpha, part);
    c->launches++;
    EVSL_TRY(check_launch(c, "sub_alpha"));
    return reduce_to(c, 1, nch, part, out_nrm2);
}

int gemv_t2(evsl_ctx *c, int64_t n, const double *B1, int k1, const double *B2, int k2,
            const double *z, double *h)
{
    int k = k1 + k2;
    if (k <= 0) return EVSL_OK;
    int64_t nch = red_nchunks(n);
    int st = EVSL_OK;
    double *part = partials(c, nch * k, &st);
    if (st) return st;
    dim3 grid((unsigned)nch, (unsigned)((k + GT_COLS - 1) / GT_COLS));
    k_gemv_t2<<<grid, RT, 0, c->stream>>>(n, nch, B1, k1, B2, k2, z, part);
    c->launches++;
    EVSL_TRY(check_launch(c, "gemv_t2"));
    return reduce_to(c, k, nch, part, h);
}

int gemv_n2(evsl_ctx *c, int64_t n, const double *B1, int k1, const double *B2, int k2,
            const double *h, double *z, double *out_nrm2)
{
    int k = k1 + k2;
    int64_t nb = (n + RT * GN_RPT - 1) / (RT * GN_RPT);
    int st = EVSL_OK;
    double *part = partials(c, nb, &st);
    if (st) return st;
    size_t smem = sizeof(double) * std::max(k, 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_gemv_n2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return ctx_cuda(c, e, "gemv_n2 smem");
    }
    k_gemv_n2<<<(unsigned)nb, RT, smem, c->stream>>>(n, B1, k1, B2, k2, h, z, part);
    c->launches++;
    EVSL_TRY(check_launch(c, "gemv_n2"));
    return reduce_to(c, 1, nb, part, out_nrm2);
}

int scale_vec(evsl_ctx *c, int64_t n, double *x, double s, double *dst)
{
    k_scale<<<nblk(n, 256), 256, 0, c->stream>>>(n, x, s, dst ? dst : x);
    c->launches++;
    return check_launch(c, "scale");
}

int colscale_inv_sqrt(evsl_ctx *c, int64_t n, int k, double *Y, const double *nrm2)
{
    if (k <= 0) return EVSL_OK;
    k_colscale<<<dim3(nblk(n, 256), k), 256, 0, c->stream>>>(n, k, Y, nrm2);
    c->launches++;
    return check_launch(c, "colscale");
}

// Large products go to the tensor-core GEMM (FP64-accurate digit splitting); small ones, whose
// splitting and launch costs would dominate, stay on the FP64 kernels below, and so does a
// product whose digit workspace does not fit under the HBM budget (same result to rounding).
static bool use_tc(const evsl_ctx *c, int64_t M, int64_t N, int64_t K)
{
    return c->tc_gemm && M >= 128 && N >= 16 && K >= 32 && 2.0 * (double)M * (double)N * (double)K >= 1e9;
}

static int try_tc(evsl_ctx *c, bool trans_a, int64_t M, int N, int64_t K, const double *A, int64_t lda,
                  const double *B, int64_t ldb, double *C, int64_t ldc, int mode, bool *done)
{
    *done = false;
    if (!use_tc(c, M, N, K)) return EVSL_OK;
    const int st = gemm_tc(c, trans_a, M, N, K, A, lda, B, ldb, C, ldc, mode);
    if (st == EVSL_ERR_NOMEM) {
        c->err.clear();
        return EVSL_OK;
    }
    *done = true;
    return st;
}

int gemm_nn(evsl_ctx *c, int64_t n, int l, int k, const double *A, int64_t lda, const double *B,
            int64_t ldb, double *C, int64_t ldc)
{
    if (n <= 0 || l <= 0) return EVSL_OK;
    bool done = false;
    EVSL_TRY(try_tc(c, false, n, l, k, A, lda, B, ldb, C, ldc, 0, &done));
    if (done) return EVSL_OK;
    dim3 grid((unsigned)((n + GB_M - 1) / GB_M), (unsigned)((l + GB_N - 1) / GB_N));
    k_gemm_nn<false><<<grid, 256, 0, c->stream>>>(n, l, k, A, lda, B, ldb, C, ldc);
    c->launches++;
    return check_launch(c, "gemm_nn");
}

int gemm_nn_sub(evsl_ctx *c, int64_t n, int l, int k, const double *A, int64_t lda, const double *B,
                int64_t ldb, double *C, int64_t ldc)
{
    if (n <= 0 || l <= 0 || k <= 0) return EVSL_OK;
    bool done = false;
    EVSL_TRY(try_tc(c, false, n, l, k, A, lda, B, ldb, C, ldc, 1, &done));
    if (done) return EVSL_OK;
    dim3 grid((unsigned)((n + GB_M - 1) / GB_M), (unsigned)((l + GB_N - 1) / GB_N));
    k_gemm_nn<true><<<grid, 256, 0, c->stream>>>(n, l, k, A, lda, B, ldb, C, ldc);
    c->launches++;
    return check_launch(c, "gemm_nn_sub");
}

int colscale(evsl_ctx *c, int64_t rows, int k, double *Y, const double *scale)
{
    if (k <= 0) return EVSL_OK;
    k_colscale_by<<<dim3(nblk(rows, 256), k), 256, 0, c->stream>>>(rows, Y, scale);
    c->launches++;
    return check_launch(c, "colscale");
}

int gemm_tn(evsl_ctx *c, int64_t n, int p, int q, const double *A, int64_t lda, const double *B,
            int64_t ldb, double *C, int64_t ldc)
{
    if (p <= 0 || q <= 0) return EVSL_OK;
    bool done = false;
    EVSL_TRY(try_tc(c, true, p, q, n, A, lda, B, ldb, C, ldc, 0, &done));
    if (done) return EVSL_OK;
    int tiles = ((p + GB_M - 1) / GB_M) * ((q + GB_N - 1) / GB_N);
    int64_t nsplit = std::max<int64_t>(1, (4 * (int64_t)c->dev_sm_count + tiles - 1) / tiles);
    nsplit = std::min<int64_t>(nsplit, std::max<int64_t>(1, n / 1024));
    int64_t rows = (n + nsplit - 1) / nsplit;
    rows = (rows + GB_K - 1) / GB_K * GB_K;
    nsplit = (n + rows - 1) / rows;
    int st = EVSL_OK;
    double *part = partials(c, nsplit * (int64_t)p * q, &st);
    if (st) return st;
    dim3 grid((unsigned)((p + GB_M - 1) / GB_M), (unsigned)((q + GB_N - 1) / GB_N), (unsigned)nsplit);
    k_gemm_tn<<<grid, 256, 0, c->stream>>>(n, p, q, A, lda, B, ldb, rows, part);
    c->launches++;
    EVSL_TRY(check_launch(c, "gemm_tn"));
    k_sum_splits<<<nblk((int64_t)p * q, 256), 256, 0, c->stream>>>(p, q, (int)nsplit, part, C, ldc);
    c->launches++;
    return check_launch(c, "gemm_tn reduce");
}

int gather_cols(evsl_ctx *c, int64_t rows, int k, const double *src, int64_t lds, const int *idx,
                double *dst, int64_t ldd)
{
    if (k <= 0) return EVSL_OK;
    k_gather<<<dim3(nblk(rows, 256), k), 256, 0, c->stream>>>(rows, k, src, lds, idx, dst, ldd);
    c->launches++;
    return check_launch(c, "gather_cols");
}

int jacobi_eig(evsl_ctx *c, int m, const double *T_host, double *w_host, double *V, int *ldv,
               int *sweeps_out)
{
    // T_host: m x m column-major.  Works on an M x M (M even) padded copy.
    int M = m + (m & 1);
    if (M < 2) M = 2;
    int st = EVSL_OK;
    double *Amat = (double *)ctx_ws(c, WS_LAN_S, sizeof(double) * (size_t)M * M, &st);
    if (st) return st;
    double *aux = (double *)ctx_ws(c, WS_JAC_PAIRS, sizeof(double) * (M + 2 * 1024 + 16), &st);
    if (st) return st;
    double *cs = aux;
    double *part = aux + M;
    int *nrot = (int *)(aux + M + 2 * 1024);
    std::vector<double> Ap((size_t)M * M, 0.0);
    for (int j = 0; j < m; j++)
        for (int i = 0; i < m; i++) Ap[(size_t)j * M + i] = T_host[(size_t)j * m + i];
    cudaError_t e = cudaMemcpyAsync(Amat, Ap.data(), sizeof(double) * (size_t)M * M,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "jacobi upload");
    k_init_eye<<<nblk((int64_t)M * M, 256), 256, 0, c->stream>>>(M, m, V);
    c->launches++;
    EVSL_TRY(check_launch(c, "jacobi init"));
    ProfGroup g;
    prof_begin(c, EVSL_K_SMALL_EIG, &g);
    int launches = 0, sweep = 0;
    const int nb_norm = 64;
    int64_t apply_threads = (int64_t)(M / 2) * (M / 2) + (int64_t)M * (M / 2);
    for (sweep = 0; sweep < 40; sweep++) {
        e = cudaMemsetAsync(nrot, 0, sizeof(int), c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "jacobi memset");
        for (int r = 0; r < M - 1; r++) {
            k_jac_params<<<nblk(M / 2, 128), 128, 0, c->stream>>>(M, m, r, Amat, cs, nrot);
            k_jac_apply<<<nblk(apply_threads, 256), 256, 0, c->stream>>>(M, r, Amat, V, cs);
            launches += 2;
        }
        c->launches += 2 * (M - 1);
        EVSL_TRY(check_launch(c, "jacobi sweep"));
        k_jac_norms<<<nb_norm, RT, 0, c->stream>>>(M, Amat, part);
        c->launches++;
        launches++;
        EVSL_TRY(check_launch(c, "jacobi norms"));
        double hp[2 * nb_norm];
        int hrot = 0;
        e = cudaMemcpyAsync(hp, part, sizeof(double) * 2 * nb_norm, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hrot, nrot, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "jacobi norms readback");
        double off = 0.0, all = 0.0;
        for (int i = 0; i < nb_norm; i++) {
            off += hp[i];
            all += hp[nb_norm + i];
        }
        if (hrot == 0 || off <= 1e-30 * all) {
            sweep++;
            break;
        }
    }
    prof_end(c, &g, launches);
    double *wd = cs;  // reuse (M >= m)
    k_diag<<<nblk(m, 128), 128, 0, c->stream>>>(m, M, Amat, wd);
    c->launches++;
    EVSL_TRY(check_launch(c, "jacobi diag"));
    e = cudaMemcpyAsync(w_host, wd, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "jacobi eigenvalues readback");
    *ldv = M;
    if (sweeps_out) *sweeps_out = sweep;
    return EVSL_OK;
}

int bisect_eigs(evsl_ctx *c, int k, int l, const double *d_host, const double *e_host, int k0,
                int k1, double lo, double hi, double *w_host)
{
    int cnt = k1 - k0;
    if (cnt <= 0) return EVSL_OK;
    int st = EVSL_OK;
    double *buf = (double *)ctx_ws(c, WS_BIS, sizeof(double) * (2 * (size_t)k + cnt + 8), &st);
    if (st) return st;
    double *dd = buf, *ee = buf + k, *ww = buf + 2 * k;
    cudaError_t e = cudaMemcpyAsync(dd, d_host, sizeof(double) * k, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ee, e_host, sizeof(double) * k, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "bisect upload");
    double emax = 1.0;
    for (int i = 0; i < k; i++) emax = std::max(emax, e_host[i] * e_host[i]);
    double pmin = 1e-290 * emax;
    ProfGroup g;
    prof_begin(c, EVSL_K_SMALL_EIG, &g);
    const size_t smem = sizeof(double) * 2 * (size_t)k;
    if (smem <= 200 * 1024) {
        // one warp per eigenvalue, four per block
        if (smem > 48 * 1024) {
            cudaError_t ea = cudaFuncSetAttribute(k_multisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (ea != cudaSuccess) return ctx_cuda(c, ea, "multisect smem");
        }
        k_multisect<<<(unsigned)((cnt + 3) / 4), 128, smem, c->stream>>>(k, l, dd, ee, k0, k1, lo, hi, pmin, ww);
    } else {
        const int tpb = std::max(1, std::min(32, (cnt + 4 * c->dev_sm_count - 1) / (4 * c->dev_sm_count)));
        k_bisect<<<nblk(cnt, tpb), tpb, 0, c->stream>>>(k, l, dd, ee, k0, k1, lo, hi, pmin, ww);
    }
    c->launches++;
    prof_end(c, &g, 1);
    EVSL_TRY(check_launch(c, "bisect"));
    e = cudaMemcpyAsync(w_host, ww, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "bisect readback");
    return EVSL_OK;
}
