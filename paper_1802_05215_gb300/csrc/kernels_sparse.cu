// Sparse kernels for sm_103a: sliced-ELLPACK upload, the fused Chebyshev filter step
// (SpMM + three-term recurrence + coefficient axpy, Eq. (2.4) with the mapping of Eq. (2.3)),
// the plain SpMV/SpMM, and the KPM moment step (Sec. 2.1) with in-kernel probe dots.
//
// Layout: one warp per 32-row slice, lane = row.  For a slice, value/column loads are
// contiguous across the warp (256 B of FP64 values, 128 B of indices per nonzero position),
// and the gathers x[col] of 32 consecutive rows of a stencil matrix are near-contiguous, so
// each pass over the matrix is one coalesced HBM stream with the vector reused from L2.
// For a block of nvec columns (column-major, ld = n) the row's nonzeros stay in registers
// and the columns are streamed, so the matrix is read once per step for all columns.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "evsl_internal.h"

namespace {

constexpr uint64_t SM_GOLDEN = 0x9E3779B97F4A7C15ull;
constexpr uint64_t SM_STREAM_MUL = 0xD1B54A32D192ED03ull;

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// key of a stream: first output of SplitMix64 seeded with seed ^ (stream * C)
__host__ __device__ __forceinline__ uint64_t sm_key(uint64_t seed, uint64_t stream)
{
    return sm_mix((seed ^ (stream * SM_STREAM_MUL)) + SM_GOLDEN);
}

// (k+1)-th output of SplitMix64 seeded with key
__device__ __forceinline__ uint64_t sm_draw(uint64_t key, uint64_t k)
{
    return sm_mix(key + (k + 1) * SM_GOLDEN);
}

constexpr int TPB = 256;  // threads per block for the warp-per-slice kernels
constexpr int WREG = 8;   // slice widths up to WREG keep their nonzeros in registers

template <typename V>
__global__ void k_sell_fill(int64_t n, int64_t nslices, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, const double *__restrict__ cv,
                            const int64_t *__restrict__ sptr, int32_t *__restrict__ col,
                            double *__restrict__ val, float *__restrict__ val32)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t s = r >> 5;
    if (s >= nslices) return;
    int lane = (int)(r & 31);
    int64_t base = sptr[s];
    int w = (int)((sptr[s + 1] - base) >> 5);
    int64_t b = 0, e = 0;
    if (r < n) { b = rp[r]; e = rp[r + 1]; }
    int32_t padc = (r < n) ? (int32_t)r : 0;
    if (e > b) padc = ci[e - 1];
    for (int j = 0; j < w; j++) {
        int64_t dst = base + (int64_t)j * 32 + lane;
        if (b + j < e) {
            col[dst] = ci[b + j];
            val[dst] = cv[b + j];
            val32[dst] = (float)cv[b + j];
        } else {
            col[dst] = padc;
            val[dst] = 0.0;
            val32[dst] = 0.0f;
        }
    }
}

// [cheb_step1 begin] -- source region fingerprinted by the profile summaries
// Fused Chebyshev step.  MODE 0: out = sc (A x - cc x); y = c0 x + cj out.
//                        MODE 1: out = sc (A x - cc x) - xprev; y += cj out.
//                        MODE 2: out = A x.
// Explicitly rounded arithmetic, so that every kernel variant (one vector, block, multi-slice)
// produces bitwise the same numbers for a column whatever the compiler's contraction choices.
__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_r(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_r(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double sub_r(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_r(float a, float b) { return __fsub_rn(a, b); }

// HAT: the values are the mapped (2/d)(A - c I), so acc is already 2 Ahat x.
template <typename T, int MODE, bool HAT>
__device__ __forceinline__ void cheb_epilogue(int64_t o, T acc, T xr, const T *xprev, T *out, T *y,
                                              T cc, T sc, T c0, T cj)
{
    if (MODE == 2) {
        out[o] = acc;
    } else {
        T wv;
        if (HAT)
            wv = (MODE == 0) ? mul_r(T(0.5), acc) : sub_r(acc, xprev[o]);
        else {
            wv = mul_r(fma_r(-cc, xr, acc), sc);
            if (MODE == 1) wv = sub_r(wv, xprev[o]);
        }
        out[o] = wv;
        if (MODE == 0)
            y[o] = fma_r(cj, wv, mul_r(c0, xr));
        else
            y[o] = fma_r(cj, wv, y[o]);
    }
}

// x[r] is needed by the unscaled recurrence and by the first step's y = c0 x + c1 w_1
template <int MODE, bool HAT>
constexpr bool needs_xr() { return MODE == 0 || (MODE == 1 && !HAT); }

// Single vector: each nonzero is used once, so nothing is cached in registers; the loop is
// unrolled so that several index loads and gathers are in flight per warp.
// STREAM: the matrix entries are read with the evict-first (streaming) policy.  When one step's
// bytes exceed L2, the entries (the bulk of them, not reused within a step) then leave room
// for the vectors (x, xprev, out, y), which the next step of the recurrence reads again.  When
// everything fits in L2 the normal policy keeps the matrix there too (the launcher decides).
template <typename T, int MODE, bool HAT, bool STREAM>
__global__ void __launch_bounds__(TPB)
k_cheb_step1(int64_t n, int64_t nslices, const int64_t *__restrict__ sptr,
             const int32_t *__restrict__ col, const T *__restrict__ val,
             const T *__restrict__ x, const T *xprev, T *out, T *y, T cc, T sc, T c0, T cj)
{
    int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (s >= nslices) return;
    int lane = threadIdx.x & 31;
    int64_t b0 = sptr[s];
    int w = (int)((sptr[s + 1] - b0) >> 5);
    const T *vp = val + b0 + lane;
    const int32_t *cp = col + b0 + lane;
    T acc = T(0);
#pragma unroll 4
    for (int j = 0; j < w; j++) {
        const T v = STREAM ? __ldcs(vp + 32 * j) : vp[32 * j];
        const int ci = STREAM ? __ldcs(cp + 32 * j) : cp[32 * j];
        acc = fma_r(v, __ldg(x + ci), acc);
    }
    int64_t r = s * 32 + lane;
    if (r < n)
        cheb_epilogue<T, MODE, HAT>(r, acc, needs_xr<MODE, HAT>() ? x[r] : T(0), xprev, out, y, cc, sc, c0, cj);
}

// [cheb_step1 end]

// Block of nvec columns (column-major, ld = n): the slice's nonzeros stay in registers and
// the columns are processed NC at a time so that NC * w gathers are in flight per warp.
// Warps are (slice, column group) pairs: with few slices the columns are split into ngroups
// contiguous groups of NC-column packs, so that enough warps run; each column's arithmetic
// is the same whatever the grouping.
// ctab/c0tab (optional, device): per-column coefficient of this degree and, in MODE 0, of
// degree 0 -- the multi-slice form, where every column carries its own filter.
template <typename T, int MODE, int NC, bool HAT>
__global__ void __launch_bounds__(TPB)
k_cheb_stepN(int64_t n, int64_t nslices, const int64_t *__restrict__ sptr,
             const int32_t *__restrict__ col, const T *__restrict__ val, int nvec, int ngroups,
             const T *__restrict__ x, const T *xprev, T *out, T *y, T cc, T sc, T c0, T cj,
             const T *__restrict__ ctab, const T *__restrict__ c0tab)
{
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (wid >= nslices * ngroups) return;
    const int64_t s = wid % nslices;
    const int grp = (int)(wid / nslices);
    const int npack = (nvec + NC - 1) / NC;
    const int lb = (int)((int64_t)grp * npack / ngroups) * NC;
    const int le = min((int)((int64_t)(grp + 1) * npack / ngroups) * NC, nvec);
    int lane = threadIdx.x & 31;
    int64_t base = sptr[s] + lane;
    int w = (int)((sptr[s + 1] - sptr[s]) >> 5);
    int64_t r = s * 32 + lane;
    T v[WREG];
    int c[WREG];
    const bool inreg = (w <= WREG);
#pragma unroll
    for (int j = 0; j < WREG; j++) {
        v[j] = (inreg && j < w) ? val[base + 32 * j] : T(0);
        c[j] = (inreg && j < w) ? col[base + 32 * j] : 0;
    }
    int l0 = lb;
    for (; l0 + NC <= le; l0 += NC) {
        T acc[NC];
#pragma unroll
        for (int q = 0; q < NC; q++) acc[q] = T(0);
        if (inreg) {
#pragma unroll
            for (int j = 0; j < WREG; j++)
                if (j < w)
#pragma unroll
                    for (int q = 0; q < NC; q++) acc[q] = fma_r(v[j], __ldg(x + (int64_t)(l0 + q) * n + c[j]), acc[q]);
        } else {
            for (int j = 0; j < w; j++) {
                T vj = val[base + 32 * j];
                int cj_ = col[base + 32 * j];
#pragma unroll
                for (int q = 0; q < NC; q++) acc[q] = fma_r(vj, __ldg(x + (int64_t)(l0 + q) * n + cj_), acc[q]);
            }
        }
        if (r < n) {
#pragma unroll
            for (int q = 0; q < NC; q++) {
                int64_t o = (int64_t)(l0 + q) * n + r;
                T cjq = ctab ? ctab[l0 + q] : cj, c0q = c0tab ? c0tab[l0 + q] : c0;
                cheb_epilogue<T, MODE, HAT>(o, acc[q], needs_xr<MODE, HAT>() ? x[o] : T(0), xprev, out, y, cc,
                                            sc, c0q, cjq);
            }
        }
    }
    for (; l0 < le; l0++) {
        const T *xl = x + (int64_t)l0 * n;
        T acc = T(0);
        if (inreg) {
#pragma unroll
            for (int j = 0; j < WREG; j++)
                if (j < w) acc = fma_r(v[j], __ldg(xl + c[j]), acc);
        } else {
            for (int j = 0; j < w; j++) acc = fma_r(val[base + 32 * j], __ldg(xl + col[base + 32 * j]), acc);
        }
        if (r < n) {
            int64_t o = (int64_t)l0 * n + r;
            T cjq = ctab ? ctab[l0] : cj, c0q = c0tab ? c0tab[l0] : c0;
            cheb_epilogue<T, MODE, HAT>(o, acc, needs_xr<MODE, HAT>() ? xl[r] : T(0), xprev, out, y, cc, sc,
                                        c0q, cjq);
        }
    }
}

// KPM block layout: row-major, row r holding its probe values contiguously with leading
// dimension ld = nvec rounded up to a multiple of 4 (the padding probes stay zero); the
// bit-packed signs are row-major too, bit (l % 32) of word bits[r * nw + l / 32] set <=>
// v_l[r] = -1.
template <typename T, int PPL> struct VecN;
template <> struct VecN<double, 2> { using type = double2; };
template <> struct VecN<float, 2> { using type = float2; };
template <> struct VecN<float, 4> { using type = float4; };

// KPM step: the same recurrence without y, plus the moment partial sums
// sum_l sum_r v_l[r] out_l[r].  One warp per 32-row slice, walking its rows; each lane covers
// PPL consecutive probes with one vector load (64 probes per pass), so a row takes 64 / PPL
// lanes and a warp works on 32 PPL / 64 rows at a time (FP64: PPL = 2, one row; FP32:
// PPL = 4, two rows), and every gathered neighbour row of the block is one coalesced load.
// The slice's matrix entries are loaded once per slice, one row per lane (coalesced, all in
// flight together), and handed to the lanes working on a row by warp shuffles, so the row loop
// waits only on the neighbour gathers; two row groups are processed per iteration to keep twice
// the gathers in flight.  Slices wider than WREG entries per row read their entries directly.
// Grid-stride over slices with a fixed grid so that the partials of one step fill exactly
// part[0..gridDim.x).  Each lane sums its share of one slice in the block's precision, row by
// row in ascending order, and adds it to an FP64 partial, so the sums across slices are FP64 in
// both precisions (FP64 issue is 1/64 of FP32 here).
// DBL (the moment-doubling form): instead of the probe-weighted sum the step accumulates
// sum out.x_row (w_{k+1}^T w_k, into part) and sum out.out (||w_{k+1}||^2, into part2).
template <typename T, bool HAT, int PPL, bool DBL>
__device__ __forceinline__ void kpm_row_epilogue(int mode, int64_t r, int l, int nvec, int ld, int nw,
                                                 const uint32_t *__restrict__ bits, const T *__restrict__ x,
                                                 const T *xprev, T *out, T cc, T sc, const T (&a)[PPL],
                                                 T &smom, T &smom2)
{
    using VL = typename VecN<T, PPL>::type;
    const int64_t o = r * ld + l;
    T w[PPL], pv[PPL];
    if (mode == 1) *reinterpret_cast<VL *>(pv) = *reinterpret_cast<const VL *>(xprev + o);
    if (HAT) {
#pragma unroll
        for (int q = 0; q < PPL; q++) w[q] = (mode == 1) ? a[q] - pv[q] : T(0.5) * a[q];
    } else {
        T xo[PPL];
        *reinterpret_cast<VL *>(xo) = *reinterpret_cast<const VL *>(x + o);
#pragma unroll
        for (int q = 0; q < PPL; q++) {
            w[q] = (a[q] - cc * xo[q]) * sc;
            if (mode == 1) w[q] -= pv[q];
        }
    }
    *reinterpret_cast<VL *>(out + o) = *reinterpret_cast<const VL *>(w);
    if (DBL) {
        T xr[PPL];
        *reinterpret_cast<VL *>(xr) = *reinterpret_cast<const VL *>(x + o);
#pragma unroll
        for (int q = 0; q < PPL; q++) {
            smom += w[q] * xr[q];     // padding probes are zero on both sides
            smom2 += w[q] * w[q];
        }
    } else {
        const uint32_t word = bits[r * nw + (l >> 5)];
        const int b = l & 31;
#pragma unroll
        for (int q = 0; q < PPL; q++)
            if (l + q < nvec) smom += ((word >> (b + q)) & 1u) ? -w[q] : w[q];
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Per-warp staging buffer of one slice (slices up to WREG entries wide): entries and columns
// in the slice's own column-major order, and the 32 row lengths.
struct KpmStage {
    float val[WREG * 32];
    int32_t col[WREG * 32];
    int32_t len[32];
};

// Copies slice s's entries (w <= WREG per row, 128 w bytes per array) and row lengths into st
// with 16-byte asynchronous copies; sptr/val/col/rlen slices are 128-byte aligned.
__device__ __forceinline__ void kpm_stage_issue(KpmStage &st, int64_t sbase, int w, int64_t s, int lane,
                                                const float *__restrict__ val, const int32_t *__restrict__ col,
                                                const int32_t *__restrict__ rlen)
{
    const int chunks = 8 * w;  // 16-byte pieces per array
    for (int c = lane; c < chunks; c += 32) {
        cp_async16(&st.val[4 * c], val + sbase + 4 * c);
        cp_async16(&st.col[4 * c], col + sbase + 4 * c);
    }
    if (lane < 8) cp_async16(&st.len[4 * lane], rlen + s * 32 + 4 * lane);
    cp_async_commit();
}

template <typename T, bool HAT, int PPL, bool DBL>
__global__ void __launch_bounds__(TPB, 4)
k_kpm_step(int mode, int64_t n, int64_t nslices, const int64_t *__restrict__ sptr,
           const int32_t *__restrict__ col, const T *__restrict__ val, const int32_t *__restrict__ rlen,
           int nvec, int ld, const uint32_t *__restrict__ bits, const T *__restrict__ x, const T *xprev,
           T *out, T cc, T sc, double *__restrict__ part, double *__restrict__ part2)
{
    using VL = typename VecN<T, PPL>::type;
    constexpr int LPR = 64 / PPL;   // lanes per row
    constexpr int RPI = 32 / LPR;   // rows per warp at a time
    constexpr int WPB = TPB / 32;
    __shared__ double red[WPB], red2[WPB];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int sub = lane % LPR, rsub = lane / LPR;
    const int nw = (nvec + 31) >> 5;
    double mom = 0.0, mom2 = 0.0;
    // FP32 with mapped values: each warp stages its next slice's entries in shared memory while
    // it works on the current one.  Slices are taken grid-stride, so the warps of the whole grid
    // work on one contiguous band of rows at a time and a neighbour row far away in the ordering
    // (the +-nx^2 planes of a 3-D stencil) is read by the bands before and after it while it is
    // still in L2; a contiguous range per block would spread the concurrent rows over the whole
    // matrix and read such rows from HBM again.
    constexpr bool STAGED = (sizeof(T) == 4) && HAT && (PPL == 4);
    if constexpr (STAGED) {
        __shared__ __align__(16) KpmStage stage[WPB][2];
        const int64_t gstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
        const int64_t s_end = nslices;
        int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        int buf = 0;
        // the first slice; a slice wider than WREG is handled directly (flagged by w_cur)
        int64_t sb_cur = 0;
        int w_cur = 0;
        if (s < s_end) {
            sb_cur = sptr[s];
            w_cur = (int)((sptr[s + 1] - sb_cur) >> 5);
            if (w_cur <= WREG) kpm_stage_issue(stage[wib][0], sb_cur, w_cur, s, lane, (const float *)val, col, rlen);
        }
        for (; s < s_end; s += gstride) {
            const int64_t sn = s + gstride;
            int64_t sb_next = 0;
            int w_next = 0;
            if (sn < s_end) {
                sb_next = sptr[sn];
                w_next = (int)((sptr[sn + 1] - sb_next) >> 5);
            }
            const bool staged_next = sn < s_end && w_next <= WREG;
            if (staged_next)
                kpm_stage_issue(stage[wib][buf ^ 1], sb_next, w_next, sn, lane, (const float *)val, col, rlen);
            if (staged_next) cp_async_wait<1>();
            else cp_async_wait<0>();
            __syncwarp();
            T smom = T(0), smom2 = T(0);
            if (w_cur <= WREG) {
                const KpmStage &st = stage[wib][buf];
                for (int rr0 = 0; rr0 < 32; rr0 += 2 * RPI) {
                    const int rA = rr0 + rsub, rB = rr0 + RPI + rsub;
                    const int64_t gA = s * 32 + rA, gB = s * 32 + rB;
                    const int lenA = st.len[rA], lenB = st.len[rB];
                    for (int l0 = 0; l0 < nvec; l0 += 64) {
                        const int l = l0 + PPL * sub;
                        const bool actA = (gA < n) && (l < nvec), actB = (gB < n) && (l < nvec);
                        const int64_t oA = gA * ld + l, oB = gB * ld + l;
                        // the rows' own operands first: out may alias xprev, so these loads
                        // must precede this iteration's stores
                        T pA[PPL], pB[PPL];
                        uint32_t wdA = 0, wdB = 0;
                        if (mode == 1 && actA) *reinterpret_cast<VL *>(pA) = *reinterpret_cast<const VL *>(xprev + oA);
                        if (mode == 1 && actB) *reinterpret_cast<VL *>(pB) = *reinterpret_cast<const VL *>(xprev + oB);
                        if (!DBL && actA) wdA = bits[gA * nw + (l >> 5)];
                        if (!DBL && actB) wdB = bits[gB * nw + (l >> 5)];
                        T aA[PPL], aB[PPL];
#pragma unroll
                        for (int q = 0; q < PPL; q++) aA[q] = aB[q] = T(0);
#pragma unroll
                        for (int j = 0; j < WREG; j++)
                            if (j < w_cur) {
                                const int cA = st.col[32 * j + rA], cB = st.col[32 * j + rB];
                                const T vA = st.val[32 * j + rA], vB = st.val[32 * j + rB];
                                T xa[PPL], xb[PPL];
                                const bool ua = actA && j < lenA, ub = actB && j < lenB;
                                if (ua) *reinterpret_cast<VL *>(xa) = __ldg(reinterpret_cast<const VL *>(x + (int64_t)cA * ld + l));
                                if (ub) *reinterpret_cast<VL *>(xb) = __ldg(reinterpret_cast<const VL *>(x + (int64_t)cB * ld + l));
                                if (ua)
#pragma unroll
                                    for (int q = 0; q < PPL; q++) aA[q] += vA * xa[q];
                                if (ub)
#pragma unroll
                                    for (int q = 0; q < PPL; q++) aB[q] += vB * xb[q];
                            }
#pragma unroll
                        for (int h = 0; h < 2; h++) {
                            const bool act = h ? actB : actA;
                            if (!act) continue;
                            const T *a = h ? aB : aA;
                            const T *pv = h ? pB : pA;
                            const uint32_t word = h ? wdB : wdA;
                            T wv[PPL];
#pragma unroll
                            for (int q = 0; q < PPL; q++) wv[q] = (mode == 1) ? a[q] - pv[q] : T(0.5) * a[q];
                            *reinterpret_cast<VL *>(out + (h ? oB : oA)) = *reinterpret_cast<const VL *>(wv);
                            if (DBL) {
                                T xo[PPL];   // x is read-only and never aliased by out
                                *reinterpret_cast<VL *>(xo) = *reinterpret_cast<const VL *>(x + (h ? oB : oA));
#pragma unroll
                                for (int q = 0; q < PPL; q++) {
                                    smom += wv[q] * xo[q];
                                    smom2 += wv[q] * wv[q];
                                }
                            } else {
                                const int b = l & 31;
#pragma unroll
                                for (int q = 0; q < PPL; q++)
                                    if (l + q < nvec) smom += ((word >> (b + q)) & 1u) ? -wv[q] : wv[q];
                            }
                        }
                    }
                }
            } else {
                for (int rr0 = 0; rr0 < 32; rr0 += RPI) {
                    const int rr = rr0 + rsub;
                    const int64_t r = s * 32 + rr;
                    const int len = (r < n) ? rlen[r] : 0;
                    for (int l0 = 0; l0 < nvec; l0 += 64) {
                        const int l = l0 + PPL * sub;
                        const bool act = (r < n) && (l < nvec);
                        T a[PPL];
#pragma unroll
                        for (int q = 0; q < PPL; q++) a[q] = T(0);
                        for (int j = 0; j < len; j++) {
                            const int64_t e = sb_cur + 32 * (int64_t)j + rr;
                            const T v = val[e];
                            const int cj = col[e];
                            if (act) {
                                T xv[PPL];
                                *reinterpret_cast<VL *>(xv) = __ldg(reinterpret_cast<const VL *>(x + (int64_t)cj * ld + l));
#pragma unroll
                                for (int q = 0; q < PPL; q++) a[q] += v * xv[q];
                            }
                        }
                        if (act)
                            kpm_row_epilogue<T, HAT, PPL, DBL>(mode, r, l, nvec, ld, nw, bits, x, xprev, out, cc, sc, a,
                                                              smom, smom2);
                    }
                }
            }
            mom += (double)smom;
            mom2 += (double)smom2;
            __syncwarp();            // the buffer just read is the next copy's target
            buf ^= 1;
            sb_cur = sb_next;
            w_cur = w_next;
        }
    } else {
        const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
        for (int64_t s = warp; s < nslices; s += nwarps) {
            const int64_t sbase = sptr[s];
            T smom = T(0), smom2 = T(0);  // this lane's share of the slice, in the block's precision
            for (int rr0 = 0; rr0 < 32; rr0 += RPI) {
                const int rr = rr0 + rsub;
                const int64_t r = s * 32 + rr;
                const int len = (r < n) ? rlen[r] : 0;
                for (int l0 = 0; l0 < nvec; l0 += 64) {
                    const int l = l0 + PPL * sub;
                    const bool act = (r < n) && (l < nvec);
                    T a[PPL];
#pragma unroll
                    for (int q = 0; q < PPL; q++) a[q] = T(0);
                    if (len <= WREG) {
#pragma unroll
                        for (int j = 0; j < WREG; j++)
                            if (j < len) {
                                const int64_t e = sbase + 32 * (int64_t)j + rr;
                                const T v = val[e];
                                const int cj = col[e];
                                if (act) {
                                    T xv[PPL];
                                    *reinterpret_cast<VL *>(xv) = __ldg(reinterpret_cast<const VL *>(x + (int64_t)cj * ld + l));
#pragma unroll
                                    for (int q = 0; q < PPL; q++) a[q] += v * xv[q];
                                }
                            }
                    } else {
                        for (int j = 0; j < len; j++) {
                            const int64_t e = sbase + 32 * (int64_t)j + rr;
                            const T v = val[e];
                            const int cj = col[e];
                            if (act) {
                                T xv[PPL];
                                *reinterpret_cast<VL *>(xv) = __ldg(reinterpret_cast<const VL *>(x + (int64_t)cj * ld + l));
#pragma unroll
                                for (int q = 0; q < PPL; q++) a[q] += v * xv[q];
                            }
                        }
                    }
                    if (act)
                        kpm_row_epilogue<T, HAT, PPL, DBL>(mode, r, l, nvec, ld, nw, bits, x, xprev, out, cc, sc, a,
                                                          smom, smom2);
                }
            }
            mom += (double)smom;
            mom2 += (double)smom2;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mom += __shfl_xor_sync(0xffffffffu, mom, off);
        if (DBL) mom2 += __shfl_xor_sync(0xffffffffu, mom2, off);
    }
    if (lane == 0) {
        red[wib] = mom;
        red2[wib] = mom2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, t2 = 0.0;
        for (int i = 0; i < WPB; i++) {
            t += red[i];
            t2 += red2[i];
        }
        part[blockIdx.x] = t;
        if (DBL) part2[blockIdx.x] = t2;
    }
}

// Probes in the row-major layout: W0[r * ld + l] = sign of draw(seed, KPM, l * n + r) for
// l < nvec, 0 for the padding probes; one warp builds one sign word of one row.
template <typename T>
__global__ void k_kpm_init(int64_t n, int nvec, int ld, uint64_t key, uint64_t first, T *W0, uint32_t *bits)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int nw = (nvec + 31) >> 5;
    const int64_t total = n * nw * 32;
    if (t >= total) return;  // whole warps exit together: total is a multiple of 32
    const int64_t r = t / (nw * 32);
    const int l = (int)(t - r * nw * 32);
    bool neg = false;
    if (l < nvec) {
        uint64_t v = sm_draw(key, (first + (uint64_t)l) * (uint64_t)n + (uint64_t)r);
        neg = (v >> 63) != 0;
    }
    if (l < ld) W0[r * ld + l] = (l < nvec) ? (neg ? T(-1) : T(1)) : T(0);
    uint32_t word = __ballot_sync(0xffffffffu, neg);
    if ((threadIdx.x & 31) == 0) bits[r * nw + (l >> 5)] = word;
}

__global__ void k_f64_to_f32(int64_t count, const double *__restrict__ x, float *__restrict__ y)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) y[i] = (float)x[i];
}

__global__ void k_f32_to_f64(int64_t count, const float *__restrict__ x, double *__restrict__ y)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) y[i] = (double)x[i];
}

// uniform(-1, 1) from draw(seed, stream, index*n + i)
__global__ void k_fill_uniform(int64_t n, uint64_t key, uint64_t index, double *x)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        uint64_t v = sm_draw(key, index * (uint64_t)n + (uint64_t)i);
        x[i] = 2.0 * ((double)(v >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
}

// +-1 from the top bit of draw(key, index*n + i): probe `index` of the KPM convention
__global__ void k_fill_sign(int64_t n, uint64_t key, uint64_t index, double *x)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = (sm_draw(key, index * (uint64_t)n + (uint64_t)i) >> 63) ? -1.0 : 1.0;
}

inline unsigned blocks_for(int64_t threads, int tpb) { return (unsigned)((threads + tpb - 1) / tpb); }

}  // namespace

// ------------------------------------------------------------------------------------------
// Builds the sliced-ELLPACK copy of a CSR matrix in M.  primary: M is the context's operator
// A (its cached graphs and tile choices are dropped with it); otherwise M is a second matrix
// (the mass matrix B of a generalized problem).  The old M survives a failed validation.
static int sell_build(evsl_ctx *c, DevMatrix &M, bool primary, const char *what, int64_t n,
                      const int64_t *rp, const int32_t *ci, const double *cv)
{
    auto release = [&]() {
        if (primary) sell_free(c);
        else dev_matrix_free(c, M);
    };
    if (n < 1 || !rp || !ci || !cv) return ctx_fail(c, EVSL_ERR_ARG, "%s: bad arguments", what);
    if (rp[0] != 0) return ctx_fail(c, EVSL_ERR_ARG, "%s: row_ptr[0] != 0", what);
    int64_t nnz = rp[n];
    if (nnz < 1 || nnz >= (int64_t(1) << 31))
        return ctx_fail(c, EVSL_ERR_ARG, "%s: nnz %lld out of range", what, (long long)nnz);
    int64_t nslices = (n + 31) / 32;
    std::vector<int64_t> sptr(nslices + 1);
    sptr[0] = 0;
    int maxw = 0;
    for (int64_t s = 0; s < nslices; s++) {
        int w = 0;
        for (int64_t r = s * 32; r < std::min(n, s * 32 + 32); r++) {
            int64_t len = rp[r + 1] - rp[r];
            if (len < 0) return ctx_fail(c, EVSL_ERR_ARG, "%s: row_ptr decreases at %lld", what, (long long)r);
            if (len > w) w = (int)len;
        }
        if (w > maxw) maxw = w;
        sptr[s + 1] = sptr[s] + 32 * (int64_t)w;
    }
    for (int64_t p = 0; p < nnz; p++)
        if (ci[p] < 0 || ci[p] >= n)
            return ctx_fail(c, EVSL_ERR_ARG, "%s: column index %d out of range at %lld", what, ci[p], (long long)p);
    std::vector<int32_t> rlen(nslices * 32, 0);   // padded to whole slices: rows past n have length 0
    bool has_diag = true;
    for (int64_t r = 0; r < n; r++) {
        rlen[r] = (int32_t)(rp[r + 1] - rp[r]);
        bool found = false;
        for (int64_t p = rp[r]; p < rp[r + 1] && !found; p++) found = (ci[p] == r);
        has_diag = has_diag && found;
    }
    release();
    DevMatrix &A = M;
    int64_t ns = sptr[nslices];
    int64_t *d_rp = nullptr;
    int32_t *d_ci = nullptr;
    double *d_cv = nullptr;
    int st = EVSL_OK;
    // sizes first, so that a failed allocation releases what was taken with the right sizes
    A.n = n;
    A.nslices = nslices;
    A.nstored = ns;
    if ((st = ctx_alloc(c, (void **)&A.sptr, sizeof(int64_t) * (nslices + 1))) ||
        (st = ctx_alloc(c, (void **)&A.col, sizeof(int32_t) * ns)) ||
        (st = ctx_alloc(c, (void **)&A.val, sizeof(double) * ns)) ||
        (st = ctx_alloc(c, (void **)&A.val32, sizeof(float) * ns)) ||
        (st = ctx_alloc(c, (void **)&A.rlen, sizeof(int32_t) * nslices * 32))) {
        release();
        return st;
    }
    A.has_diag = has_diag;
    A.nnz = nnz;
    A.maxw = maxw;
    if ((st = ctx_alloc(c, (void **)&d_rp, sizeof(int64_t) * (n + 1))) ||
        (st = ctx_alloc(c, (void **)&d_ci, sizeof(int32_t) * nnz)) ||
        (st = ctx_alloc(c, (void **)&d_cv, sizeof(double) * nnz))) {
        ctx_free(c, d_rp, sizeof(int64_t) * (n + 1));
        ctx_free(c, d_ci, sizeof(int32_t) * nnz);
        release();
        return st;
    }
    cudaStream_t s = c->stream;
    cudaError_t e = cudaMemcpyAsync(A.sptr, sptr.data(), sizeof(int64_t) * (nslices + 1),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rp, rp, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ci, ci, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cv, cv, sizeof(double) * nnz, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(A.rlen, rlen.data(), sizeof(int32_t) * nslices * 32, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_sell_fill<double><<<blocks_for(nslices * 32, 256), 256, 0, s>>>(n, nslices, d_rp, d_ci, d_cv,
                                                                          A.sptr, A.col, A.val, A.val32);
        c->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ctx_free(c, d_rp, sizeof(int64_t) * (n + 1));
    ctx_free(c, d_ci, sizeof(int32_t) * nnz);
    ctx_free(c, d_cv, sizeof(double) * nnz);
    if (e != cudaSuccess) {
        release();
        return ctx_cuda(c, e, what);
    }
    return EVSL_OK;
}

int sell_upload(evsl_ctx *c, int64_t n, const int64_t *rp, const int32_t *ci, const double *cv)
{
    return sell_build(c, c->A, true, "set_csr", n, rp, ci, cv);
}

int sell_upload_b(evsl_ctx *c, int64_t n, const int64_t *rp, const int32_t *ci, const double *cv)
{
    return sell_build(c, c->B, false, "set_csr_b", n, rp, ci, cv);
}

void sell_free(evsl_ctx *c)
{
    filter_graphs_clear(c);
    c->tune.clear();
    dev_matrix_free(c, c->A);
}

void dev_matrix_free(evsl_ctx *c, DevMatrix &A)
{
    ctx_free(c, A.sptr, sizeof(int64_t) * (A.nslices + 1));
    ctx_free(c, A.col, sizeof(int32_t) * A.nstored);
    ctx_free(c, A.val, sizeof(double) * A.nstored);
    ctx_free(c, A.val32, sizeof(float) * A.nstored);
    ctx_free(c, A.rlen, sizeof(int32_t) * A.nslices * 32);
    ctx_free(c, A.vhat, sizeof(double) * A.nstored);
    ctx_free(c, A.vhat32, sizeof(float) * A.nstored);
    A = DevMatrix();
}

// Tile shapes of the multi-column step: NC columns per warp pass (the gathers in flight per
// warp) and a multiplier on the number of column groups (the warps per slice).  The autotuner
// (tune_cheb_block) picks one per (matrix, column count, precision); every shape computes each
// column with the same operations in the same order.
struct ChebTile {
    int nc, gmul;
};
constexpr ChebTile TILES_F64[] = {{2, 1}, {1, 1}, {4, 1}, {2, 2}, {4, 2}};
constexpr ChebTile TILES_F32[] = {{4, 1}, {2, 1}, {8, 1}, {4, 2}, {8, 2}};
constexpr int NTILES = 5;

template <typename T, int MODE, int NC, bool HAT>
static void launch_stepN(evsl_ctx *c, int gmul, int nvec, const T *val, const T *x, const T *xprev, T *out,
                         T *y, T cc, T sc, T c0, T cj, const T *ctab, const T *c0tab)
{
    const DevMatrix &A = c->A;
    // (slice, column group) warps: about 64 warps per SM, times the tile's multiplier
    const int npack = (nvec + NC - 1) / NC;
    const int64_t want = (int64_t)c->dev_sm_count * 64 * gmul;
    const int ngroups = (int)std::max<int64_t>(1, std::min<int64_t>(npack, (want + A.nslices - 1) / A.nslices));
    const unsigned g2 = blocks_for(A.nslices * 32 * (int64_t)ngroups, TPB);
    k_cheb_stepN<T, MODE, NC, HAT><<<g2, TPB, 0, c->stream>>>(A.n, A.nslices, A.sptr, A.col, val, nvec, ngroups,
                                                             x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
}

template <typename T>
static ChebTile current_tile(evsl_ctx *c, int nvec)
{
    const int t = tune_lookup(c, nvec, sizeof(T));
    return sizeof(T) == 8 ? TILES_F64[t] : TILES_F32[t];
}

// Whether one single-vector step's bytes (matrix entries, row offsets, five vector streams)
// exceed half of L2, so that the matrix is better streamed evict-first (k_cheb_step1).
bool stream_matrix(const evsl_ctx *c, int64_t nstored, int64_t n, int value_bytes)
{
    const double step = (double)nstored * (value_bytes + 4) + 8.0 * (n + 1) + 5.0 * n * value_bytes;
    return c->l2_bytes > 0 && step > 0.5 * (double)c->l2_bytes;
}

template <typename T, int MODE, bool HAT>
static void launch_cheb(evsl_ctx *c, unsigned grid, int nvec, const T *val, const T *x, const T *xprev,
                        T *out, T *y, T cc, T sc, T c0, T cj, const T *ctab, const T *c0tab)
{
    const DevMatrix &A = c->A;
    if (nvec == 1 && !ctab) {
        if (stream_matrix(c, A.nstored, A.n, (int)sizeof(T)))
            k_cheb_step1<T, MODE, HAT, true><<<grid, TPB, 0, c->stream>>>(A.n, A.nslices, A.sptr, A.col, val, x,
                                                                         xprev, out, y, cc, sc, c0, cj);
        else
            k_cheb_step1<T, MODE, HAT, false><<<grid, TPB, 0, c->stream>>>(A.n, A.nslices, A.sptr, A.col, val, x,
                                                                          xprev, out, y, cc, sc, c0, cj);
        return;
    }
    const ChebTile tl = current_tile<T>(c, nvec);
    if constexpr (sizeof(T) == 8) {
        if (tl.nc == 1)
            launch_stepN<T, MODE, 1, HAT>(c, tl.gmul, nvec, val, x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
        else if (tl.nc == 4)
            launch_stepN<T, MODE, 4, HAT>(c, tl.gmul, nvec, val, x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
        else
            launch_stepN<T, MODE, 2, HAT>(c, tl.gmul, nvec, val, x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
    } else {
        if (tl.nc == 2)
            launch_stepN<T, MODE, 2, HAT>(c, tl.gmul, nvec, val, x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
        else if (tl.nc == 8)
            launch_stepN<T, MODE, 8, HAT>(c, tl.gmul, nvec, val, x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
        else
            launch_stepN<T, MODE, 4, HAT>(c, tl.gmul, nvec, val, x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
    }
}

template <typename T, bool HAT>
static void launch_cheb_mode(evsl_ctx *c, int mode, unsigned grid, int nvec, const T *val, const T *x,
                             const T *xprev, T *out, T *y, T cc, T sc, T c0, T cj, const T *ctab,
                             const T *c0tab)
{
    if (mode == 0)
        launch_cheb<T, 0, HAT>(c, grid, nvec, val, x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
    else if (mode == 1)
        launch_cheb<T, 1, HAT>(c, grid, nvec, val, x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
    else
        launch_cheb<T, 2, HAT>(c, grid, nvec, val, x, xprev, out, y, cc, sc, c0, cj, ctab, c0tab);
}

// hat: use the mapped values (2/d)(A - cc I), made current by the caller with ensure_mapped
template <typename T>
static int cheb_step_t(evsl_ctx *c, int mode, int nvec, const T *x, const T *xprev, T *out,
                       T *y, double cc, double sc, double c0, double cj, const T *val, bool hat,
                       const T *ctab = nullptr, const T *c0tab = nullptr)
{
    const DevMatrix &A = c->A;
    unsigned grid = blocks_for(A.nslices * 32, TPB);
    T tcc = (T)cc, tsc = (T)sc, tc0 = (T)c0, tcj = (T)cj;
    hat = hat && mode != 2 && A.vhat;
    if (hat) {
        const T *hv = sizeof(T) == 8 ? (const T *)A.vhat : (const T *)A.vhat32;
        launch_cheb_mode<T, true>(c, mode, grid, nvec, hv, x, xprev, out, y, tcc, tsc, tc0, tcj, ctab, c0tab);
    } else {
        launch_cheb_mode<T, false>(c, mode, grid, nvec, val, x, xprev, out, y, tcc, tsc, tc0, tcj, ctab, c0tab);
    }
    c->launches++;
    return check_launch(c, "cheb_step");
}

int cheb_step_multi_f64(evsl_ctx *c, int mode, int nvec, const double *x, const double *xprev,
                        double *out, double *y, double cc, double sc, const double *ctab,
                        const double *c0tab, bool hat)
{
    return cheb_step_t<double>(c, mode, nvec, x, xprev, out, y, cc, sc, 0.0, 0.0, c->A.val, hat, ctab, c0tab);
}

int cheb_step_multi_f32(evsl_ctx *c, int mode, int nvec, const float *x, const float *xprev,
                        float *out, float *y, double cc, double sc, const float *ctab,
                        const float *c0tab, bool hat)
{
    return cheb_step_t<float>(c, mode, nvec, x, xprev, out, y, cc, sc, 0.0, 0.0, c->A.val32, hat, ctab, c0tab);
}

// mapped values (2/d)(A - cc I): padding entries stay zero
__global__ void k_make_mapped(int64_t n, int64_t nslices, const int64_t *__restrict__ sptr,
                              const int32_t *__restrict__ col, const double *__restrict__ val,
                              const int32_t *__restrict__ rlen, double cc, double sc, double *__restrict__ vhat,
                              float *__restrict__ vhat32)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t s = r >> 5;
    if (s >= nslices) return;
    int lane = (int)(r & 31);
    int64_t base = sptr[s] + lane;
    int w = (int)((sptr[s + 1] - sptr[s]) >> 5);
    int len = (r < n) ? rlen[r] : 0;
    for (int j = 0; j < w; j++) {
        int64_t e = base + 32 * (int64_t)j;
        double v = 0.0;
        if (j < len) {
            v = val[e];
            if (col[e] == r) v -= cc;
            v *= sc;
        }
        vhat[e] = v;
        vhat32[e] = (float)v;
    }
}

bool ensure_mapped(evsl_ctx *c, double cc, double d, int *status)
{
    DevMatrix &A = c->A;
    if (!A.has_diag || A.n == 0) return false;
    if (A.vhat && A.hat_c == cc && A.hat_d == d) return true;
    if (!A.vhat) {
        int st = ctx_alloc(c, (void **)&A.vhat, sizeof(double) * A.nstored);
        if (st == EVSL_OK) st = ctx_alloc(c, (void **)&A.vhat32, sizeof(float) * A.nstored);
        if (st != EVSL_OK) {
            // not enough room for the mapped copy: the unscaled kernels still work
            ctx_free(c, A.vhat, sizeof(double) * A.nstored);
            A.vhat = nullptr;
            A.vhat32 = nullptr;
            c->err.clear();
            return false;
        }
    }
    k_make_mapped<<<blocks_for(A.nslices * 32, 256), 256, 0, c->stream>>>(A.n, A.nslices, A.sptr, A.col, A.val,
                                                                         A.rlen, cc, 2.0 / d, A.vhat, A.vhat32);
    c->launches++;
    int st = check_launch(c, "make_mapped");
    if (st != EVSL_OK) {
        *status = st;
        return false;
    }
    A.hat_c = cc;
    A.hat_d = d;
    return true;
}

int cheb_step_f64(evsl_ctx *c, int mode, int nvec, const double *x, const double *xprev,
                  double *out, double *y, double cc, double sc, double c0, double cj, bool hat)
{
    return cheb_step_t<double>(c, mode, nvec, x, xprev, out, y, cc, sc, c0, cj, c->A.val, hat);
}

int cheb_step_f32(evsl_ctx *c, int mode, int nvec, const float *x, const float *xprev,
                  float *out, float *y, double cc, double sc, double c0, double cj, bool hat)
{
    return cheb_step_t<float>(c, mode, nvec, x, xprev, out, y, cc, sc, c0, cj, c->A.val32, hat);
}

int spmv_f64(evsl_ctx *c, int nvec, const double *X, double *Y)
{
    return cheb_step_t<double>(c, 2, nvec, X, nullptr, Y, nullptr, 0.0, 1.0, 0.0, 0.0, c->A.val, false);
}

// ------------------------------------------------------------------------------------------
// Autotuner of the multi-column filter step.  For a (matrix, column count, precision) seen for
// the first time, every tile shape runs the plain block SpMV (mode 2) on the caller's block
// into a scratch block: one untimed launch, then three timed with CUDA events; the fastest is
// kept in the context (cleared when the matrix changes).  Must not run while the stream is
// being captured.
// column counts are bucketed by powers of two; a count whose bucket has not been timed uses
// the nearest timed bucket above it (the batch's full width), else the default shape
static int tune_bucket(int nvec)
{
    int b = 1;
    while (b < nvec && b < (1 << 20)) b <<= 1;
    return b;
}

static uint64_t tune_key(int64_t n, int bucket, int bytes)
{
    return ((uint64_t)n << 24) ^ ((uint64_t)bucket << 4) ^ (uint64_t)bytes;
}

int tune_lookup(evsl_ctx *c, int nvec, int bytes)
{
    if (c->tune.empty()) return 0;
    for (int b = tune_bucket(nvec); b <= (1 << 20); b <<= 1) {
        auto it = c->tune.find(tune_key(c->A.n, b, bytes));
        if (it != c->tune.end()) return it->second;
    }
    return 0;
}

template <typename T>
static int tune_block_t(evsl_ctx *c, int nvec, const T *X, const T *val)
{
    const uint64_t key = tune_key(c->A.n, tune_bucket(nvec), sizeof(T));
    if (c->tune.count(key)) return EVSL_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return EVSL_OK;  // the caller is capturing: keep the default shape, time nothing
    }
    int st = EVSL_OK;
    T *scratch = (T *)ctx_ws(c, WS_TUNE, sizeof(T) * c->A.n * (size_t)nvec, &st);
    if (st) return st;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return ctx_cuda(c, cudaGetLastError(), "tune event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ctx_cuda(c, cudaGetLastError(), "tune event");
    }
    int best = 0;
    float best_ms = 1e30f;
    float times[NTILES] = {0};
    for (int t = 0; t < NTILES && st == EVSL_OK; t++) {
        c->tune[key] = t;
        for (int rep = 0; rep < 4 && st == EVSL_OK; rep++) {
            if (rep == 1) cudaEventRecord(e0, c->stream);
            launch_cheb<T, 2, false>(c, 0, nvec, val, X, nullptr, scratch, nullptr, T(0), T(1), T(0), T(0), nullptr,
                                     nullptr);
            c->launches++;
            st = check_launch(c, "tune");
        }
        cudaEventRecord(e1, c->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) st = ctx_cuda(c, e, "tune");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        times[t] = ms / 3.0f;
        if (st == EVSL_OK && ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune[key] = best;
    const char *venv = getenv("EVSL_VERBOSE");
    if (venv && venv[0] == '1') {
        const ChebTile *tl = sizeof(T) == 8 ? TILES_F64 : TILES_F32;
        fprintf(stderr, "[evsl] tune %s n=%lld columns<=%d:", sizeof(T) == 8 ? "fp64" : "fp32",
                (long long)c->A.n, tune_bucket(nvec));
        for (int t = 0; t < NTILES; t++) fprintf(stderr, " (nc %d, x%d) %.1f us", tl[t].nc, tl[t].gmul, times[t] * 1e3f);
        fprintf(stderr, " -> (nc %d, x%d)\n", tl[best].nc, tl[best].gmul);
    }
    return st;
}

int tune_block_f64(evsl_ctx *c, int nvec, const double *X)
{
    if (nvec < 2) return EVSL_OK;
    return tune_block_t<double>(c, nvec, X, c->A.val);
}

int tune_block_f32(evsl_ctx *c, int nvec, const float *X)
{
    if (nvec < 2) return EVSL_OK;
    return tune_block_t<float>(c, nvec, X, c->A.val32);
}

int kpm_nblocks(evsl_ctx *c)
{
    // one wave: the KPM step keeps 4 blocks of TPB threads resident per SM (64 registers)
    int64_t need = (c->A.nslices * 32 + TPB - 1) / TPB;
    int64_t cap = (int64_t)c->dev_sm_count * 4;
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

int kpm_ld(int nvec) { return (nvec + 3) & ~3; }

static uint32_t *kpm_bits(evsl_ctx *c, int nvec, int *st)
{
    const int nw = (nvec + 31) >> 5;
    return (uint32_t *)ctx_ws(c, WS_TMP_STAGE, sizeof(uint32_t) * c->A.n * nw, st);
}

template <typename T>
static int kpm_init_t(evsl_ctx *c, int nvec, uint64_t seed, T *W0, uint64_t first = 0)
{
    int st = EVSL_OK;
    uint32_t *bits = kpm_bits(c, nvec, &st);
    if (st) return st;
    const int64_t total = c->A.n * (int64_t)(((nvec + 31) >> 5) * 32);
    k_kpm_init<T><<<blocks_for(total, 256), 256, 0, c->stream>>>(c->A.n, nvec, kpm_ld(nvec),
                                                                 sm_key(seed, SM_STREAM_KPM), first, W0, bits);
    c->launches++;
    return check_launch(c, "kpm_init");
}

int kpm_init_f64(evsl_ctx *c, int nvec, uint64_t seed, double *W0, uint64_t first)
{
    return kpm_init_t(c, nvec, seed, W0, first);
}
int kpm_init_f32(evsl_ctx *c, int nvec, uint64_t seed, float *W0, uint64_t first)
{
    return kpm_init_t(c, nvec, seed, W0, first);
}

// Per-probe sums sum_r v_l[r] W[r, l] of a row-major probe block (ld columns): block b adds its
// KPM_DOT_ROWS rows in order for every probe, then out[l] = sum_b part[b][l] in block order.
// The order of every probe's sum depends on n only, not on which other probes share the block.
constexpr int KPM_DOT_ROWS = 2048;

template <typename T>
__global__ void k_kpm_probe_dots(int64_t n, int np, int ld, const uint32_t *__restrict__ bits,
                                 const T *__restrict__ W, double *__restrict__ part)
{
    const int nw = (np + 31) >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * KPM_DOT_ROWS, r1 = min(n, r0 + KPM_DOT_ROWS);
    for (int l = threadIdx.x; l < np; l += blockDim.x) {
        double s = 0.0;
        for (int64_t r = r0; r < r1; r++) {
            const double w = (double)W[r * ld + l];
            s += ((bits[r * nw + (l >> 5)] >> (l & 31)) & 1u) ? -w : w;
        }
        part[(int64_t)blockIdx.x * np + l] = s;
    }
}

__global__ void k_kpm_probe_reduce(int np, int nblk, const double *__restrict__ part, double *__restrict__ out)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= np) return;
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += part[(int64_t)b * np + l];
    out[l] = s;
}

template <typename T>
static int kpm_probe_dots_t(evsl_ctx *c, int np, const T *W, double *part, double *out)
{
    const int64_t n = c->A.n;
    const int nblk = (int)((n + KPM_DOT_ROWS - 1) / KPM_DOT_ROWS);
    int st = EVSL_OK;
    uint32_t *bits = kpm_bits(c, np, &st);
    if (st) return st;
    k_kpm_probe_dots<T><<<nblk, 128, 0, c->stream>>>(n, np, kpm_ld(np), bits, W, part);
    c->launches++;
    EVSL_TRY(check_launch(c, "kpm_probe_dots"));
    k_kpm_probe_reduce<<<blocks_for(np, 128), 128, 0, c->stream>>>(np, nblk, part, out);
    c->launches++;
    return check_launch(c, "kpm_probe_reduce");
}

int kpm_probe_dots_f64(evsl_ctx *c, int np, const double *W, double *part, double *out)
{
    return kpm_probe_dots_t(c, np, W, part, out);
}
int kpm_probe_dots_f32(evsl_ctx *c, int np, const float *W, double *part, double *out)
{
    return kpm_probe_dots_t(c, np, W, part, out);
}
int kpm_probe_dot_blocks(evsl_ctx *c) { return (int)((c->A.n + KPM_DOT_ROWS - 1) / KPM_DOT_ROWS); }

template <typename T, bool DBL>
static void launch_kpm(evsl_ctx *c, bool hat, const T *val, int mode, int nvec, int ld, const uint32_t *bits,
                       const T *x, const T *xprev, T *out, T cc, T sc, int nblk, double *p1, double *p2)
{
    const DevMatrix &A = c->A;
    constexpr int PPL = sizeof(T) == 8 ? 2 : 4;
    if (hat)
        k_kpm_step<T, true, PPL, DBL><<<nblk, TPB, 0, c->stream>>>(mode, A.n, A.nslices, A.sptr, A.col, val, A.rlen,
                                                                    nvec, ld, bits, x, xprev, out, cc, sc, p1, p2);
    else
        k_kpm_step<T, false, PPL, DBL><<<nblk, TPB, 0, c->stream>>>(mode, A.n, A.nslices, A.sptr, A.col, val, A.rlen,
                                                                     nvec, ld, bits, x, xprev, out, cc, sc, p1, p2);
}

// dbl: the doubling form; the step's partials go to rows 2j-1 (w_j^T w_{j-1}) and 2j
// (||w_j||^2) of `part` for the step that forms w_j (k = j), else to row k
template <typename T>
static int kpm_step_t(evsl_ctx *c, int mode, int nvec, const T *x, const T *xprev, T *out,
                      double cc, double sc, double *part, int k, int nblk, const T *val, bool hat,
                      bool dbl = false)
{
    int st = EVSL_OK;
    uint32_t *bits = kpm_bits(c, nvec, &st);
    if (st) return st;
    const DevMatrix &A = c->A;
    const int ld = kpm_ld(nvec);
    const bool h = hat && A.vhat;
    const T *v = h ? (sizeof(T) == 8 ? (const T *)A.vhat : (const T *)A.vhat32) : val;
    if (dbl)
        launch_kpm<T, true>(c, h, v, mode, nvec, ld, bits, x, xprev, out, (T)cc, (T)sc, nblk,
                            part + (int64_t)(2 * k - 1) * nblk, part + (int64_t)(2 * k) * nblk);
    else
        launch_kpm<T, false>(c, h, v, mode, nvec, ld, bits, x, xprev, out, (T)cc, (T)sc, nblk,
                             part + (int64_t)k * nblk, nullptr);
    c->launches++;
    return check_launch(c, "kpm_step");
}

int kpm_step_f64(evsl_ctx *c, int mode, int nvec, uint64_t, const double *x, const double *xprev,
                 double *out, double cc, double sc, double *part, int k, int nblk, bool hat, bool dbl)
{
    return kpm_step_t<double>(c, mode, nvec, x, xprev, out, cc, sc, part, k, nblk, c->A.val, hat, dbl);
}

int kpm_step_f32(evsl_ctx *c, int mode, int nvec, uint64_t, const float *x, const float *xprev,
                 float *out, double cc, double sc, double *part, int k, int nblk, bool hat, bool dbl)
{
    return kpm_step_t<float>(c, mode, nvec, x, xprev, out, cc, sc, part, k, nblk, c->A.val32, hat, dbl);
}

int convert_f64_to_f32(evsl_ctx *c, int64_t count, const double *x, float *y)
{
    k_f64_to_f32<<<blocks_for(count, 256), 256, 0, c->stream>>>(count, x, y);
    c->launches++;
    return check_launch(c, "f64_to_f32");
}

int convert_f32_to_f64(evsl_ctx *c, int64_t count, const float *x, double *y)
{
    k_f32_to_f64<<<blocks_for(count, 256), 256, 0, c->stream>>>(count, x, y);
    c->launches++;
    return check_launch(c, "f32_to_f64");
}

int fill_uniform_f64(evsl_ctx *c, int64_t n, uint64_t seed, int stream, uint64_t index, double *x)
{
    k_fill_uniform<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, sm_key(seed, (uint64_t)stream), index, x);
    c->launches++;
    return check_launch(c, "fill_uniform");
}

int fill_rademacher_f64(evsl_ctx *c, int64_t n, uint64_t seed, int stream, uint64_t index, double *x)
{
    k_fill_sign<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, sm_key(seed, (uint64_t)stream), index, x);
    c->launches++;
    return check_launch(c, "fill_rademacher");
}

// ------------------------------------------------------------------------------------------
// Allocation-free filter application.  The recurrence temporaries live in one fixed device
// array shared by all calls on a device; its device address is looked up once per device.
namespace {

__device__ __align__(256) double g_noalloc_scratch[2 * (size_t)EVSL_NOALLOC_MAX_ELEMS];

constexpr int NOALLOC_MAX_DEVICES = 64;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
std::mutex g_noalloc_mu;

}  // namespace

extern "C" int evsl_filter_apply_noalloc(evsl_ctx *c, const evsl_polfilt *pol, int nvec,
                                         const double *X, double *Y)
{
    if (!c) return EVSL_ERR_ARG;
    c->err.clear();
    if (!pol || !pol->coef || pol->deg < 0 || nvec < 1 || !X || !Y)
        return ctx_fail(c, EVSL_ERR_ARG, "filter_apply_noalloc: bad arguments");
    if (c->A.n == 0) return ctx_fail(c, EVSL_ERR_STATE, "filter_apply_noalloc: no matrix set");
    const int64_t N = c->A.n * (int64_t)nvec;
    if (N > (int64_t)EVSL_NOALLOC_MAX_ELEMS)
        return ctx_fail(c, EVSL_ERR_ARG,
                        "filter_apply_noalloc: n * nvec = %lld exceeds EVSL_NOALLOC_MAX_ELEMS = %d",
                        (long long)N, EVSL_NOALLOC_MAX_ELEMS);
    if (c->device < 0 || c->device >= NOALLOC_MAX_DEVICES)
        return ctx_fail(c, EVSL_ERR_ARG, "filter_apply_noalloc: device ordinal %d not supported", c->device);
    // the caller's current device is put back on every return path
    int prev_dev = -1;
    cudaError_t e = cudaGetDevice(&prev_dev);
    if (e != cudaSuccess) return ctx_cuda(c, e, "filter_apply_noalloc get device");
    struct DeviceRestore {
        int dev;
        ~DeviceRestore() { cudaSetDevice(dev); }
    } restore{prev_dev};
    e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return ctx_cuda(c, e, "filter_apply_noalloc set device");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[c->device]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return ctx_cuda(c, e, "filter_apply_noalloc symbol address");
            g_noalloc_ptr[c->device] = (double *)p;
        }
        scratch = g_noalloc_ptr[c->device];
    }
    double *B0 = scratch, *B1 = scratch + EVSL_NOALLOC_MAX_ELEMS;
    const double cc = 0.5 * (pol->lmax + pol->lmin), d = 0.5 * (pol->lmax - pol->lmin);
    const double *coef = pol->coef;
    int st;
    if (pol->deg == 0) {
        st = scale_vec(c, N, const_cast<double *>(X), coef[0], Y);
    } else {
        const bool hat = c->A.vhat && c->A.hat_c == cc && c->A.hat_d == d;
        st = cheb_step_f64(c, 0, nvec, X, nullptr, B0, Y, cc, 1.0 / d, coef[0], coef[1], hat);
        const double *prev = X;
        double *cur = B0;
        for (int j = 2; j <= pol->deg && st == EVSL_OK; j++) {
            double *out = (j == 2) ? B1 : const_cast<double *>(prev);
            st = cheb_step_f64(c, 1, nvec, cur, prev, out, Y, cc, 2.0 / d, 0.0, coef[j], hat);
            prev = cur;
            cur = out;
        }
    }
    if (st != EVSL_OK) return st;
    e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "filter_apply_noalloc");
}
