// FP64-accurate dense GEMMs on the tensor cores (tcgen05.mma, TMEM accumulators, TMA loads).
//
// Where the method needs them: the Ritz vectors Y = Q S of Algorithm 2's restart (a tall n x k
// basis times a small k x l eigenvector block) and the Rayleigh-Ritz / Gram projections
// C = W^T Z (contraction over the n rows).  Both must be FP64 to reach 1e-8 residuals, and FP64
// arithmetic on this part runs at about 1.1 TFLOP/s, so they are computed here on the BF16
// tensor cores by exact digit splitting: Ozaki scheme I (Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), in its fixed-width integer-digit form.
//
//  * Every row i of op(A) is scaled by 2^e_i (|a_ik| < 2^e_i) and written as nine signed 6-bit
//    digits, a_ik = 2^e_i sum_{s=1..9} A_s[i,k] 2^(-6 s) + (error < 2^(e_i - 54)), by
//    truncating the 54-bit fixed-point value of |a_ik| 2^(54 - e_i).  Columns of B likewise
//    (2^f_j, digits B_t).  Digits are integers of magnitude <= 63: exact in BF16.
//  * C_ij = 2^(e_i + f_j) sum_{s+t<=11} 2^(-6(s+t)) (A_s B_t)_ij.  The 53 digit products with
//    s + t <= 11 are kept: the dropped ones are below the representation error, and the result
//    is then at least as accurate as a plain FP64 dot product (about 4e-17 of sum_k |a||b| on
//    random data, against 1.6e-16 for FP64 summation).  Products of one diagonal d = s + t share
//    their scale and are summed into one FP32 TMEM accumulator.
//  * Exactness: a diagonal holds at most 9 products of at most 63 * 63 per k, so over a K-chunk of
//    448 its partial sums stay below 9 * 3969 * 448 < 2^24 and the FP32 accumulation of integer
//    products is exact.  After each chunk the ten accumulators are read back (tcgen05.ld),
//    converted to integers and added, shifted by 6 (11 - d) bits, into a 128-bit integer per
//    output element; the sum F_ij is exact, and C_ij = 2^(e_i + f_j - 66) F_ij is rounded once
//    to FP64 at the end.  The result is deterministic and independent of the tiling.
//
// Kernel: one CTA per 128 x 48 output tile, 320 threads.  Warp 0 issues TMA loads of one K-block
// (32 wide) of all nine A digit tiles (128 x 32) and B digit tiles (48 x 32) into a two-stage
// shared-memory ring (64-byte swizzle); warp 1 owns the TMEM allocation and issues 15 MMAs per
// K-step of 16: for A digit s, one MMA multiplies it by up to five B digit tiles stacked along N
// (N <= 240), writing diagonals s+t..s+t+4 at once (diagonal d lives in TMEM columns
// 48 (d - 2) .. 48 (d - 1)); warps 2-9 drain the accumulators after each chunk and finally
// convert, scale and store their 128 x 48 FP64 results.  Every wait on an mbarrier is bounded;
// on expiry the kernel records EVSL_ERR_TIMEOUT in a device flag, stops all roles, waits
// (bounded) for its copies and MMAs in flight and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "evsl_internal.h"

namespace {

constexpr int OZ_S = 9;             // digits per element
constexpr int OZ_BETA = 6;          // bits per digit
constexpr int OZ_BM = 128;          // tile rows (MMA M)
constexpr int OZ_BN = 48;           // tile columns (per diagonal in TMEM)
constexpr int OZ_BK = 32;           // K per pipeline stage (64-byte rows)
constexpr int OZ_KC = 448;          // K per exact chunk (14 stages)
constexpr int OZ_KB_PER_CHUNK = OZ_KC / OZ_BK;
constexpr int OZ_STAGES = 2;
constexpr int OZ_A_TILE = OZ_BM * OZ_BK * 2;                    // 8192 B per digit
constexpr int OZ_B_TILE = OZ_BN * OZ_BK * 2;                    // 3072 B per digit
constexpr int OZ_STAGE_A = OZ_S * OZ_A_TILE;                    // 73728 B
constexpr int OZ_STAGE_BYTES = OZ_S * (OZ_A_TILE + OZ_B_TILE);  // 101376 B
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_THREADS = 320;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES + 1024 /* barriers */ + 1024 /* alignment */;
constexpr int OZ_DMAX = OZ_S + 2;                               // highest diagonal kept
constexpr int OZ_ND = OZ_DMAX - 1;                              // diagonals 2..11
constexpr int OZ_FIX_SHIFT = OZ_DMAX * OZ_BETA;                 // 66
constexpr uint32_t OZ_WAIT_LIMIT = 1u << 24;

static_assert(OZ_KC % OZ_BK == 0, "chunk must hold whole stages");
static_assert(OZ_S * (OZ_BETA == 6 ? 3969 : 0) * OZ_KC < (1 << 24), "chunk sums must stay exact in FP32");
static_assert(OZ_ND * OZ_BN <= OZ_TMEM_COLS, "diagonals must fit in TMEM");

// MMA groups of one K-step: A digit s times B digits t0 .. t0 + nb - 1 (stacked along N), all
// 53 pairs with s + t <= 11.  The first three cover every diagonal exactly once (2-6, 7-10, 11)
// and overwrite them at the start of a chunk; the others accumulate.
struct Grp {
    int s, t0, nb;
};
__constant__ Grp c_grp[15] = {{1, 1, 5}, {1, 6, 4}, {2, 9, 1}, {2, 1, 5}, {2, 6, 3}, {3, 1, 5}, {3, 6, 3}, {4, 1, 5},
                              {4, 6, 2}, {5, 1, 5}, {5, 6, 1}, {6, 1, 5}, {7, 1, 4}, {8, 1, 3}, {9, 1, 2}};
constexpr int OZ_NGRP = 15;
constexpr int OZ_NINIT = 3;

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `parity` to complete; false if it did not within the limit or
// (when abort_flag is given) another role gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    for (uint32_t i = 0; i < OZ_WAIT_LIMIT; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255) {
            if (abort_flag && *abort_flag) return false;
            __nanosleep(128);
        }
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                            int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
            "r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulation, M = 128
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on `bar` once every MMA issued so far by this thread has completed
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 24 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per lane), waited for in
// the same statement so the registers are valid on return
__device__ __forceinline__ void tmem_ld24(uint32_t taddr, uint32_t (&r)[24])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%24];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%25];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(taddr), "r"(taddr + 16)
        : "memory");
}

// Instruction descriptor of kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12
// = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor of a K-major tile with 64-byte rows and the 64-byte swizzle:
// start address >> 4 (bits 0-13), leading offset 16 B (unused when K fits in the swizzle row),
// stride 512 B between 8-row groups (bits 32-45), fixed 0b001 in bits 46-48, swizzle code 4.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// ------------------------------------------------------------------ digit splitting
__device__ __forceinline__ int biased_exp(double a) { return (int)((__double_as_longlong(a) >> 52) & 0x7FF); }

// BF16 bit patterns of the integers 0..63
__device__ __forceinline__ uint16_t bf16_small_int(uint32_t d)
{
    if (d == 0) return 0;
    const int e = 31 - __clz(d);                       // 0..5
    return (uint16_t)(((127 + e) << 7) | ((d << (7 - e)) & 0x7F));
}

// The nine signed digits of a relative to the row scale 2^e_i, e_i = max(emax, 1) - 1022 with
// emax the largest biased exponent of the row: truncation of |a| 2^(54 - e_i) to an integer.
__device__ __forceinline__ void split9(double a, int emax_eff, uint16_t (&dg)[OZ_S])
{
    const uint64_t bits = (uint64_t)__double_as_longlong(a);
    const int ea = (int)((bits >> 52) & 0x7FF);
    const uint64_t mant = (bits & ((1ull << 52) - 1)) | (ea ? (1ull << 52) : 0ull);
    const int sh = max(ea, 1) - emax_eff + 1;          // <= 1
    uint64_t m = 0;
    if (sh >= 0) m = mant << sh;
    else if (sh > -64) m = mant >> (-sh);
    const uint16_t sign = (uint16_t)((bits >> 63) << 15);
#pragma unroll
    for (int s = 0; s < OZ_S; s++) {
        const uint32_t d = (uint32_t)(m >> ((OZ_S - 1 - s) * OZ_BETA)) & 63u;
        const uint16_t v = bf16_small_int(d);
        dg[s] = v ? (uint16_t)(v | sign) : (uint16_t)0;
    }
}

// Vectors stored contiguously: vector i is X[i * ldx + k], k < K.  One warp per vector: the
// largest exponent, then the digits, written to out[s][i][k] (row stride kp BF16).
__global__ void k_oz_split_vec(int64_t R, int64_t K, const double *__restrict__ X, int64_t ldx, int64_t kp,
                               uint16_t *__restrict__ out, int *__restrict__ E)
{
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= R) return;
    const double *x = X + i * ldx;
    int me = 0;
    for (int64_t k = lane; k < K; k += 32) me = max(me, biased_exp(x[k]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) me = max(me, __shfl_xor_sync(0xffffffffu, me, off));
    const int emax_eff = max(me, 1);
    if (lane == 0) E[i] = emax_eff - 1022;
    const int64_t plane = R * kp;
    uint16_t *o = out + i * kp;
    for (int64_t k = lane; k < K; k += 32) {
        uint16_t dg[OZ_S];
        split9(x[k], emax_eff, dg);
#pragma unroll
        for (int s = 0; s < OZ_S; s++) o[s * plane + k] = dg[s];
    }
}

// Rows of a column-major matrix: row i is X[i + k * ldx], k < K.  One thread per row; digits of
// 8 consecutive k are packed into one 16-byte store per digit plane.
__global__ void k_oz_split_rows(int64_t R, int64_t K, const double *__restrict__ X, int64_t ldx, int64_t kp,
                                uint16_t *__restrict__ out, int *__restrict__ E)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= R) return;
    int me = 0;
    for (int64_t k = 0; k < K; k++) me = max(me, biased_exp(X[i + k * ldx]));
    const int emax_eff = max(me, 1);
    E[i] = emax_eff - 1022;
    const int64_t plane = R * kp;
    for (int64_t k0 = 0; k0 < K; k0 += 8) {
        uint32_t w[OZ_S][4];
#pragma unroll
        for (int s = 0; s < OZ_S; s++) w[s][0] = w[s][1] = w[s][2] = w[s][3] = 0;
#pragma unroll
        for (int t = 0; t < 8; t++) {
            if (k0 + t < K) {
                uint16_t dg[OZ_S];
                split9(X[i + (k0 + t) * ldx], emax_eff, dg);
#pragma unroll
                for (int s = 0; s < OZ_S; s++) w[s][t >> 1] |= (uint32_t)dg[s] << (16 * (t & 1));
            }
        }
#pragma unroll
        for (int s = 0; s < OZ_S; s++)
            *reinterpret_cast<uint4 *>(out + s * plane + i * kp + k0) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
}

// ------------------------------------------------------------------ the tensor-core kernel
// mode 0: C = result; 1: C -= result; 2: C += result
__global__ void __launch_bounds__(OZ_THREADS, 1)
k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t M, int N,
          int64_t K, const int *__restrict__ eA, const int *__restrict__ eB, double *__restrict__ C, int64_t ldc,
          int mode, int *__restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + OZ_STAGES * OZ_STAGE_BYTES);
    // bars: full[0..1], empty[0..1], tmem_full, tmem_empty, done
    uint32_t *tmem_slot = (uint32_t *)(bars + 8);
    volatile int *abort_flag = (volatile int *)(bars + 9);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[2]);
    const uint32_t tmem_full = smem_u32(&bars[4]), tmem_empty = smem_u32(&bars[5]), done = smem_u32(&bars[6]);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * OZ_BN;
    const int64_t m0 = (int64_t)blockIdx.y * OZ_BM;
    const int nkb = (int)((K + OZ_BK - 1) / OZ_BK);
    const int nchunk = (nkb + OZ_KB_PER_CHUNK - 1) / OZ_KB_PER_CHUNK;

    if (threadIdx.x == 0) {
        mbar_init(full0, 1);
        mbar_init(full0 + 8, 1);
        mbar_init(empty0, 1);
        mbar_init(empty0 + 8, 1);
        mbar_init(tmem_full, 1);
        mbar_init(tmem_empty, 8);
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), OZ_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    bool timed_out = false;

    if (warp == 0) {
        // ---------------- TMA producer
        int issued = 0;
        if (lane == 0) {
            for (int it = 0; it < nkb; it++) {
                const int st = it & 1;
                const uint32_t par = ((it >> 1) & 1) ^ 1;
                if (!mbar_wait(empty0 + 8 * st, par, abort_flag)) {
                    timed_out = true;
                    break;
                }
                const uint32_t sa = smem_u32(smem + st * OZ_STAGE_BYTES);
                mbar_expect_tx(full0 + 8 * st, OZ_STAGE_BYTES);
                tma_load_3d(sa, &tmA, full0 + 8 * st, it * OZ_BK, (int)m0, 0);
                tma_load_3d(sa + OZ_STAGE_A, &tmB, full0 + 8 * st, it * OZ_BK, n0, 0);
                issued = it + 1;
            }
            if (timed_out) {
                // let the copies already issued land before the shared memory is released
                for (int it = std::max(0, issued - OZ_STAGES); it < issued; it++)
                    mbar_wait(full0 + 8 * (it & 1), (it >> 1) & 1, nullptr);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int issued_any = 0;
            for (int it = 0; it < nkb && !timed_out; it++) {
                const int st = it & 1;
                const int kb = it % OZ_KB_PER_CHUNK, chunk = it / OZ_KB_PER_CHUNK;
                if (kb == 0 && chunk > 0 && !mbar_wait(tmem_empty, (chunk - 1) & 1, abort_flag)) {
                    timed_out = true;
                    break;
                }
                if (!mbar_wait(full0 + 8 * st, (it >> 1) & 1, abort_flag)) {
                    timed_out = true;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + st * OZ_STAGE_BYTES);
                const uint32_t sb = sa + OZ_STAGE_A;
#pragma unroll
                for (int ks = 0; ks < OZ_BK / 16; ks++) {
#pragma unroll
                    for (int g = 0; g < OZ_NGRP; g++) {
                        const Grp gr = c_grp[g];
                        const uint64_t ad = sdesc_sw64(sa + (gr.s - 1) * OZ_A_TILE + ks * 32);
                        const uint64_t bd = sdesc_sw64(sb + (gr.t0 - 1) * OZ_B_TILE + ks * 32);
                        const uint32_t col = (uint32_t)((gr.s + gr.t0 - 2) * OZ_BN);
                        const uint32_t acc = (kb == 0 && ks == 0 && g < OZ_NINIT) ? 0u : 1u;
                        umma_bf16(tmem_base + col, ad, bd, idesc_bf16(OZ_BM, OZ_BN * gr.nb), acc);
                    }
                }
                issued_any = 1;
                umma_commit(empty0 + 8 * st);                        // frees the stage when done
                if (kb == OZ_KB_PER_CHUNK - 1 || it == nkb - 1) umma_commit(tmem_full);
            }
            if (issued_any) {
                // every MMA (and the arrivals it triggers) completes before TMEM is freed
                umma_commit(done);
                if (!mbar_wait(done, 0, nullptr)) timed_out = true;
            }
        }
    } else {
        // ---------------- drain and epilogue (warps 2..9)
        const int q = warp & 3;                 // TMEM lane quadrant of this warp
        const int half = (warp - 2) >> 2;       // which 24 of the 48 columns
        const uint32_t lane_addr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 24);
        uint64_t lo[24];
        int64_t hi[24];
#pragma unroll
        for (int j = 0; j < 24; j++) {
            lo[j] = 0;
            hi[j] = 0;
        }
        for (int ch = 0; ch < nchunk; ch++) {
            // every lane waits; the warp proceeds (to warp-wide TMEM loads) only together
            const bool ok = __all_sync(0xffffffffu, mbar_wait(tmem_full, ch & 1, abort_flag));
            if (!ok) {
                timed_out = true;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int di = 0; di < OZ_ND; di++) {
                uint32_t r[24];
                tmem_ld24(lane_addr + (uint32_t)(di * OZ_BN), r);
                const int sh = (OZ_DMAX - 2 - di) * OZ_BETA;  // diagonal d = di + 2 -> 6 (11 - d)
#pragma unroll
                for (int j = 0; j < 24; j++) {
                    const int64_t v = __float2int_rn(__uint_as_float(r[j]));
                    const uint64_t xl = (uint64_t)v << sh;
                    const int64_t xh = sh ? (v >> (64 - sh)) : (v >> 63);
                    const uint64_t nl = lo[j] + xl;
                    hi[j] += xh + (int64_t)(nl < lo[j]);
                    lo[j] = nl;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_empty);
        }
        if (!timed_out) {
            const int64_t i = m0 + q * 32 + lane;
            if (i < M) {
                const int ei = eA[i];
#pragma unroll
                for (int j = 0; j < 24; j++) {
                    const int col = n0 + half * 24 + j;
                    if (col < N) {
                        // |F| as two 64-bit halves, converted with one rounding
                        uint64_t l = lo[j];
                        int64_t h = hi[j];
                        const bool neg = h < 0;
                        if (neg) {
                            l = ~l + 1;
                            h = ~h + (int64_t)(l == 0);
                        }
                        double mag = fma((double)h, 18446744073709551616.0, (double)l);
                        const double val = ldexp(neg ? -mag : mag, ei + eB[col] - OZ_FIX_SHIFT);
                        double *cp = C + (int64_t)col * ldc + i;
                        if (mode == 0) *cp = val;
                        else if (mode == 1) *cp -= val;
                        else *cp += val;
                    }
                }
            }
        }
    }
    if (timed_out) {
        *abort_flag = 1;
        atomicExch(err, (int)EVSL_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, OZ_TMEM_COLS);
    }
}

// ------------------------------------------------------------------ host side
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// 3-D map over digit planes [S][rows][kp] (BF16): box 32 (k) x box_rows x 9 planes, 64-byte
// swizzle, zero fill past K and past the rows
bool make_map(CUtensorMap *map, const uint16_t *base, int64_t rows, int64_t K, int64_t kp, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)OZ_S};
    cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)rows * kp * 2};
    cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, (cuuint32_t)OZ_S};
    cuuint32_t estr[3] = {1, 1, 1};
    std::memset(map, 0, sizeof(*map));
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr size_t OZ_WS_CAP = (size_t)1 << 31;   // digit planes of one panel: at most 2 GiB

inline unsigned nblk(int64_t threads, int tpb) { return (unsigned)((threads + tpb - 1) / tpb); }

int oz_launch(evsl_ctx *c, const uint16_t *Ad, const int *Ea, int64_t M, const uint16_t *Bd, const int *Eb, int N,
              int64_t K, int64_t kp, double *C, int64_t ldc, int mode, int *dflag)
{
    CUtensorMap ma, mb;
    if (!make_map(&ma, Ad, M, K, kp, OZ_BM) || !make_map(&mb, Bd, N, K, kp, OZ_BN))
        return ctx_fail(c, EVSL_ERR_CUDA, "tensor-core GEMM: cannot encode the TMA maps");
    // the attribute belongs to the current device: set it on every call (a host-side call of
    // about a microsecond), not once per process
    cudaError_t ea = cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    if (ea != cudaSuccess) return ctx_cuda(c, ea, "tensor-core GEMM shared memory");
    dim3 grid((unsigned)((N + OZ_BN - 1) / OZ_BN), (unsigned)((M + OZ_BM - 1) / OZ_BM));
    k_oz_gemm<<<grid, OZ_THREADS, OZ_SMEM, c->stream>>>(ma, mb, M, N, K, Ea, Eb, C, ldc, mode, dflag);
    c->launches++;
    return check_launch(c, "tensor-core GEMM");
}

}  // namespace

// C (M x N, ldc) {=, -=, +=} op(A) B in FP64 accuracy on the tensor cores.
//   trans_a = false: A is M x K column-major (lda)  -- Ritz vectors Y = Q S
//   trans_a = true:  A is K x M column-major (lda), op(A) = A^T  -- projections W^T Z
//   B is K x N column-major (ldb).  mode: 0 store, 1 subtract, 2 add.
int gemm_tc(evsl_ctx *c, bool trans_a, int64_t M, int N, int64_t K, const double *A, int64_t lda, const double *B,
            int64_t ldb, double *C, int64_t ldc, int mode)
{
    if (M <= 0 || N <= 0) return EVSL_OK;
    int st = EVSL_OK;
    int *dflag = (int *)ctx_ws(c, WS_OZ_FLAG, 256, &st);
    if (st) return st;
    cudaError_t e = cudaMemsetAsync(dflag, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "tensor-core GEMM flag");
    if (K <= 0) {
        if (mode != 0) return EVSL_OK;
        e = cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * M, N, c->stream);
        return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "tensor-core GEMM zero");
    }
    if (!trans_a) {
        // panels of rows of A; B's digits once
        const int64_t kp = (K + 7) & ~(int64_t)7;
        int64_t P = (int64_t)(OZ_WS_CAP / ((size_t)OZ_S * kp * 2)) / OZ_BM * OZ_BM;
        P = std::min<int64_t>(P, (int64_t)65535 * OZ_BM);          // grid.y limit
        P = std::max<int64_t>(OZ_BM, std::min<int64_t>(P, (M + OZ_BM - 1) / OZ_BM * OZ_BM));
        uint16_t *Bd = (uint16_t *)ctx_ws(c, WS_OZ_B, sizeof(uint16_t) * OZ_S * (size_t)N * kp, &st);
        if (st) return st;
        uint16_t *Ad = (uint16_t *)ctx_ws(c, WS_OZ_A, sizeof(uint16_t) * OZ_S * (size_t)P * kp, &st);
        if (st) return st;
        int *E = (int *)ctx_ws(c, WS_OZ_E, sizeof(int) * (size_t)(P + N + 64), &st);
        if (st) return st;
        int *Ea = E, *Eb = E + P + 32;
        k_oz_split_vec<<<nblk((int64_t)N * 32, 256), 256, 0, c->stream>>>(N, K, B, ldb, kp, Bd, Eb);
        c->launches++;
        EVSL_TRY(check_launch(c, "GEMM split B"));
        for (int64_t r0 = 0; r0 < M; r0 += P) {
            const int64_t rows = std::min(P, M - r0);
            k_oz_split_rows<<<nblk(rows, 128), 128, 0, c->stream>>>(rows, K, A + r0, lda, kp, Ad, Ea);
            c->launches++;
            EVSL_TRY(check_launch(c, "GEMM split A"));
            EVSL_TRY(oz_launch(c, Ad, Ea, rows, Bd, Eb, N, K, kp, C + r0, ldc, mode, dflag));
        }
    } else {
        // panels of the contraction dimension; the first applies `mode`, later ones add (or
        // subtract) their partial products in FP64
        int64_t KP = (int64_t)(OZ_WS_CAP / ((size_t)OZ_S * 2 * (size_t)(M + N))) / OZ_KC * OZ_KC;
        KP = std::max<int64_t>(OZ_KC, std::min<int64_t>(KP, (K + OZ_KC - 1) / OZ_KC * OZ_KC));
        const int64_t kp = KP;
        uint16_t *Ad = (uint16_t *)ctx_ws(c, WS_OZ_A, sizeof(uint16_t) * OZ_S * (size_t)M * kp, &st);
        if (st) return st;
        uint16_t *Bd = (uint16_t *)ctx_ws(c, WS_OZ_B, sizeof(uint16_t) * OZ_S * (size_t)N * kp, &st);
        if (st) return st;
        int *E = (int *)ctx_ws(c, WS_OZ_E, sizeof(int) * (size_t)(M + N + 64), &st);
        if (st) return st;
        int *Ea = E, *Eb = E + M + 32;
        for (int64_t k0 = 0; k0 < K; k0 += KP) {
            const int64_t kl = std::min(KP, K - k0);
            k_oz_split_vec<<<nblk(M * 32, 256), 256, 0, c->stream>>>(M, kl, A + k0, lda, kp, Ad, Ea);
            c->launches++;
            k_oz_split_vec<<<nblk((int64_t)N * 32, 256), 256, 0, c->stream>>>(N, kl, B + k0, ldb, kp, Bd, Eb);
            c->launches++;
            EVSL_TRY(check_launch(c, "GEMM split"));
            const int md = (k0 == 0) ? mode : (mode == 1 ? 1 : 2);
            EVSL_TRY(oz_launch(c, Ad, Ea, M, Bd, Eb, N, kl, kp, C, ldc, md, dflag));
        }
    }
    int flag = 0;
    e = cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "tensor-core GEMM");
    if (flag) return ctx_fail(c, EVSL_ERR_TIMEOUT, "tensor-core GEMM: a bounded pipeline wait expired");
    return EVSL_OK;
}
