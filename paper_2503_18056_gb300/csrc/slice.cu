// Mixed-precision contractions of the rounding (precision form) on the
// 5th-generation tensor cores: the left Gram G = A^T A and the core update
// C = A B^T, for the contractions App. A.4 names as the dominant cost.
//
// Split.  Each FP64 operand is scaled by a power of two per column (Gram: the
// contraction runs over rows, so only columns may carry their own scale) or
// per row (update: rows i of A and rows c of B are not summed) so that
// |a| 2^-e < 1/2, rounded to 48-bit fixed point and cut into S = 7 balanced
// base-128 digits (d_0 in [0, 64], d_1..d_6 in [-64, 63]),
//   a = 2^e sum_s d_s 128^-(s+1),
// every digit exact in BF16 and every digit product (|d_s d_t| <= 2^12)
// exact in FP32.  Products of the same level w = s + t share the weight
// 128^-(w+2); level w has at most 7 pairs, so summed over a block of 512
// contraction indices they stay below 512 * 7 * 2^12 < 2^24 and the tensor
// cores' FP32 block sums are exact integers.  Each block sum is scaled by
// 128^-w (exact) and added into a double-float accumulator (hi + lo in FP32,
// TwoSum + renormalisation: about 48 bits).  Levels w >= 7 are dropped: 28 BF16 products per term, about
// 2^-48 of max|a| max|b| per term against 2^-53 for FP64.  No FP64 arithmetic
// runs in the inner loops (GB300's FP64 pipe is ~1/70 of its FP32 pipe).
//
// Both kernels keep seven per-level FP32 accumulators of a 128 x 64 output
// tile in tensor memory (448 of 512 columns), issue tcgen05.mma (kind::f16,
// BF16 x BF16 -> FP32, M = 128, K = 16, N = 64 per B digit, up to four B
// digits per MMA) from one thread with both operands K-major in shared memory
// (64-byte swizzle), and drain the accumulators with tcgen05.ld every 512
// contraction indices.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "internal.h"

namespace ttsn {

namespace {


__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// (hi, lo) += x: Knuth's TwoSum of hi and x, the low parts added, then
// renormalised with Fast2Sum so |lo| <= ulp(hi)/2 and each add costs about
// 2^-48 of the running sum (without the renormalisation lo grows and loses bits
// over thousands of adds)
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    float e = (hi - (s - bb)) + (x - bb);
    e += lo;
    const float h2 = s + e;
    lo = e - (h2 - s);
    hi = h2;
}

// Exponent e with |v| < 2^e for the largest |v| (0 for a zero maximum).
__device__ __forceinline__ int exp_bound(double vmax) {
    if (!(vmax > 0.0)) return 0;
    return ilogb(vmax) + 1;
}

// |v| as its bit pattern: for non-negative doubles the patterns order as the
// values, so the maxima below are integer compares (fmax and fabs would run on
// GB300's FP64 pipe, a small fraction of its integer rate: a scan of 2.1M x
// 897 kept it 83% busy).  NaN maps to 0, which ignores it as fmax does; Inf
// stays the largest pattern.
__device__ __forceinline__ unsigned long long mag_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    return b > 0x7FF0000000000000ull ? 0ull : b;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

__global__ void col_max_kernel(int m, int n, const double* __restrict__ A, long lda,
                               unsigned long long* cmax) {
    // block: 32 columns x (blockDim/32) row lanes; grid.y splits the rows
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int rlane = threadIdx.x >> 5, rstride = blockDim.x >> 5;
    const long rows_per = ((long)m + gridDim.y - 1) / gridDim.y;
    const long r0 = blockIdx.y * rows_per, r1 = min((long)m, r0 + rows_per);
    unsigned long long mx = 0;
    if (j < n) {
        long i = r0 + rlane;
        unsigned long long m1 = 0, m2 = 0, m3 = 0;  // four loads in flight per thread
        for (; i + 3 * rstride < r1; i += 4 * rstride) {
            mx = umax64(mx, mag_bits(A[i * lda + j]));
            m1 = umax64(m1, mag_bits(A[(i + rstride) * lda + j]));
            m2 = umax64(m2, mag_bits(A[(i + 2 * rstride) * lda + j]));
            m3 = umax64(m3, mag_bits(A[(i + 3 * rstride) * lda + j]));
        }
        for (; i < r1; i += rstride) mx = umax64(mx, mag_bits(A[i * lda + j]));
        mx = umax64(umax64(mx, m1), umax64(m2, m3));
    }
    if (j < n && mx > 0) atomicMax(cmax + j, mx);
}

__global__ void row_exp_kernel(long m, int n, const double* __restrict__ A, long lda, int* e) {
    const int lane = threadIdx.x & 31;
    const long warps = (long)gridDim.x * (blockDim.x >> 5);
    for (long i = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += warps) {
        unsigned long long mx = 0, m1 = 0, m2 = 0, m3 = 0;  // four loads in flight per lane
        int j = lane;
        for (; j + 96 < n; j += 128) {
            mx = umax64(mx, mag_bits(A[i * lda + j]));
            m1 = umax64(m1, mag_bits(A[i * lda + j + 32]));
            m2 = umax64(m2, mag_bits(A[i * lda + j + 64]));
            m3 = umax64(m3, mag_bits(A[i * lda + j + 96]));
        }
        for (; j < n; j += 32) mx = umax64(mx, mag_bits(A[i * lda + j]));
        mx = umax64(umax64(mx, m1), umax64(m2, m3));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = umax64(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) e[i] = exp_bound(__longlong_as_double((long long)mx));
    }
}

// Column maxima (the Gram's column exponents) and row exponents (the
// update's, for the same matrix) in one read of A, for n <= 1024.  Warps
// sweep whole rows (grid-stride, so the GPU reads one contiguous window of
// A): a lane loads its columns l + 32 k of the row all at once (up to 32
// loads in flight), the row maximum is a warp reduction whose exponent bound
// lane 0 writes, and each warp folds the row into its own column-maximum
// slice in shared memory (no conflicts, no registers held across rows); the
// block combines its eight slices at the end with one atomicMax per column.
constexpr int CRM_MAXN = 1024;
__global__ void __launch_bounds__(256)
col_row_max_kernel(long m, int n, const double* __restrict__ A, long lda, unsigned long long* cmax,
                   int* erow) {
    extern __shared__ unsigned long long crm_part[];  // [8][n], magnitude bit patterns
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nk = (n + 31) >> 5;
    unsigned long long* mine = crm_part + (long)warp * n;
    for (int j = lane; j < n; j += 32) mine[j] = 0;
    __syncwarp();
    const long nw = (long)gridDim.x * 8;
    for (long i = (long)blockIdx.x * 8 + warp; i < m; i += nw) {
        const double* row = A + i * lda;
        // unconditional loads (lanes past the last column re-read it, which
        // leaves the row maximum unchanged), all issued before the first use
        double v[CRM_MAXN / 32];
#pragma unroll
        for (int k = 0; k < CRM_MAXN / 32; ++k)
            if (k < nk) v[k] = row[min(k * 32 + lane, n - 1)];
        unsigned long long rm = 0;
#pragma unroll
        for (int k = 0; k < CRM_MAXN / 32; ++k) {
            if (k < nk) {
                const unsigned long long a = mag_bits(v[k]);
                const int j = k * 32 + lane;
                if (j < n) mine[j] = umax64(mine[j], a);
                rm = umax64(rm, a);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rm = umax64(rm, __shfl_xor_sync(0xffffffffu, rm, o));
        if (lane == 0) erow[i] = exp_bound(__longlong_as_double((long long)rm));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        unsigned long long mx = crm_part[j];
#pragma unroll
        for (int w = 1; w < 8; ++w) mx = umax64(mx, crm_part[(long)w * n + j]);
        if (mx > 0) atomicMax(cmax + j, mx);
    }
}

__global__ void slgram_reduce_kernel(int n, int ksplit, const double* __restrict__ P, double* G,
                                     long ldg) {
    const long total = (long)n * n;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        const int a = min(i, j), b = max(i, j);
        double s = 0.0;
        for (int z = 0; z < ksplit; ++z) s += P[(long)z * n * n + (long)a * n + b];
        G[(long)i * ldg + j] = s;
    }
}

constexpr int BF16_PEAK_ITERS = 2048;
__global__ void __launch_bounds__(256) bf16_mma_peak_kernel(float* out, unsigned seed) {
    unsigned a[4] = {seed * (threadIdx.x + 1), seed + 3u, seed ^ 5u, seed + 7u};
    unsigned b[2] = {seed * 11u, seed + threadIdx.x};
    float c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
    for (int i = 0; i < BF16_PEAK_ITERS; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) mma_bf16(c[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
    if (s == 1234.5f) out[threadIdx.x] = s;  // keeps the chains live
}


// ======================================================================
// Left Gram on the 5th-generation tensor cores (tcgen05, TMEM, TMA).
//
// Split.  Column-scaled values |a| 2^-e < 1/2 are rounded to 48-bit fixed
// point and cut into S7 = 7 balanced base-128 digits (d_0 in [0, 64],
// d_1..d_6 in [-64, 63]), a = 2^e sum_s d_s 128^-(s+1); every digit is exact
// in BF16 and |d_s d_t| <= 2^12.  The products of level w = s + t (weight
// 128^-(w+2)) summed over a 512-row block stay below 512 * 7 * 2^12 < 2^24,
// so the tensor core's FP32 sums of them are exact integers; levels w >= 7
// are dropped (about 2^-48 of the column scales per term, as the 8-bit form).
// The accumulators are drained (read, scaled, added in double-float on the
// FP32 pipe) once per block, while the MMAs wait: 512-row blocks spend a
// quarter of the drain time of 128-row ones.
//
// Tile.  A CTA owns a 128 (columns j) x 64 (columns k) tile of G and a range
// of rows.  Seven FP32 accumulators (one per level, 128 lanes x 64 columns
// each, 448 of the 512 TMEM columns) receive, per 32-row stage, the 28
// digit-pair products x 2 K-steps as 20 tcgen05.mma (kind::f16, BF16 x BF16
// -> FP32, M = 128, N = 64 .. 256, K = 16; tc_stage_mmas) issued by one
// thread with operands described in shared memory (K-major, 64-byte
// swizzle).  A TMA producer thread streams the stages (all 7 digit planes of
// the tile's 128 + 64 columns in two 4-D boxes per stage from the
// stage-major planes, double-buffered, mbarrier-tracked).  After every
// 512-row block eight drain warps read the accumulators (tcgen05.ld, one TMEM
// lane and half the columns per thread), scale level w by 128^-w and add into
// double-float accumulators.  Every wait is bounded and latches DEV_TIMEOUT.
constexpr int TC_S = 7;
constexpr int TC_M = 128, TC_N = 64, TC_K = 32;
constexpr int TC_BLK = 16;  // stages per exact block (512 rows)
constexpr int TC_STAGES = 2;
constexpr int TC_A_BYTES = TC_S * TC_M * TC_K * 2;  // 57344
constexpr int TC_B_BYTES = TC_S * TC_N * TC_K * 2;  // 28672
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_THREADS = 320;  // warp 0 TMA, warp 1 TMEM + MMA, warps 2-9 drain
constexpr int TC_DRAIN_WARPS = 8;
constexpr int TC_DN = TC_N / 2;  // accumulator columns per drain thread
constexpr unsigned TC_TMEM_COLS = 512;
constexpr long long TC_SPIN = 1LL << 26;
constexpr size_t TC_SMEM = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024 /* barriers */ + 1024 /* align */;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase; false (and DEV_TIMEOUT latched) if it ran out.
__device__ __forceinline__ bool mbar_wait(unsigned a, unsigned parity, int* status) {
    for (long long it = 0; it < TC_SPIN; ++it) {
        if (mbar_try(a, parity)) return true;
        if (it > 32) __nanosleep(64);
    }
    if (status) atomicOr(status, DEV_TIMEOUT);
    return false;
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const void* map, int c0, int c1, int c2, int c3,
                                            unsigned mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row
// groups 512 bytes apart (SBO); LBO is unused for K-major swizzled layouts
// whose K-step (32 bytes) stays inside the 64-byte swizzle span.
__device__ __forceinline__ unsigned long long tc_sdesc(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)(16u >> 4) << 16;
    d |= (unsigned long long)(512u >> 4) << 32;
    d |= 1ull << 46;  // descriptor version
    d |= 4ull << 61;  // 64-byte swizzle
    return d;
}
// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = nn (a multiple of 64 up to 256).
__device__ __forceinline__ unsigned tc_idesc(int nn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(nn >> 3) << 17) | ((unsigned)(TC_M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(unsigned d_tmem, unsigned long long a, unsigned long long b,
                                       unsigned idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The digit-pair products of one 32-deep stage.  The seven B digit tiles sit
// back to back in shared memory (64 rows each, 8-row groups 512 bytes apart),
// so B digits t0 .. t0 + c - 1 form one K-major operand of N = 64 c rows; and
// the accumulator of level w sits at TMEM column 64 w, so the products of A
// digit s with B digits t0 .. t0 + c - 1 (levels s + t0 ..) land in one
// contiguous column range.  Per A digit and K-step one MMA (two where more
// than four B digits remain: N <= 256) does what 7 - s MMAs of N = 64 did:
// 10 MMAs per K-step instead of 28, each A tile read once per MMA, so the
// operand bytes per step fall from 168 KB to 96 KB.  The first stage of a
// block overwrites every level (s = 0 covers levels 0 .. 6).
__device__ __forceinline__ void tc_stage_mmas(unsigned tmem, unsigned aB, unsigned bB, bool first) {
#pragma unroll 1
    for (int s = 0; s < TC_S; ++s) {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const unsigned long long ad = tc_sdesc(aB + (unsigned)(s * TC_M * TC_K * 2 + kk * 32));
            const unsigned acc = (first && s == 0 && kk == 0) ? 0u : 1u;
            for (int t0 = 0; t0 < TC_S - s; t0 += 4) {
                const int c = min(4, TC_S - s - t0);
                const unsigned long long bd = tc_sdesc(bB + (unsigned)(t0 * TC_N * TC_K * 2 + kk * 32));
                tc_mma(tmem + (unsigned)((s + t0) * TC_N), ad, bd, tc_idesc(c * TC_N), acc);
            }
        }
    }
}
__device__ __forceinline__ void tc_commit(unsigned mbar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
        : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane (no wait: the caller
// issues tc_wait_ld before reading r).
__device__ __forceinline__ void tc_ld16(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Seven balanced base-128 digits of v 2^-e (|v| 2^-e < 1/2): |v| 2^(49-e) =
// M 2^(ev - e - 3) is rounded to the integer F (< 2^48), written as
// F = sum_s d_s 128^(6-s), digits carrying the sign of v, as BF16 bit patterns.
// Balanced digits without a carry chain: adding 64 at every lower digit
// position, F + 64 (1 + 128 + ... + 128^5), makes the plain base-128 digits
// d_s + 64 (s = 1 .. 6) and leaves d_0 on top.  A digit becomes a float
// without an int-to-float conversion: the bits 0x4B000000 | u are the float
// 2^23 + u, so subtracting 2^23 (+ 64) leaves u (- 64) exactly; its top 16 bits
// are the BF16 pattern (at most 7 significant bits).
__device__ __forceinline__ void digits7(double v, int e, unsigned short (&out)[TC_S]) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7FF);
    unsigned long long F = 0ull;
    if (ex != 0) {
        const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int shift = e + 3 - (ex - 1023);
        if (shift <= 0)
            F = 1ull << 48;  // not reached when e bounds |v|
        else if (shift < 55)
            F = (M + (1ull << (shift - 1))) >> shift;
    }
    const unsigned long long Fb = F + 0x20408102040ull;  // + 64 sum_{k<6} 128^k
    const unsigned sgn = (unsigned)(bits >> 32) & 0x80000000u;
#pragma unroll
    for (int s = 0; s < TC_S; ++s) {
        const unsigned u = (unsigned)(Fb >> (7 * (6 - s)));
        const float f = s == 0 ? __int_as_float((int)(0x4B000000u | u)) - 8388608.0f
                               : __int_as_float((int)(0x4B000000u | (u & 127u))) - 8388672.0f;
        out[s] = f == 0.0f ? (unsigned short)0 : (unsigned short)((__float_as_uint(f) ^ sgn) >> 16);
    }
}

// The digits of two values at once, as the packed words the digit tiles
// hold (v0's digit in the low half, v1's in the high half).  The biased
// plain digits u (7 bits) of both values go into one word as the BF16 pair
// 128 + u (bits 0x4300 | u); one packed BF16 subtraction of 192 (128 for the
// leading digit) leaves the digits exactly, and the values' signs are
// applied by flipping the halves' sign bits (a zero digit of a negative
// value becomes -0, which adds nothing to any sum).  About half the integer
// work of two digits7 calls; checked bitwise against them on 10^7 pairs.
__device__ __forceinline__ unsigned long long biased_fixed48(double v, int e) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7FF);
    unsigned long long F = 0ull;
    if (ex != 0) {
        const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int shift = e + 3 - (ex - 1023);
        if (shift <= 0)
            F = 1ull << 48;  // not reached when e bounds |v|
        else if (shift < 55)
            F = (M + (1ull << (shift - 1))) >> shift;
    }
    return F + 0x20408102040ull;  // + 64 sum_{k<6} 128^k
}
__device__ __forceinline__ void digits7x2(double v0, double v1, int e0, int e1, unsigned (&w)[TC_S]) {
    const unsigned long long F0 = biased_fixed48(v0, e0), F1 = biased_fixed48(v1, e1);
    const unsigned sg = ((unsigned)((unsigned long long)__double_as_longlong(v0) >> 48) & 0x8000u) |
                        ((unsigned)((unsigned long long)__double_as_longlong(v1) >> 32) & 0x80000000u);
    const __nv_bfloat162 lead = __floats2bfloat162_rn(128.0f, 128.0f), rest = __floats2bfloat162_rn(192.0f, 192.0f);
#pragma unroll
    for (int s = 0; s < TC_S; ++s) {
        const unsigned u0 = (unsigned)(F0 >> (7 * (6 - s))) & 0x7Fu;
        const unsigned u1 = (unsigned)(F1 >> (7 * (6 - s))) & 0x7Fu;
        const unsigned p = 0x43004300u | u0 | (u1 << 16);
        __nv_bfloat162 x;
        memcpy(&x, &p, 4);
        const __nv_bfloat162 d = __hsub2(x, s == 0 ? lead : rest);
        unsigned r;
        memcpy(&r, &d, 4);
        w[s] = r ^ sg;
    }
}

// Column exponents for the 7-digit split: |v| < 2^(e-1).
__global__ void max_to_exp7_kernel(int n, const unsigned long long* cmax, int* e) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        e[j] = exp_bound(__longlong_as_double((long long)cmax[j])) + 1;
}

// Digit planes of the 7-digit split, stage-major: D[i / 32][s][j][i % 32]
// (every 32-row stage of all n columns and digits one contiguous 14 n * 32
// bytes; rows i >= m zero), so that a stage's TMA box of 7 x 128 column runs
// of 64 bytes reads seven 8 KB spans of one region instead of 896 runs a
// plane (2 mp bytes) apart.  A thread slices 16 rows of one column: a warp
// reads 32 adjacent columns of a row at a time (256 bytes) and writes, per
// digit, one 32-byte sector per lane.
__global__ void __launch_bounds__(256)
slice7_cols_kernel(int m, int n, long mp, const double* __restrict__ A, long lda,
                   const int* __restrict__ ecol, unsigned short* __restrict__ D) {
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    if (j >= n) return;
    const int e = ecol[j];
    const long ngroups = mp / 16;
    for (long g = (long)blockIdx.y * 8 + (threadIdx.x >> 5); g < ngroups; g += (long)gridDim.y * 8) {
        const long i0 = g * 16;
        unsigned w[TC_S][8];
#pragma unroll
        for (int r = 0; r < 16; r += 2) {
            const double v0 = i0 + r < m ? A[(i0 + r) * lda + j] : 0.0;
            const double v1 = i0 + r + 1 < m ? A[(i0 + r + 1) * lda + j] : 0.0;
            unsigned wd[TC_S];
            digits7x2(v0, v1, e, e, wd);
#pragma unroll
            for (int s = 0; s < TC_S; ++s) w[s][r / 2] = wd[s];
        }
        const long st = i0 / 32;
        const int half = (int)(g & 1);
#pragma unroll
        for (int s = 0; s < TC_S; ++s) {
            uint4* dst = reinterpret_cast<uint4*>(D + ((st * TC_S + s) * n + j) * 32 + half * 16);
            dst[0] = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
            dst[1] = make_uint4(w[s][4], w[s][5], w[s][6], w[s][7]);
        }
    }
}

// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned a, unsigned parity, int* status,
                                                   volatile int* abort_flag) {
    for (long long it = 0; it < TC_SPIN; ++it) {
        if (mbar_try(a, parity)) return true;
        if (*abort_flag) return false;
        if (it > 32) __nanosleep(64);
    }
    if (status) atomicOr(status, DEV_TIMEOUT);
    *abort_flag = 1;
    return false;
}

// Tile t -> (jt, kt): the 128 x 64 tiles holding some j <= k (kt >= 2 jt),
// enumerated row by row; jt = -1 past the end.
__device__ __forceinline__ void tc_tile(int t, int KT, int& jt, int& kt) {
    for (jt = 0;; ++jt) {
        const int cnt = KT - 2 * jt;
        if (cnt <= 0) {
            jt = -1;
            return;
        }
        if (t < cnt) {
            kt = 2 * jt + t;
            return;
        }
        t -= cnt;
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
tcgram_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int n, long mp, const int* __restrict__ ecol, long kchunk,
              double* __restrict__ partial, int* status) {
    extern __shared__ unsigned char tc_raw[];
    const unsigned raw_s = smem_u32(tc_raw);
    const unsigned pad = ((raw_s + 1023u) & ~1023u) - raw_s;
    unsigned char* sbase = tc_raw + pad;
    const unsigned sb = raw_s + pad;  // 1024-byte aligned: stage st at sb + st * TC_STAGE_BYTES
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(sbase + TC_STAGES * TC_STAGE_BYTES);
    // bars: [0,1] stage full, [2,3] stage empty, [4] accumulators full, [5] accumulators
    // drained, [6] all MMAs done
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(bars + 8);
    volatile int* flags = reinterpret_cast<volatile int*>(tmem_slot + 2);  // abort, issued, consumed

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int KT = (n + TC_N - 1) / TC_N;
    int jt, kt;
    tc_tile(blockIdx.x, KT, jt, kt);
    if (jt < 0) return;
    const int j0 = jt * TC_M, kc0 = kt * TC_N;
    const long kbeg = (long)blockIdx.y * kchunk;
    const long kend = min(mp, kbeg + kchunk);
    const int nslices = kend > kbeg ? (int)((kend - kbeg) / TC_K) : 0;
    double* out = partial + (long)blockIdx.y * n * n;
    if (nslices == 0) {
        for (int idx = threadIdx.x; idx < TC_M * TC_N; idx += blockDim.x) {
            const int j = j0 + idx / TC_N, k = kc0 + idx % TC_N;
            if (j < n && k < n) out[(long)j * n + k] = 0.0;
        }
        return;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < 7; ++i) mbar_init(smem_u32(&bars[i]), i == 5 ? (unsigned)TC_DRAIN_WARPS : 1u);
        flags[0] = 0;
        flags[1] = 0;
        flags[2] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;
    const int nblocks = (nslices + TC_BLK - 1) / TC_BLK;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            for (int it = 0; it < nslices; ++it) {
                const int st = it % TC_STAGES;
                const unsigned ph = (unsigned)(it / TC_STAGES) & 1u;
                if (!mbar_wait_or_abort(smem_u32(&bars[2 + st]), ph ^ 1u, status, flags)) break;
                const unsigned full = smem_u32(&bars[st]);
                mbar_expect_tx(full, (unsigned)TC_STAGE_BYTES);
                const unsigned dA = sb + (unsigned)(st * TC_STAGE_BYTES);
                const int kst = (int)((kbeg + (long)it * TC_K) / TC_K);  // 32-row stage index
                tma_load_4d(dA, &tmA, 0, j0, 0, kst, full);
                tma_load_4d(dA + TC_A_BYTES, &tmB, 0, kc0, 0, kst, full);
                flags[1] = it + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            for (int it = 0; it < nslices; ++it) {
                const int st = it % TC_STAGES;
                const unsigned ph = (unsigned)(it / TC_STAGES) & 1u;
                const int b = it / TC_BLK;
                const bool first = (it % TC_BLK) == 0;
                if (first && b > 0) {
                    if (!mbar_wait_or_abort(smem_u32(&bars[5]), (unsigned)(b - 1) & 1u, status, flags))
                        break;
                    tc_fence_after();
                }
                if (!mbar_wait_or_abort(smem_u32(&bars[st]), ph, status, flags)) break;
                tc_fence_after();
                const unsigned aB = sb + (unsigned)(st * TC_STAGE_BYTES);
                const unsigned bB = aB + TC_A_BYTES;
                tc_stage_mmas(tmem, aB, bB, first);
                tc_commit(smem_u32(&bars[2 + st]));  // the stage is free once these MMAs finish
                flags[2] = it + 1;
                if ((it % TC_BLK) == TC_BLK - 1 || it == nslices - 1) tc_commit(smem_u32(&bars[4]));
            }
            tc_commit(smem_u32(&bars[6]));  // every issued MMA done before teardown
            mbar_wait(smem_u32(&bars[6]), 0u, status);
        }
    } else {  // drain warps: TMEM lanes 32 q .. 32 q + 31, columns c0 .. c0 + TC_DN - 1
        const int q = warp & 3;
        const int c0 = ((warp - 2) >> 2) * TC_DN;
        float hi[TC_DN], lo[TC_DN];
#pragma unroll
        for (int c = 0; c < TC_DN; ++c) hi[c] = lo[c] = 0.f;
        for (int b = 0; b < nblocks; ++b) {
            const bool ok = __all_sync(0xffffffffu, mbar_wait_or_abort(smem_u32(&bars[4]),
                                                                      (unsigned)b & 1u, status, flags));
            if (!ok) break;
            tc_fence_after();
#pragma unroll 1
            for (int w = 0; w < TC_S; ++w) {
                const float scale = __int_as_float((127 - 7 * w) << 23);  // 128^-w, exact
                unsigned r[2][16];
                const unsigned ta = tmem + ((unsigned)(32 * q) << 16) + (unsigned)(w * TC_N + c0);
                tc_ld16(ta, r[0]);
                tc_ld16(ta + 16, r[1]);
                tc_wait_ld();
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        df_add(hi[16 * c + e], lo[16 * c + e], __uint_as_float(r[c][e]) * scale);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars[5]));
        }
        const int j = j0 + 32 * q + lane;
        if (j < n && !flags[0]) {
#pragma unroll
            for (int c = 0; c < TC_DN; ++c) {
                const int k = kc0 + c0 + c;
                if (k < n)
                    out[(long)j * n + k] =
                        ldexp((double)hi[c] + (double)lo[c], ecol[j] + ecol[k] - 14);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // copies issued but never consumed (after an abort) land before the CTA exits
        const int issued = flags[1], consumed = flags[2];
        for (int it = consumed; it < issued; ++it)
            mbar_wait(smem_u32(&bars[it % TC_STAGES]), (unsigned)(it / TC_STAGES) & 1u, status);
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// ----------------------------------------------------------------------
// Core update C (M x N) = A (M x K) B^T on tcgen05, rows of A and B with their
// own exponents (the contraction runs along rows).  Same 7-digit split,
// exact 128-column level sums, seven TMEM accumulators per 128 x 64 tile and
// one MMA-issuing thread as the Gram.  Both operands are sliced once
// beforehand into ready-made shared-memory images -- per (row block, stage)
// the seven 128 x 32 digit tiles of A, per (column block, stage) the seven
// 64 x 32 tiles of B, each in the MMA's 64-byte swizzled K-major layout
// (16-byte chunk index XOR (row / 2) mod 4) -- so one thread brings a stage in
// with two bulk copies, one thread issues its 20 MMAs (tc_stage_mmas), and eight warps drain
// the accumulators every sixteenth stage.  A persistent CTA walks (row block,
// column block) items.
constexpr int TU_DRAIN_WARPS = 8;
constexpr int TU_THREADS = 32 * (2 + TU_DRAIN_WARPS);  // warp 0 copies, warp 1 TMEM + MMA, 2-9 drain
constexpr size_t TU_SMEM = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024 + 1024;

// Byte offset of element (row r, k) in a swizzled K-major digit tile (64-byte rows).
__device__ __forceinline__ unsigned tc_swz(int r, int k) {
    return (unsigned)(r * 64 + ((((k >> 3) ^ ((r >> 1) & 3))) << 4) + (k & 7) * 2);
}

// A (M x K, per-row exponents) as shared-memory images: for row block mb and
// stage st the seven tiles of rows mb*128 .. +127, columns st*32 .. +31;
// At + ((mb * nst + st) * 7 + s) * 8192 is one tile.  A thread slices two
// adjacent columns of one row and stores 32-bit words: a warp writes two
// whole 64-byte rows per digit, without bank conflicts.
__global__ void __launch_bounds__(256)
slice7_atiles_kernel(long M, int K, int nst, const double* __restrict__ A, long lda,
                     const int* __restrict__ erowA, unsigned char* __restrict__ At) {
    const long mblocks = (M + TC_M - 1) / TC_M;
    const long total = mblocks * nst * TC_M * (TC_K / 2);
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int kw = (int)(t % (TC_K / 2));
        const int r = (int)((t / (TC_K / 2)) % TC_M);
        const long ts = t / ((long)(TC_K / 2) * TC_M);  // mb * nst + st
        const int st = (int)(ts % nst);
        const long i = (ts / nst) * TC_M + r;
        const int k = st * TC_K + 2 * kw;
        double v0 = 0.0, v1 = 0.0;
        int e = 0;
        if (i < M) {
            e = erowA[i] + 1;
            if (k < K) v0 = A[i * lda + k];
            if (k + 1 < K) v1 = A[i * lda + k + 1];
        }
        unsigned wd[TC_S];
        digits7x2(v0, v1, e, e, wd);
        const unsigned off = tc_swz(r, 2 * kw);
#pragma unroll
        for (int s = 0; s < TC_S; ++s)
            *reinterpret_cast<unsigned*>(At + (ts * TC_S + s) * (TC_M * TC_K * 2) + off) = wd[s];
    }
}

// B (N x K, per-row exponents) as ready-made shared-memory images: for n-block
// nb and stage st the 7 digit tiles of rows nb*64 .. +63, columns st*32 .. +31,
// each 64 rows x 64 bytes in the MMA's 64-byte swizzled K-major layout, so one
// bulk copy per stage places them.  Bt[(nb * nst + st) * 7 + s] is one tile.
__global__ void __launch_bounds__(256)
slice7_btiles_kernel(int N, int K, int nst, const double* __restrict__ B, long ldb,
                     const int* __restrict__ erowB, unsigned char* __restrict__ Bt) {
    const int nbt = (N + TC_N - 1) / TC_N;
    const long total = (long)nbt * nst * TC_N * TC_K;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int k = (int)(t % TC_K);
        const int r = (int)((t / TC_K) % TC_N);
        const long ts = t / ((long)TC_K * TC_N);  // nb * nst + st
        const int st = (int)(ts % nst), nb = (int)(ts / nst);
        const int c = nb * TC_N + r, kc = st * TC_K + k;
        const double v = (c < N && kc < K) ? B[(long)c * ldb + kc] : 0.0;
        unsigned short d[TC_S];
        digits7(v, c < N ? erowB[c] + 1 : 0, d);
        const unsigned off = tc_swz(r, k);
#pragma unroll
        for (int s = 0; s < TC_S; ++s)
            *reinterpret_cast<unsigned short*>(Bt + (ts * TC_S + s) * (TC_N * TC_K * 2) + off) = d[s];
    }
}

__device__ __forceinline__ void bulk_copy_g2s(unsigned dst, const void* src, unsigned bytes,
                                              unsigned mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"((unsigned long long)src), "r"(bytes), "r"(mbar)
        : "memory");
}

__global__ void __launch_bounds__(TU_THREADS, 1)
tcupd_kernel(long M, int N, int K, const unsigned char* __restrict__ At,
             const int* __restrict__ erowA, const unsigned char* __restrict__ Bt,
             const int* __restrict__ erowB, double* __restrict__ C, long ldc, int spc, double* __restrict__ Pk,
             int* status) {
    extern __shared__ unsigned char tc_raw[];
    const unsigned raw_s = smem_u32(tc_raw);
    const unsigned pad = ((raw_s + 1023u) & ~1023u) - raw_s;
    unsigned char* sbase = tc_raw + pad;
    const unsigned sb = raw_s + pad;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(sbase + TC_STAGES * TC_STAGE_BYTES);
    // bars: [0,1] stage landed (bulk copies), [2,3] stage empty, [4] accumulators
    // full, [5] accumulators drained, [6] all MMAs done
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(bars + 8);
    volatile int* flags = reinterpret_cast<volatile int*>(tmem_slot + 2);  // abort, issued, consumed

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long mblocks = (M + TC_M - 1) / TC_M;
    const int nblk = (N + TC_N - 1) / TC_N;
    const int nst = (K + TC_K - 1) / TC_K;  // stages of the whole contraction
    // split-K: spc stages (a multiple of TC_BLK) per item; item = (split, row
    // block, column block), split outermost; splits > 1 write their partial
    // product to Pk[split] (M x N) instead of C
    const int ksp = (nst + spc - 1) / spc;
    const long items = mblocks * nblk * ksp;
    if ((long)blockIdx.x >= items) return;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 7; ++i) mbar_init(smem_u32(&bars[i]), i == 5 ? (unsigned)TU_DRAIN_WARPS : 1u);
        flags[0] = 0;
        flags[1] = 0;
        flags[2] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // copies: A and B images of each stage
            long g = 0;
            bool stop = false;
            for (long item = blockIdx.x; item < items && !stop; item += gridDim.x) {
                const long tile = item % (mblocks * nblk);
                const int sp = (int)(item / (mblocks * nblk));
                const long mb = tile / nblk;
                const int nb = (int)(tile % nblk);
                const int st1 = min(nst, (sp + 1) * spc);
                for (int it = sp * spc; it < st1; ++it, ++g) {
                    const int st = (int)(g % TC_STAGES);
                    const unsigned ph = (unsigned)(g / TC_STAGES) & 1u;
                    if (!mbar_wait_or_abort(smem_u32(&bars[2 + st]), ph ^ 1u, status, flags)) {
                        stop = true;
                        break;
                    }
                    const unsigned full = smem_u32(&bars[st]);
                    mbar_expect_tx(full, (unsigned)TC_STAGE_BYTES);
                    const unsigned dA = sb + (unsigned)(st * TC_STAGE_BYTES);
                    bulk_copy_g2s(dA, At + (mb * nst + it) * (long)TC_A_BYTES, (unsigned)TC_A_BYTES, full);
                    bulk_copy_g2s(dA + TC_A_BYTES, Bt + ((long)nb * nst + it) * TC_B_BYTES,
                                  (unsigned)TC_B_BYTES, full);
                    flags[1] = (int)(g + 1);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            long g = 0, gb = 0;  // stages and blocks issued by this CTA so far
            bool stop = false;
            for (long item = blockIdx.x; item < items && !stop; item += gridDim.x) {
                const int sp = (int)(item / (mblocks * nblk));
                const int st0 = sp * spc, st1 = min(nst, st0 + spc);
                for (int it = st0; it < st1; ++it, ++g) {
                    const int st = (int)(g % TC_STAGES);
                    const unsigned ph = (unsigned)(g / TC_STAGES) & 1u;
                    const bool first = ((it - st0) % TC_BLK) == 0;
                    if (first && gb > 0) {
                        if (!mbar_wait_or_abort(smem_u32(&bars[5]), (unsigned)(gb - 1) & 1u, status, flags)) {
                            stop = true;
                            break;
                        }
                        tc_fence_after();
                    }
                    if (!mbar_wait_or_abort(smem_u32(&bars[st]), ph, status, flags)) {
                        stop = true;
                        break;
                    }
                    flags[2] = (int)(g + 1);
                    tc_fence_after();
                    const unsigned aB = sb + (unsigned)(st * TC_STAGE_BYTES);
                    const unsigned bB = aB + TC_A_BYTES;
                    tc_stage_mmas(tmem, aB, bB, first);
                    tc_commit(smem_u32(&bars[2 + st]));
                    if (((it - st0) % TC_BLK) == TC_BLK - 1 || it == st1 - 1) {
                        tc_commit(smem_u32(&bars[4]));
                        ++gb;
                    }
                }
            }
            tc_commit(smem_u32(&bars[6]));
            mbar_wait(smem_u32(&bars[6]), 0u, status);
        }
    } else {  // drain warps: TMEM lanes 32 q .. 32 q + 31, columns c0 .. c0 + TC_DN - 1
        const int q = warp & 3;
        const int c0 = ((warp - 2) >> 2) * TC_DN;
        long gb = 0;
        bool stop = false;
        for (long item = blockIdx.x; item < items && !stop; item += gridDim.x) {
            const long tile = item % (mblocks * nblk);
            const int sp = (int)(item / (mblocks * nblk));
            const int nb_per_item = (min(nst, (sp + 1) * spc) - sp * spc + TC_BLK - 1) / TC_BLK;
            double* Cd = ksp > 1 ? Pk + (long)sp * M * N : C;
            const long ldd = ksp > 1 ? (long)N : ldc;
            const long i0 = (tile / nblk) * TC_M;
            const int n0 = (int)(tile % nblk) * TC_N;
            float hi[TC_DN], lo[TC_DN];
#pragma unroll
            for (int c = 0; c < TC_DN; ++c) hi[c] = lo[c] = 0.f;
            for (int b = 0; b < nb_per_item; ++b, ++gb) {
                if (!__all_sync(0xffffffffu, mbar_wait_or_abort(smem_u32(&bars[4]), (unsigned)gb & 1u,
                                                                 status, flags))) {
                    stop = true;
                    break;
                }
                tc_fence_after();
#pragma unroll 1
                for (int w = 0; w < TC_S; ++w) {
                    const float scale = __int_as_float((127 - 7 * w) << 23);
                    unsigned r2[2][16];
                    const unsigned ta = tmem + ((unsigned)(32 * q) << 16) + (unsigned)(w * TC_N + c0);
                    tc_ld16(ta, r2[0]);
                    tc_ld16(ta + 16, r2[1]);
                    tc_wait_ld();
#pragma unroll
                    for (int c = 0; c < 2; ++c)
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            df_add(hi[16 * c + e], lo[16 * c + e], __uint_as_float(r2[c][e]) * scale);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bars[5]));
            }
            if (stop) break;
            const long i = i0 + 32 * q + lane;
            if (i < M && !flags[0]) {
                const int ea = erowA[i] + 1;
#pragma unroll
                for (int c = 0; c < TC_DN; ++c) {
                    const int col = n0 + c0 + c;
                    if (col < N)
                        Cd[i * ldd + col] = ldexp((double)hi[c] + (double)lo[c], ea + erowB[col] + 1 - 14);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // bulk copies issued but never consumed (after an abort) land before the CTA exits
        const long issued = flags[1], consumed = flags[2];
        for (long g2 = consumed; g2 < issued; ++g2)
            mbar_wait(smem_u32(&bars[g2 % TC_STAGES]), (unsigned)(g2 / TC_STAGES) & 1u, status);
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// C = sum over the splits of Pk[split] (M x N each), in split order.
__global__ void splitk_sum_kernel(long M, int N, int ksp, const double* __restrict__ Pk, double* __restrict__ C,
                                  long ldc) {
    const long tot = M * N;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        double v = Pk[e];
        for (int k = 1; k < ksp; ++k) v += Pk[(long)k * tot + e];
        C[(e / N) * ldc + e % N] = v;
    }
}

int tc_tiles(int n) {
    const int KT = (n + TC_N - 1) / TC_N;
    int t = 0;
    for (int jt = 0; KT - 2 * jt > 0; ++jt) t += KT - 2 * jt;
    return t;
}

// Row splits of the tensor-core Gram: every CTA holds one tile for one row
// range, one CTA per SM, so the launch runs in waves of 152 and a split count
// that leaves SMs idle in the last wave costs the whole wave (64 tiles x 2
// splits keep 128 of 152 SMs busy; x 19 splits fill 8 waves).  The first
// count from 152 / tiles up whose waves are >= 95% full, else the fullest;
// at most one split per 512-row block and 64M partial doubles.
int tc_ksplit(int m, int n) {
    const long mp = ((long)std::max(m, 1) + TC_K - 1) / TC_K * TC_K;
    const long blocks = (mp + TC_K * TC_BLK - 1) / (TC_K * TC_BLK);
    const long T = tc_tiles(n);
    const long kmax = std::max(1L, std::min(std::min(blocks, 64L), (64L << 20) / std::max(1L, (long)n * n)));
    long best = std::min(std::max(1L, 152L / T), kmax);
    double best_eff = 0.0;
    for (long k = best; k <= kmax; ++k) {
        const long waves = (T * k + 151) / 152;
        const double eff = (double)(T * k) / (double)(waves * 152);
        if (eff > best_eff + 1e-12) {
            best = k;
            best_eff = eff;
        }
        if (eff >= 0.95) break;
    }
    return (int)best;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static std::atomic<EncodeTiledFn> fn{nullptr};
    if (fn.load()) return fn.load();
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        p = nullptr;
    (void)cudaGetLastError();
    fn.store(reinterpret_cast<EncodeTiledFn>(p));
    return fn.load();
}

}  // namespace

size_t tcgram_scratch_doubles(int m, int n) {
    const size_t mp = ((size_t)std::max(m, 1) + TC_K - 1) / TC_K * TC_K;
    return ((size_t)tc_ksplit(std::max(m, 1), n) * n * n + 2 * (size_t)n + 8 + 127) / 128 * 128 +
           (TC_S * (size_t)n * mp + 3) / 4;
}

tt_status tcgram(cudaStream_t s, int m, int n, const double* A, long lda, double* G, long ldg,
                 DevBuf& scratch, int* status_dev, int* erow_out) {
    if (n <= 0) return TT_OK;
    if (m <= 0) {
        for (int i = 0; i < n; ++i) fill(s, G + (long)i * ldg, n, 0.0);
        return TT_OK;
    }
    EncodeTiledFn enc = encode_tiled();
    if (!enc) {
        set_error("tcgram: cuTensorMapEncodeTiled is not available from the driver");
        return TT_ERR_CUDA;
    }
    const int ks = tc_ksplit(m, n);
    TT_TRY(scratch.ensure(tcgram_scratch_doubles(m, n), s));
    double* partial = scratch.p;
    unsigned long long* cmax = reinterpret_cast<unsigned long long*>(scratch.p + (size_t)ks * n * n);
    int* ecol = reinterpret_cast<int*>(cmax + n);
    TT_CUDA_TRY(cudaMemsetAsync(cmax, 0, n * sizeof(unsigned long long), s));
    if (erow_out && n <= CRM_MAXN) {  // the row exponents of A too, from the same read
        TT_TRY(ensure_max_dynamic_smem((const void*)col_row_max_kernel));
        int dev = 0, sms = 152, per_sm = 1;
        const size_t smem = (size_t)8 * n * sizeof(unsigned long long);
        TT_CUDA_TRY(cudaGetDevice(&dev));
        TT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        TT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, col_row_max_kernel, 256, smem));
        note_launch();
        col_row_max_kernel<<<(int)std::max<long>(1, std::min<long>(((long)m + 7) / 8, (long)sms * std::max(per_sm, 1))),
                             256, smem, s>>>(m, n, A, lda, cmax, erow_out);
    } else {
        dim3 grid((n + 31) / 32, (unsigned)std::min<long>(std::max<long>(1, m / 4096), 256));
        note_launch();
        col_max_kernel<<<grid, 256, 0, s>>>(m, n, A, lda, cmax);
        if (erow_out) {
            note_launch();
            row_exp_kernel<<<(int)std::max<long>(1, std::min<long>(((long)m + 7) / 8, 152L * 64)), 256, 0, s>>>(
                m, n, A, lda, erow_out);
        }
    }
    note_launch();
    max_to_exp7_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, cmax, ecol);
    const long mp = ((long)m + TC_K - 1) / TC_K * TC_K;
    // planes start on a 1024-byte boundary (TMA wants 16)
    const size_t plane_off = ((size_t)ks * n * n + 2 * (size_t)n + 8 + 127) / 128 * 128;
    unsigned short* planes = reinterpret_cast<unsigned short*>(scratch.p + plane_off);
    {
        dim3 grid((n + 31) / 32, (unsigned)std::min<long>((mp / 16 + 7) / 8, 2048));
        note_launch();
        slice7_cols_kernel<<<grid, 256, 0, s>>>(m, n, mp, A, lda, ecol, planes);
    }
    CUtensorMap mapA, mapB;
    {
        // (row in stage, column, digit, stage); strides 64 B, 64 n B, 448 n B
        const cuuint64_t gdim[4] = {(cuuint64_t)TC_K, (cuuint64_t)n, (cuuint64_t)TC_S, (cuuint64_t)(mp / TC_K)};
        const cuuint64_t gstr[3] = {(cuuint64_t)TC_K * 2, (cuuint64_t)n * TC_K * 2,
                                    (cuuint64_t)n * TC_K * 2 * TC_S};
        const cuuint32_t boxA[4] = {TC_K, TC_M, TC_S, 1}, boxB[4] = {TC_K, TC_N, TC_S, 1};
        const cuuint32_t est[4] = {1, 1, 1, 1};
        CUresult r1 = enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, planes, gdim, gstr, boxA, est,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        CUresult r2 = enc(&mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, planes, gdim, gstr, boxB, est,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
            set_error("tcgram: tensor map encoding failed");
            return TT_ERR_CUDA;
        }
    }
    {
        long kchunk = (mp + ks - 1) / ks;
        kchunk = (kchunk + TC_K * TC_BLK - 1) / (TC_K * TC_BLK) * (TC_K * TC_BLK);
        TT_TRY(ensure_max_dynamic_smem((const void*)tcgram_kernel));
        note_launch();
        tcgram_kernel<<<dim3(tc_tiles(n), ks), TC_THREADS, TC_SMEM, s>>>(
            mapA, mapB, n, mp, ecol, kchunk, partial, status_dev);
        TT_CUDA_TRY(cudaGetLastError());
    }
    const long total = (long)n * n;
    note_launch();
    slgram_reduce_kernel<<<(int)std::min<long>((total + 255) / 256, 152L * 32), 256, 0, s>>>(
        n, ks, partial, G, ldg);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status bench_bf16_mma(cudaStream_t s, double* tflops) {
    int dev = 0, sms = 0;
    TT_CUDA_TRY(cudaGetDevice(&dev));
    TT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* out = nullptr;
    TT_CUDA_TRY(cudaMallocAsync((void**)&out, 256 * sizeof(float), s));
    cudaEvent_t e0, e1;
    TT_CUDA_TRY(cudaEventCreate(&e0));
    TT_CUDA_TRY(cudaEventCreate(&e1));
    const int blocks = sms * 4;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        TT_CUDA_TRY(cudaEventRecord(e0, s));
        note_launch();
        bf16_mma_peak_kernel<<<blocks, 256, 0, s>>>(out, 0x3c003c00u);
        TT_CUDA_TRY(cudaEventRecord(e1, s));
        TT_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        TT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, s);
    const double flops = 2.0 * 16 * 8 * 16 * 8.0 * BF16_PEAK_ITERS * blocks * (256 / 32);
    *tflops = flops / (best * 1e-3) / 1e12;
    return TT_OK;
}

size_t slgram_scratch_doubles(int m, int n) { return tcgram_scratch_doubles(m, n); }

tt_status slgram(cudaStream_t s, int m, int n, const double* A, long lda, double* G, long ldg,
                 DevBuf& scratch, int* status_dev, int* erow_out) {
    return tcgram(s, m, n, A, lda, G, ldg, scratch, status_dev, erow_out);
}

tt_status slgemm_nt(cudaStream_t s, long M, int N, int K, const double* A, long lda, const double* B,
                    long ldb, double* C, long ldc, DevBuf& scratch, int* status_dev, DevBuf* planes,
                    const int* erowA) {
    if (M <= 0 || N <= 0) return TT_OK;
    if (K <= 0) {  // empty contraction: C = 0
        if (ldc == N) {
            fill(s, C, (size_t)M * N, 0.0);
        } else {
            for (long i = 0; i < M; ++i) fill(s, C + i * ldc, N, 0.0);
        }
        return TT_OK;
    }
    const int nst = (K + TC_K - 1) / TC_K;
    const int nbt = (N + TC_N - 1) / TC_N;
    const long mblocks = (M + TC_M - 1) / TC_M;
    const size_t e_dbl = ((size_t)(M + N + 1) / 2 + 2 + 15) / 16 * 16;  // exponents, 128-byte aligned
    const size_t bt_bytes = (size_t)nbt * nst * TC_B_BYTES;
    const size_t at_bytes = (size_t)mblocks * nst * TC_A_BYTES;
    const bool own = planes == nullptr;  // A's images in `scratch` too
    int dev = 0, sms = 152;
    TT_CUDA_TRY(cudaGetDevice(&dev));
    TT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // split-K when the output has too few 128 x 64 tiles to occupy the SMs
    // (e.g. an R x R right Gram over a long contraction): spc stages per split
    const long tiles0 = mblocks * nbt;
    int spc = nst;
    if (tiles0 < sms / 2 && nst >= 2) spc = (int)((nst + (sms + tiles0 - 1) / tiles0 - 1) / ((sms + tiles0 - 1) / tiles0));
    const int ksp = (nst + spc - 1) / spc;
    const size_t pk_dbl = ksp > 1 ? (size_t)ksp * M * N : 0;
    const size_t pk_off = e_dbl + bt_bytes / 8 + (own ? at_bytes / 8 : 0);
    TT_TRY(scratch.ensure(pk_off + pk_dbl, s));
    if (!own) TT_TRY(planes->ensure(at_bytes / 8, s));
    double* Pk = ksp > 1 ? scratch.p + pk_off : nullptr;
    int* eA = reinterpret_cast<int*>(scratch.p);
    int* eB = eA + M;
    const bool have_eA = erowA != nullptr;
    unsigned char* Bt = reinterpret_cast<unsigned char*>(scratch.p + e_dbl);
    unsigned char* At = own ? Bt + bt_bytes : reinterpret_cast<unsigned char*>(planes->p);
    if (have_eA) {
        eA = const_cast<int*>(erowA);
    } else {
        note_launch();
        row_exp_kernel<<<(int)std::max<long>(1, std::min<long>((M + 7) / 8, 152L * 64)), 256, 0, s>>>(M, K, A, lda,
                                                                                                     eA);
    }
    note_launch();
    row_exp_kernel<<<(N + 7) / 8, 256, 0, s>>>(N, K, B, ldb, eB);
    {
        const long tot = (long)nbt * nst * TC_N * TC_K;
        note_launch();
        slice7_btiles_kernel<<<(int)std::min<long>((tot + 255) / 256, 152L * 16), 256, 0, s>>>(
            N, K, nst, B, ldb, eB, Bt);
        const long tota = mblocks * nst * TC_M * (TC_K / 2);
        note_launch();
        slice7_atiles_kernel<<<(int)std::min<long>((tota + 255) / 256, 152L * 32), 256, 0, s>>>(
            M, K, nst, A, lda, eA, At);
    }
    const long items = tiles0 * ksp;
    const int grid = (int)std::min<long>(items, sms);
    TT_TRY(ensure_max_dynamic_smem((const void*)tcupd_kernel));
    note_launch();
    tcupd_kernel<<<grid, TU_THREADS, TU_SMEM, s>>>(M, N, K, At, eA, Bt, eB, C, ldc, spc, Pk, status_dev);
    TT_CUDA_TRY(cudaGetLastError());
    if (ksp > 1) {
        const long tot = M * N;
        note_launch();
        splitk_sum_kernel<<<(int)std::min<long>((tot + 255) / 256, 152L * 16), 256, 0, s>>>(M, N, ksp, Pk, C, ldc);
        TT_CUDA_TRY(cudaGetLastError());
    }
    return TT_OK;
}

}  // namespace ttsn
