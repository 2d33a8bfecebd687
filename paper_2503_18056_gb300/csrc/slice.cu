// Mixed-precision contractions of the rounding (precision form): the left Gram
// G = A^T A and the core update C = A B^T on the BF16 tensor pipe with exact
// split products, for the contractions App. A.4 names as the dominant cost.
//
// Split.  Each FP64 operand is scaled by a power of two per column (Gram: the
// contraction runs over rows, so only columns may carry their own scale) or
// per row (update: rows i of A and rows c of B are not summed), so every scaled
// value lies in (-1, 1), and is cut into S signed base-256 digits:
//   a = 2^e sum_{s<S} d_s 256^-(s+1) + r,   |r| <= 2^e 256^-S / 2,
// balanced digits d_0 in [0, 256], d_1..d_5 in [-128, 127] (with a's sign).
// Every digit is exact in BF16.  A digit product is at most 2^16 and exact in
// FP32; the products of level w = s + t (weight 256^-(w+2)) summed over a
// 32-row block stay below 2^22, so the FP32 block sums are exact; then
// each block sum is scaled by 256^-w (exact) and added into a double-float
// accumulator (hi + lo in FP32, TwoSum + renormalisation: about 48 bits).  Levels
// with s + t >= S are dropped, so the result carries about 2^-8S relative to
// the column (row) scale: 21 BF16 products for S = 6, accurate to ~1e-13 of
// max|a| max|b| per term, against 2^-53 for FP64.  No FP64 arithmetic runs in
// the inner loop (GB300's FP64 pipe is ~1/70 of its FP32 pipe).
//
// Tiles: 64 x 64 outputs per CTA, four warps of 32 x 32, mma.sync m16n8k16
// bf16 with FP32 accumulators, shared-memory digit tiles [S][64][32] per
// operand (K-contiguous, XOR-swizzled for conflict-free fragment loads).  The Gram slices each
// column once into digit planes in global memory and streams them with a
// two-stage cp.async pipeline; the update GEMM produces digits on the fly
// (its B operand is small and its A tile is read by few CTAs).
#include <algorithm>
#include <atomic>

#include "internal.h"

namespace ttsn {

namespace {

constexpr int SL_S = 6;           // digits per value
constexpr int SL_BM = 64, SL_BN = 64, SL_BK = 32, SL_LD = 32;  // smem row = 32 bf16 = 64 B
constexpr int SL_THREADS = 128;

__device__ __forceinline__ unsigned short bf16_bits_of_int(int v) {
    // |v| <= 255: exact in bf16; take the top 16 bits of the fp32 value
    const float f = (float)v;
    return (unsigned short)(__float_as_uint(f) >> 16);
}

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

// Digits of v * 2^-e (|v| 2^-e < 1) into out[0..S), from the bit pattern with
// integer operations only.  |v| 2^(8S-e) = M 2^(ev-e-4) for S = 6 (M the 53-bit
// significand) is rounded to the nearest integer F (a right shift by
// e + 4 - ev >= 5 with rounding), then written in balanced base 256: digits
// d_1..d_5 in [-128, 127] and d_0 in [0, 256], F = sum_s d_s 256^(5-s), all
// carrying the sign of v.  Rounding and balanced digits make both the residual
// and the dropped high-level products zero-mean, so they do not bias sums of
// squares.  Every digit (|d| <= 256) is exact in BF16.  Subnormal inputs
// (|v| < 2^-1022) contribute zero digits.
__device__ __forceinline__ void digits(double v, int e, unsigned short (&out)[SL_S]) {
    static_assert(SL_S == 6, "fixed-point width is 8 * SL_S = 48 bits");
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7FF);
    unsigned long long F = 0ull;
    if (ex != 0) {
        const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int shift = e + 4 - (ex - 1023);
        if (shift <= 0)
            F = 1ull << 48;  // not reached when e bounds |v|; saturate at 2^48
        else if (shift < 55)
            F = (M + (1ull << (shift - 1))) >> shift;
    }
    const unsigned short sign = (unsigned short)((bits >> 48) & 0x8000u);
    int d[SL_S];
#pragma unroll
    for (int s = SL_S - 1; s >= 1; --s) {
        int x = (int)(F & 0xFFull);
        F >>= 8;
        if (x >= 128) {
            x -= 256;
            F += 1;
        }
        d[s] = x;
    }
    d[0] = (int)F;  // 0 .. 256
#pragma unroll
    for (int s = 0; s < SL_S; ++s) {
        const int x = d[s];
        if (x == 0) {
            out[s] = 0;
        } else {
            const unsigned short b = bf16_bits_of_int(x < 0 ? -x : x);
            out[s] = (unsigned short)(b | (x < 0 ? (sign ^ 0x8000u) : sign));
        }
    }
}

// Exponent e with |v| < 2^e for the largest |v| (0 for a zero maximum).
__device__ __forceinline__ int exp_bound(double vmax) {
    if (!(vmax > 0.0)) return 0;
    return ilogb(vmax) + 1;
}

__global__ void col_max_kernel(int m, int n, const double* __restrict__ A, long lda,
                               unsigned long long* cmax) {
    // block: 32 columns x (blockDim/32) row lanes; grid.y splits the rows
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int rlane = threadIdx.x >> 5, rstride = blockDim.x >> 5;
    const long rows_per = ((long)m + gridDim.y - 1) / gridDim.y;
    const long r0 = blockIdx.y * rows_per, r1 = min((long)m, r0 + rows_per);
    double mx = 0.0;
    if (j < n)
        for (long i = r0 + rlane; i < r1; i += rstride) mx = fmax(mx, fabs(A[i * lda + j]));
    if (j < n && mx > 0.0) atomicMax(cmax + j, (unsigned long long)__double_as_longlong(mx));
}

__global__ void max_to_exp_kernel(int n, const unsigned long long* cmax, int* e) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        e[j] = exp_bound(__longlong_as_double((long long)cmax[j]));
}

__global__ void row_exp_kernel(long m, int n, const double* __restrict__ A, long lda, int* e) {
    const int lane = threadIdx.x & 31;
    const long warps = (long)gridDim.x * (blockDim.x >> 5);
    for (long i = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += warps) {
        double mx = 0.0;
        for (int j = lane; j < n; j += 32) mx = fmax(mx, fabs(A[i * lda + j]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) e[i] = exp_bound(mx);
    }
}

// Shared-memory digit tiles: [S][64 rows][32] bf16, row = output index, col = K.
// Rows are 64 bytes (16 words); 32-bit word w of row r is stored at word
// w ^ 4 ((r >> 1) & 3), so the fragment loads of 8 rows x 4 words hit 32
// distinct banks, and 16-byte chunks stay contiguous (the XOR is a multiple of
// 4 words).
struct SlTiles {
    unsigned short d[SL_S][SL_BM][SL_LD];
};
__device__ __forceinline__ int swz_word(int r, int w) { return w ^ (((r >> 1) & 3) << 2); }
__device__ __forceinline__ int swz_elem(int r, int k) { return (swz_word(r, k >> 1) << 1) | (k & 1); }
__device__ __forceinline__ unsigned ld_word(const SlTiles& T, int s, int r, int k) {
    return *reinterpret_cast<const unsigned*>(&T.d[s][r][swz_word(r, k >> 1) << 1]);
}

// Fragment loads and the 21 digit products of one 32-row block for a warp's
// 32 x 32 sub-tile, drained level by level into the double-float accumulators.
__device__ __forceinline__ void block_products(const SlTiles& TA, const SlTiles& TB, int wm, int wn,
                                               int lane, float (&hi)[2][4][4], float (&lo)[2][4][4]) {
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll 1
    for (int w = 0; w < SL_S; ++w) {
        float acc[2][4][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
#pragma unroll 1
        for (int s = 0; s <= w; ++s) {
            const int t = w - s;
#pragma unroll
            for (int kk = 0; kk < SL_BK; kk += 16) {
                unsigned af[2][4], bfr[4][2];
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    const int r0 = wm + mi * 16 + g;
                    const int c0 = kk + t4 * 2;
                    af[mi][0] = ld_word(TA, s, r0, c0);
                    af[mi][1] = ld_word(TA, s, r0 + 8, c0);
                    af[mi][2] = ld_word(TA, s, r0, c0 + 8);
                    af[mi][3] = ld_word(TA, s, r0 + 8, c0 + 8);
                }
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) {
                    const int nn = wn + ni * 8 + g;
                    const int k0 = kk + t4 * 2;
                    bfr[ni][0] = ld_word(TB, t, nn, k0);
                    bfr[ni][1] = ld_word(TB, t, nn, k0 + 8);
                }
#pragma unroll
                for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                    for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
            }
        }
        const float scale = __int_as_float((127 - 8 * w) << 23);  // 256^-w, exact
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) df_add(hi[a][b][c], lo[a][b][c], acc[a][b][c] * scale);
    }
}

// C (M x N) = A (M x K) B^T (B: N x K); both row-major FP64 with per-row exponents.
__global__ void __launch_bounds__(SL_THREADS)
slgemm_nt_kernel(int M, int N, int K, const double* __restrict__ A, long lda,
                 const int* __restrict__ erowA, const double* __restrict__ B, long ldb,
                 const int* __restrict__ erowB, double* __restrict__ C, long ldc) {
    extern __shared__ unsigned char smraw[];
    SlTiles& TA = *reinterpret_cast<SlTiles*>(smraw);
    SlTiles& TB = *reinterpret_cast<SlTiles*>(smraw + sizeof(SlTiles));
    const long M0 = (long)blockIdx.y * SL_BM;
    const int N0 = blockIdx.x * SL_BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float hi[2][4][4], lo[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) hi[a][b][c] = lo[a][b][c] = 0.f;
    for (int k0 = 0; k0 < K; k0 += SL_BK) {
        // element (row r, k): coalesced along k; stored [r][k]
#pragma unroll 4
        for (int it = 0; it < (SL_BK * SL_BM) / SL_THREADS; ++it) {
            const int idx = tid + it * SL_THREADS;
            const int kk = idx % SL_BK, r = idx / SL_BK;
            const int gk = k0 + kk;
            unsigned short da[SL_S], db[SL_S];
            const long gr = M0 + r;
            const double va = (gr < M && gk < K) ? A[gr * lda + gk] : 0.0;
            digits(va, gr < M ? erowA[gr] : 0, da);
            const int gc = N0 + r;
            const double vb = (gc < N && gk < K) ? B[(long)gc * ldb + gk] : 0.0;
            digits(vb, gc < N ? erowB[gc] : 0, db);
            const int pk = swz_elem(r, kk);
#pragma unroll
            for (int s = 0; s < SL_S; ++s) {
                TA.d[s][r][pk] = da[s];
                TB.d[s][r][pk] = db[s];
            }
        }
        __syncthreads();
        block_products(TA, TB, wm, wn, lane, hi, lo);
        __syncthreads();
    }
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const long i = M0 + wm + mi * 16 + g + (c >= 2 ? 8 : 0);
                const int j = N0 + wn + ni * 8 + t4 * 2 + (c & 1);
                if (i < M && j < N) {
                    const double v = (double)hi[mi][ni][c] + (double)lo[mi][ni][c];
                    C[i * ldc + j] = ldexp(v, erowA[i] + erowB[j] - 16);
                }
            }
}

// Digit planes of the column-scaled operand: D[s][j][i] (n x mp, i contiguous),
// rows i >= m padded with zero digits.  A CTA slices a 32 (i) x 64 (j) block,
// coalesced along j on the FP64 read, and writes 64-byte runs along i through
// a shared-memory transpose.
__global__ void __launch_bounds__(256)
slice_cols_kernel(int m, int n, long mp, const double* __restrict__ A, long lda,
                  const int* __restrict__ ecol, unsigned short* __restrict__ D) {
    __shared__ unsigned short t[SL_S][64][34];
    const int j0 = blockIdx.x * 64;
    for (long ib = blockIdx.y; ib < mp / 32; ib += gridDim.y) {
    const long i0 = ib * 32;
    __syncthreads();  // previous block's transpose reads are done
    for (int idx = threadIdx.x; idx < 32 * 64; idx += blockDim.x) {
        const int j = idx % 64, i = idx / 64;
        const long gi = i0 + i;
        const int gj = j0 + j;
        const double v = (gi < m && gj < n) ? A[gi * lda + gj] : 0.0;
        unsigned short d[SL_S];
        digits(v, gj < n ? ecol[gj] : 0, d);
#pragma unroll
        for (int s = 0; s < SL_S; ++s) t[s][j][i] = d[s];
    }
    __syncthreads();
    // write: for each (s, j), 32 consecutive i as 16 words of 2 digits
    for (int idx = threadIdx.x; idx < SL_S * 64 * 16; idx += blockDim.x) {
        const int w = idx % 16, j = (idx / 16) % 64, s = idx / (16 * 64);
        const int gj = j0 + j;
        if (gj >= n) continue;
        const unsigned v = (unsigned)t[s][j][2 * w] | ((unsigned)t[s][j][2 * w + 1] << 16);
        unsigned* dst = reinterpret_cast<unsigned*>(D + ((long)s * n + gj) * mp + i0) + w;
        *dst = v;
    }
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

// Gram from digit planes: grid (T, T, ksplit) over upper tiles, 32-row blocks
// streamed with a two-stage cp.async pipeline.  Stage layout: [2 operands]
// SlTiles (64 x 40 bf16 rows, 16-byte aligned: 80-byte rows).
__global__ void __launch_bounds__(SL_THREADS)
slgram_planes_kernel(int n, long mp, const unsigned short* __restrict__ D,
                     const int* __restrict__ ecol, int kchunk, double* __restrict__ partial) {
    const int tn = blockIdx.x, tm = blockIdx.y, ks = blockIdx.z;
    if (tn < tm) return;
    extern __shared__ unsigned char smraw[];
    SlTiles* stage = reinterpret_cast<SlTiles*>(smraw);  // [2 stages][2 operands]
    const bool diag = (tn == tm);
    const int J0 = tm * SL_BM, K0 = tn * SL_BN;
    const long kbeg = (long)ks * kchunk;
    const long kend = min(mp, kbeg + kchunk);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int nops = diag ? 1 : 2;
    auto issue = [&](int st, long k0) {
        // chunks: operand o, digit s, row r (64), 4 x 16 B along i
        const int total = nops * SL_S * 64 * 4;
        for (int c = tid; c < total; c += SL_THREADS) {
            const int q = c & 3, r = (c >> 2) & 63, s = (c >> 8) % SL_S, o = c / (256 * SL_S);
            const int gj = (o == 0 ? J0 : K0) + r;
            SlTiles& T = stage[st * 2 + o];
            unsigned short* dst = &T.d[s][r][swz_word(r, q * 4) << 1];
            if (gj < n) {
                cp_async16(dst, D + ((long)s * n + gj) * mp + k0 + q * 8);
            } else {
                *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        cp_async_commit();
    };
    float hi[2][4][4], lo[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) hi[a][b][c] = lo[a][b][c] = 0.f;
    if (kbeg < kend) issue(0, kbeg);
    int st = 0;
    for (long k0 = kbeg; k0 < kend; k0 += SL_BK) {
        const bool more = k0 + SL_BK < kend;
        if (more) issue(st ^ 1, k0 + SL_BK);
        if (more) cp_async_wait<1>(); else cp_async_wait<0>();
        __syncthreads();
        const SlTiles& TJ = stage[st * 2];
        const SlTiles& TK = diag ? stage[st * 2] : stage[st * 2 + 1];
        block_products(TJ, TK, wm, wn, lane, hi, lo);
        __syncthreads();
        st ^= 1;
    }
    double* out = partial + (long)ks * n * n;
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = J0 + wm + mi * 16 + g + (c >= 2 ? 8 : 0);
                const int k = K0 + wn + ni * 8 + t4 * 2 + (c & 1);
                if (j < n && k < n) {
                    const double v = (double)hi[mi][ni][c] + (double)lo[mi][ni][c];
                    out[(long)j * n + k] = ldexp(v, ecol[j] + ecol[k] - 16);
                }
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

long sl_resident() {
    static std::atomic<long> cached{0};  // the same value from any thread
    if (cached.load()) return cached.load();
    int dev = 0, sms = 152, per = 1;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    (void)ensure_max_dynamic_smem((const void*)slgram_planes_kernel);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, slgram_planes_kernel, SL_THREADS,
                                                      4 * sizeof(SlTiles)) != cudaSuccess || per < 1)
        per = 1;
    (void)cudaGetLastError();
    cached.store((long)sms * per);
    return cached.load();
}

int sl_ksplit(int m, int n) {
    const long T = (n + SL_BN - 1) / SL_BN;
    const long tiles = T * (T + 1) / 2;
    long ks = std::max<long>(1, sl_resident() / tiles);
    ks = std::min<long>(ks, std::max<long>(1, m / 256));
    return (int)std::max<long>(1, std::min<long>(ks, 1024));
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

}  // namespace

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

size_t slgram_scratch_doubles(int m, int n) {
    // split partials + per-column maxima (as 64-bit words) + exponents + digit planes
    const size_t mp = ((size_t)std::max(m, 1) + SL_BK - 1) / SL_BK * SL_BK;
    return ((size_t)sl_ksplit(std::max(m, 1), n) * n * n + 2 * (size_t)n + 8 + 31) / 32 * 32 +
           (SL_S * (size_t)n * mp + 3) / 4;
}

tt_status slgram(cudaStream_t s, int m, int n, const double* A, long lda, double* G, long ldg,
                 DevBuf& scratch) {
    if (n <= 0) return TT_OK;
    if (m <= 0) {
        for (int i = 0; i < n; ++i) fill(s, G + (long)i * ldg, n, 0.0);
        return TT_OK;
    }
    const int ks = sl_ksplit(m, n);
    TT_TRY(scratch.ensure(slgram_scratch_doubles(m, n), s));
    double* partial = scratch.p;
    unsigned long long* cmax = reinterpret_cast<unsigned long long*>(scratch.p + (size_t)ks * n * n);
    int* ecol = reinterpret_cast<int*>(cmax + n);
    TT_CUDA_TRY(cudaMemsetAsync(cmax, 0, n * sizeof(unsigned long long), s));
    {
        dim3 grid((n + 31) / 32, (unsigned)std::min<long>(std::max<long>(1, m / 4096), 256));
        note_launch();
        col_max_kernel<<<grid, 256, 0, s>>>(m, n, A, lda, cmax);
        note_launch();
        max_to_exp_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, cmax, ecol);
    }
    const long mp = ((long)m + SL_BK - 1) / SL_BK * SL_BK;
    // digit planes start on a 256-byte boundary (cp.async moves 16-byte chunks)
    const size_t plane_off = ((size_t)ks * n * n + 2 * (size_t)n + 8 + 31) / 32 * 32;
    unsigned short* planes = reinterpret_cast<unsigned short*>(scratch.p + plane_off);
    {
        dim3 grid((n + 63) / 64, (unsigned)std::min<long>(mp / 32, 16384));
        note_launch();
        slice_cols_kernel<<<grid, 256, 0, s>>>(m, n, mp, A, lda, ecol, planes);
    }
    {
        long kchunk = (mp + ks - 1) / ks;
        kchunk = ((kchunk + SL_BK - 1) / SL_BK) * SL_BK;
        const size_t smem = 4 * sizeof(SlTiles);
        TT_TRY(ensure_max_dynamic_smem((const void*)slgram_planes_kernel));
        const int T = (n + SL_BN - 1) / SL_BN;
        note_launch();
        slgram_planes_kernel<<<dim3(T, T, ks), SL_THREADS, smem, s>>>(n, mp, planes, ecol, (int)kchunk, partial);
        TT_CUDA_TRY(cudaGetLastError());
    }
    const long total = (long)n * n;
    note_launch();
    slgram_reduce_kernel<<<(int)std::min<long>((total + 255) / 256, 152L * 32), 256, 0, s>>>(n, ks, partial, G, ldg);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status slgemm_nt(cudaStream_t s, long M, int N, int K, const double* A, long lda, const double* B,
                    long ldb, double* C, long ldc, DevBuf& scratch) {
    if (M <= 0 || N <= 0) return TT_OK;
    if (K <= 0) {
        for (long i = 0; i < M; ++i) fill(s, C + i * ldc, N, 0.0);
        return TT_OK;
    }
    TT_TRY(scratch.ensure((size_t)(M + N + 1) / 2 + 2, s));
    int* eA = reinterpret_cast<int*>(scratch.p);
    int* eB = eA + M;
    note_launch();
    row_exp_kernel<<<(int)std::max<long>(1, std::min<long>((M + 7) / 8, 152L * 64)), 256, 0, s>>>(M, K, A, lda, eA);
    note_launch();
    row_exp_kernel<<<(N + 7) / 8, 256, 0, s>>>(N, K, B, ldb, eB);
    const size_t smem = 2 * sizeof(SlTiles);
    TT_TRY(ensure_max_dynamic_smem((const void*)slgemm_nt_kernel));
    const long gy = (M + SL_BM - 1) / SL_BM;
    if (gy > 65535L) {
        set_error("slgemm_nt: too many rows");
        return TT_ERR_TOO_LARGE;
    }
    note_launch();
    slgemm_nt_kernel<<<dim3((N + SL_BN - 1) / SL_BN, (unsigned)gy), SL_THREADS, smem, s>>>(
        (int)M, N, K, A, lda, eA, B, ldb, eB, C, ldc);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

}  // namespace ttsn
