// FP64 contractions of the Gram-SVD rounding (App. A.2 of arXiv 2503.18056):
// a general row-major GEMM and the tall-skinny left Gram G_A = A^T A, both on
// the FP64 tensor pipe (mma.sync m8n8k4.f64).  On GB300 the FP64 tensor pipe
// is about 4x the FP64 FMA pipe, and the contractions are deeply compute
// bound (about 14 flop per clock per SM), so a 64x64x16 shared-memory tile
// with four warps of 32x32 each keeps the pipe fed; operand staging is plain
// coalesced loads.
#include <algorithm>
#include <atomic>

#include "internal.h"

namespace ttsn {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, PADM = 4;
constexpr int THREADS = 128;

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
    asm volatile(
        "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
        : "+d"(c[0]), "+d"(c[1])
        : "d"(a), "d"(b));
}

// One 64 x 64 output tile: C[m0.., n0..] = alpha op(A) op(B) (+ beta C) over
// the K range [kbeg, kend).  A warp skips the 8 x 8 products whose rows or
// columns lie wholly outside M x N (a ragged last tile, e.g. the grown rank
// 7 r + 1) and, with tri on a diagonal tile, those wholly below the diagonal
// (a symmetric product whose lower triangle is never read): the stored
// entries are the same bits, the tensor pipe does only the work that is read.
template <bool TA, bool TB>
__device__ __forceinline__ void gemm_tile(int M, int N, double alpha, const double* __restrict__ A, long lda,
                                          const double* __restrict__ B, long ldb, double beta,
                                          double* __restrict__ C, long ldc, int kbeg, int kend, int m0,
                                          int n0, bool tri = false) {
    __shared__ double As[BK][BM + PADM];
    __shared__ double Bs[BK][BN + PADM];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    // live[i] bit j: the warp's 8 x 8 product (i, j) is needed
    unsigned live = 0;
    {
        const bool diag = tri && m0 == n0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r0 = m0 + wm + i * 8, c0 = n0 + wn + j * 8;
                const bool need = r0 < M && c0 < N && !(diag && r0 >= c0 + 8);
                live |= (need ? 1u : 0u) << (i * 4 + j);
            }
    }
    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // stage op(A) tile: (kk, mm) = op(A)(m0+mm, k0+kk)
#pragma unroll
        for (int it = 0; it < (BM * BK) / THREADS; ++it) {
            const int idx = tid + it * THREADS;
            int kk, mm;
            if (TA) { mm = idx % BM; kk = idx / BM; }
            else    { kk = idx % BK; mm = idx / BK; }
            const int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < kend) v = TA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk];
            As[kk][mm] = v;
        }
#pragma unroll
        for (int it = 0; it < (BN * BK) / THREADS; ++it) {
            const int idx = tid + it * THREADS;
            int kk, nn;
            if (TB) { kk = idx % BK; nn = idx / BK; }
            else    { nn = idx % BN; kk = idx / BN; }
            const int gn = n0 + nn, gk = k0 + kk;
            double v = 0.0;
            if (gn < N && gk < kend) v = TB ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk + (lane & 3)][wm + i * 8 + (lane >> 2)];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk + (lane & 3)][wn + j * 8 + (lane >> 2)];
            if (live == 0xFFFFu) {  // a full tile: the unconditional chain
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) dmma(acc[i][j], a[i], bb[j]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (live & (1u << (i * 4 + j))) dmma(acc[i][j], a[i], bb[j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + wm + i * 8 + (lane >> 2);
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int gn = n0 + wn + j * 8 + (lane & 3) * 2 + e;
                if (gn >= N) continue;
                double* dst = C + (long)gm * ldc + gn;
                const double v = alpha * acc[i][j][e];
                *dst = (beta == 0.0) ? v : v + beta * (*dst);
            }
        }
    }
}

// grid: x = N tiles, y = M tiles, z = batch * ksplit.
// Batch entry b, split ks: rows of K in [ks*kchunk, min(K,(ks+1)*kchunk)), output
// to C + b*sC + ks*sCsplit.  upper_only: skip tiles strictly below the diagonal.
template <bool TA, bool TB>
__global__ void __launch_bounds__(THREADS, 4)
dgemm_kernel(int M, int N, int K, double alpha, const double* __restrict__ A, long lda, long sA,
             const double* __restrict__ B, long ldb, long sB, double beta, double* __restrict__ C,
             long ldc, long sC, int ksplit, int kchunk, long sCsplit, int upper_only) {
    const int tn = blockIdx.x, tm = blockIdx.y;
    if (upper_only && tn < tm) return;
    const int b = blockIdx.z / ksplit, ks = blockIdx.z % ksplit;
    A += b * sA;
    B += b * sB;
    C += b * sC + ks * sCsplit;
    const int kbeg = ks * kchunk;
    const int kend = min(K, kbeg + kchunk);
    gemm_tile<TA, TB>(M, N, alpha, A, lda, B, ldb, beta, C, ldc, kbeg, kend, tm * BM, tn * BN, upper_only != 0);
}

// The same product with its sizes read from device memory (a captured step
// whose ranks the device decides): desc = M, N, K, lda, ldb, ldc.  The grid
// covers the largest sizes the step can reach; CTAs outside the step's tile
// grid or split count return at once.  mode 0: one pass into C (as dgemm);
// mode 1: dgemm_sk's split rule (one pass into C when it gives one split,
// else partials into P, plane z at z M N with leading dimension N); mode 2:
// the Gram's row split (gram_split_rule with `resident`, upper tiles only,
// partials into P with leading dimension N, every split written).  Each
// decision equals the host path's for the same sizes, so the results are
// the same bits.
template <bool TA, bool TB>
__global__ void __launch_bounds__(THREADS, 4)
dgemm_dyn_kernel(const int* __restrict__ desc, double alpha, const double* __restrict__ A,
                 const double* __restrict__ B, double* __restrict__ C, double* __restrict__ P, int mode,
                 long resident) {
    const int M = desc[0], N = desc[1], K = desc[2];
    const long lda = desc[3], ldb = desc[4], ldc = desc[5];
    const int TM = (M + BM - 1) / BM, TN = (N + BN - 1) / BN;
    int tm, tn, z = 0;
    int ks = 1, kchunk = K;
    if (mode == 0) {  // a 2-D grid of tiles sized for the capacity
        tn = blockIdx.x;
        tm = blockIdx.y;
        if (tm >= TM || tn >= TN) return;
    } else {
        // modes 1 and 2: a 1-D grid of (split, tile) items, sized on the host
        // for the most items any size up to the capacity takes; items past
        // this step's count return at once
        if (mode == 1) {
            sk_split(M, N, K, &ks, &kchunk);
        } else {
            ks = gram_split_rule(K, M, resident);
            kchunk = (K + ks - 1) / ks;
            kchunk = (kchunk + BK - 1) / BK * BK;
        }
        const int per = mode == 2 ? TM * (TM + 1) / 2 : TM * TN;  // Gram: upper-triangle tiles
        const long item = blockIdx.x;
        if (item >= (long)per * ks) return;
        z = (int)(item / per);
        int t = (int)(item % per);
        if (mode == 2) {
            tm = 0;
            while (t >= TM - tm) {  // row tm of the upper triangle holds TM - tm tiles
                t -= TM - tm;
                ++tm;
            }
            tn = tm + t;
        } else {
            tm = t / TN;
            tn = t % TN;
        }
    }
    const int kbeg = z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    if (mode == 2 || ks > 1)
        gemm_tile<TA, TB>(M, N, 1.0, A, lda, B, ldb, 0.0, P + (long)z * M * N, N, kbeg, kend, tm * BM,
                          tn * BN, mode == 2);
    else
        gemm_tile<TA, TB>(M, N, alpha, A, lda, B, ldb, 0.0, C, ldc, kbeg, kend, tm * BM, tn * BN);
}

// mode 1 partials -> C (nothing to do when the rule gave one split)
__global__ void splitk_reduce_dyn_kernel(const int* __restrict__ desc, const double* __restrict__ P,
                                         double alpha, double* C) {
    const int M = desc[0], N = desc[1], K = desc[2];
    const long ldc = desc[5];
    int ks = 1, kchunk = K;
    sk_split(M, N, K, &ks, &kchunk);
    if (ks == 1) return;
    const long total = (long)M * N;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < ks; ++z) s += P[(long)z * total + t];
        C[(t / N) * ldc + t % N] = alpha * s;
    }
}

// mode 2 partials -> the symmetric G (leading dimension desc[5])
__global__ void gram_reduce_dyn_kernel(const int* __restrict__ desc, const double* __restrict__ P,
                                       long resident, double* G) {
    const int n = desc[0], m = desc[2];
    const long ldg = desc[5];
    const int ks = gram_split_rule(m, n, resident);
    const long total = (long)n * n;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        const int a = min(i, j), b = max(i, j);
        double s = 0.0;
        for (int z = 0; z < ks; ++z) s += P[(long)z * total + (long)a * n + b];
        G[(long)i * ldg + j] = s;
    }
}

// out[i][j] = in[i][j] * f(v[i]) with rows, cols, ldi, ldo = desc[0..3]
__global__ void scale_rows_dyn_kernel(const int* __restrict__ desc, const double* in, const double* v, int mode,
                                      double* out) {
    const int rows = desc[0], cols = desc[1];
    const long ldi = desc[2], ldo = desc[3];
    const long total = (long)rows * cols;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t / cols), j = (int)(t % cols);
        const double x = v[i];
        double f;
        switch (mode) {
            case 0: f = x; break;
            case 1: f = sqrt(x); break;
            case 2: f = 1.0 / sqrt(x); break;
            default: f = 1.0 / x; break;
        }
        out[(long)i * ldo + j] = in[(long)i * ldi + j] * f;
    }
}

// C[i][j] = alpha sum_z P[z][i][j] (fixed order => reproducible)
__global__ void splitk_reduce_kernel(int M, int N, int ksplit, const double* __restrict__ P,
                                     double alpha, double* C, long ldc) {
    const long total = (long)M * N;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < ksplit; ++z) s += P[(long)z * total + t];
        C[(t / N) * ldc + t % N] = alpha * s;
    }
}

// G[i][j] = sum_z P[z][min(i,j)][max(i,j)]  (fixed order => reproducible, symmetric)
__global__ void gram_reduce_kernel(int n, int ksplit, const double* __restrict__ P, double* G,
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

__global__ void scale_rows_kernel(int rows, int cols, const double* in, long ldi, const double* v,
                                  int mode, double* out, long ldo) {
    const long total = (long)rows * cols;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t / cols), j = (int)(t % cols);
        const double x = v[i];
        double f;
        switch (mode) {
            case 0: f = x; break;
            case 1: f = sqrt(x); break;
            case 2: f = 1.0 / sqrt(x); break;
            default: f = 1.0 / x; break;
        }
        out[(long)i * ldo + j] = in[(long)i * ldi + j] * f;
    }
}

__global__ void fill_kernel(double* p, size_t n, double value) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x)
        p[t] = value;
}

__global__ void copy2d_kernel(int rows, int cols, const double* in, long ldi, double* out,
                              long ldo) {
    const long total = (long)rows * cols;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t / cols), j = (int)(t % cols);
        out[(long)i * ldo + j] = in[(long)i * ldi + j];
    }
}

// out[j] = alpha sum_i A[i][j] v[i] for tall A (m x ncols, m >> ncols): block b
// sums its chunk of rows for every column (row groups of the block split the
// chunk and meet in shared memory in a fixed order), a second kernel adds the
// block partials in block order -- deterministic, one pass over A.
constexpr int GEMV_THREADS = 256;
__global__ void __launch_bounds__(GEMV_THREADS)
gemv_t_partial_kernel(long m, int ncols, const double* __restrict__ A, long lda,
                      const double* __restrict__ v, long chunk, double* __restrict__ part) {
    __shared__ double red[GEMV_THREADS];
    const int cw = min(GEMV_THREADS, ((ncols + 31) / 32) * 32);
    const int rg = GEMV_THREADS / cw;
    const int t = threadIdx.x, c0 = t % cw, g = t / cw;
    const long i0 = blockIdx.x * chunk, i1 = min(m, i0 + chunk);
    for (int cb = 0; cb < ncols; cb += cw) {
        const int col = cb + c0;
        double acc = 0.0;
        if (g < rg && col < ncols)
            for (long i = i0 + g; i < i1; i += rg) acc += A[i * lda + col] * v[i];
        red[t] = acc;
        __syncthreads();
        if (g == 0 && col < ncols) {
            double s = red[c0];
            for (int q = 1; q < rg; ++q) s += red[q * cw + c0];
            part[(long)blockIdx.x * ncols + col] = s;
        }
        __syncthreads();
    }
}

__global__ void gemv_t_final_kernel(int nblk, int ncols, double alpha, const double* part,
                                    double* out) {
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < ncols; col += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(long)b * ncols + col];
        out[col] = alpha * s;
    }
}

}  // namespace

// Autotuned splits (tt_autotune): for a product of t < 152 output tiles
// (bucket floor(log2 t)) and depth K (bucket floor(log2 K)), the split of K
// that measured fastest on this GPU; 0 keeps the rule below.  One copy for
// the host and one in device memory, installed together, so a captured step
// decides as the host path does.
__device__ int d_sk_table[AT_TILE_BUCKETS * AT_K_BUCKETS];
static int h_sk_table[AT_TILE_BUCKETS * AT_K_BUCKETS];

__host__ __device__ inline int floor_log2(long x) {
    int b = 0;
    while (x > 1) {
        x >>= 1;
        ++b;
    }
    return b;
}

// Split of K for dgemm_sk: one 64 x 64 x 16 tile step is ~131 kflop, about
// 19 us of one SM's FP64 pipe on GB300, so a product with a handful of tiles
// runs for (K / 16) x 19 us on a handful of SMs; where the tile grid leaves
// SMs idle, K is split so that there are about two CTAs per SM, each with at
// least two K tiles, unless the autotuned table holds a measured split for
// the product's bucket.  Host and device use the same rule (a captured step
// decides it on the device from the sizes of that step).
__host__ __device__ void sk_split(int M, int N, int K, int* ks_out, int* kchunk_out) {
    const long tiles = (long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    int ks = 1;
    if (tiles < 152 && K >= 4 * BK) {
        long a = (304 + tiles - 1) / tiles, b = K / (2 * BK);
        ks = (int)(a < b ? a : b);
        const int tb = floor_log2(tiles), kb = floor_log2(K);
        if (tb < AT_TILE_BUCKETS && kb < AT_K_BUCKETS) {
#ifdef __CUDA_ARCH__
            const int tuned = d_sk_table[tb * AT_K_BUCKETS + kb];
#else
            const int tuned = h_sk_table[tb * AT_K_BUCKETS + kb];
#endif
            if (tuned > 0) ks = (int)(tuned < b ? tuned : b);
        }
        ks = ks < 1 ? 1 : (ks > 64 ? 64 : ks);
    }
    int kchunk = K;
    if (ks > 1) {
        kchunk = (K + ks - 1) / ks;
        kchunk = (kchunk + BK - 1) / BK * BK;
        ks = (K + kchunk - 1) / kchunk;
    }
    *ks_out = ks;
    *kchunk_out = kchunk;
}

// Row split of the Gram (gram_ksplit) from the number of resident CTAs.
// Small problems (16 or more splits fit in one wave of the resident slots)
// take one wave.  For larger ones one wave leaves slots idle (105 upper tiles
// at 5 splits fill 525 of 608) and the tiles differ in work: gemm_tile
// computes only the 8 x 8 products of the upper triangle that the matrix
// reaches, W = B (B + 1) / 2 of them for B = ceil(n / 8).  Dealt in many
// waves (GRAM_MULTI_SPLITS splits), the slots stay busy and the time is
// about W / (64 resident) + 1 / (2 splits) of one unsplit tile's, against
// 1 / ks0 for one wave; the shorter is taken (integer arithmetic, so the
// host and a captured step's device agree).  Every split keeps at least 256
// rows.
__host__ __device__ int gram_split_rule(int m, int n, long resident) {
    const long T = (n + BN - 1) / BN;
    const long tiles = T * (T + 1) / 2;
    long cap = m / 256 < 1 ? 1 : m / 256;
    if (cap > 1024) cap = 1024;
    if (resident < 1) resident = 1;
    long ks0 = resident / tiles;
    if (ks0 < 1) ks0 = 1;
    if (ks0 > cap) ks0 = cap;
    if (ks0 >= 16) return (int)ks0;
    const long km = cap < GRAM_MULTI_SPLITS ? cap : GRAM_MULTI_SPLITS;
    if (km <= ks0) return (int)ks0;
    const long long B = (n + 7) / 8;
    const long long W = B * (B + 1) / 2;
    const long long slots = 64LL * resident;
    // (W / slots + 1 / (2 km)) < 0.97 / ks0, times 2 slots km ks0 100
    if ((2 * W * km + slots) * ks0 * 100 < 97LL * 2 * slots * km) return (int)km;
    return (int)ks0;
}

namespace {

inline int grid_for(long total, int threads = 256) {
    long b = (total + threads - 1) / threads;
    return (int)std::max<long>(1, std::min<long>(b, 152L * 32));
}

tt_status launch_gemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                      const double* A, long lda, long sA, const double* B, long ldb, long sB,
                      double beta, double* C, long ldc, long sC, int batch, int ksplit,
                      int kchunk, long sCsplit, int upper) {
    if (M <= 0 || N <= 0 || batch <= 0) return TT_OK;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch * ksplit);
    if (grid.y > 65535 || grid.z > 65535) {
        set_error("dgemm: problem too large for the tile grid");
        return TT_ERR_TOO_LARGE;
    }
    note_launch();
    if (ta && tb)
        dgemm_kernel<true, true><<<grid, THREADS, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, ksplit, kchunk, sCsplit, upper);
    else if (ta)
        dgemm_kernel<true, false><<<grid, THREADS, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, ksplit, kchunk, sCsplit, upper);
    else if (tb)
        dgemm_kernel<false, true><<<grid, THREADS, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, ksplit, kchunk, sCsplit, upper);
    else
        dgemm_kernel<false, false><<<grid, THREADS, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, ksplit, kchunk, sCsplit, upper);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

}  // namespace

tt_status dgemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                const double* A, long lda, const double* B, long ldb, double beta, double* C,
                long ldc, int batch, long strideA, long strideB, long strideC) {
    if (M < 0 || N < 0 || K < 0) {
        set_error("dgemm: negative size");
        return TT_ERR_ARG;
    }
    if (K == 0) {  // C = beta C
        if (beta == 0.0) {
            for (int b = 0; b < batch; ++b)
                for (int i = 0; i < M; ++i) fill(s, C + b * strideC + (long)i * ldc, N, 0.0);
        }
        return TT_OK;
    }
    return launch_gemm(s, ta, tb, M, N, K, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc,
                       strideC, batch, 1, K, 0, 0);
}

tt_status dgemm_sk(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                   const double* A, long lda, const double* B, long ldb, double* C, long ldc,
                   DevBuf& scratch) {
    int ks = 1, kchunk = K;
    sk_split(M, N, K, &ks, &kchunk);
    if (ks == 1 || M <= 0 || N <= 0)
        return dgemm(s, ta, tb, M, N, K, alpha, A, lda, B, ldb, 0.0, C, ldc);
    const long per = (long)M * N;
    TT_TRY(scratch.ensure((size_t)ks * per, s));
    TT_TRY(launch_gemm(s, ta, tb, M, N, K, 1.0, A, lda, 0, B, ldb, 0, 0.0, scratch.p, N, 0, 1, ks,
                       kchunk, per, 0));
    note_launch();
    splitk_reduce_kernel<<<grid_for(per), 256, 0, s>>>(M, N, ks, scratch.p, alpha, C, ldc);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

namespace {
// CTAs of dgemm_kernel<true,false> resident on the whole GPU at once.
long resident_gram_ctas() {
    static std::atomic<long> cached{0};  // the same value from any thread
    if (cached.load()) return cached.load();
    int dev = 0, sms = 152, per = 4;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dgemm_kernel<true, false>, THREADS, 0) !=
            cudaSuccess || per < 1)
        per = 4;
    (void)cudaGetLastError();
    cached.store((long)sms * per);
    return cached.load();
}

// Row-split factor of the Gram (gram_split_rule on this GPU's resident slots).
int gram_ksplit(int m, int n) { return gram_split_rule(m, n, resident_gram_ctas()); }
}  // namespace

size_t gram_scratch_doubles(int m, int n) {
    return (size_t)gram_ksplit(m, n) * (size_t)n * (size_t)n;
}

tt_status gram_with_scratch(cudaStream_t s, int m, int n, const double* A, long lda, double* G,
                            long ldg, double* scratch, size_t scratch_doubles) {
    if (m < 0 || n < 0) {
        set_error("gram: negative size");
        return TT_ERR_ARG;
    }
    if (n == 0) return TT_OK;
    if (m == 0) {
        for (int i = 0; i < n; ++i) fill(s, G + (long)i * ldg, n, 0.0);
        return TT_OK;
    }
    const int ks = gram_ksplit(m, n);
    if (scratch_doubles < (size_t)ks * n * n) {
        set_error("gram: scratch too small");
        return TT_ERR_TOO_LARGE;
    }
    int kchunk = (m + ks - 1) / ks;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    // op(A) = A^T (stored m x n => trans), op(B) = A (not trans): (n x m)(m x n)
    TT_TRY(launch_gemm(s, true, false, n, n, m, 1.0, A, lda, 0, A, lda, 0, 0.0, scratch, n, 0, 1,
                       ks, kchunk, (long)n * n, 1));
    note_launch();
    gram_reduce_kernel<<<grid_for((long)n * n), 256, 0, s>>>(n, ks, scratch, G, ldg);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status gram_fixed_scratch(cudaStream_t s, int m, int n, const double* A, long lda, double* G,
                             long ldg, double* scratch, size_t scratch_doubles) {
    if (n == 0) return TT_OK;
    if (m == 0) {
        for (int i = 0; i < n; ++i) fill(s, G + (long)i * ldg, n, 0.0);
        return TT_OK;
    }
    const size_t per = (size_t)n * n;
    if (per > scratch_doubles) {
        set_error("gram: scratch smaller than one n x n partial");
        return TT_ERR_TOO_LARGE;
    }
    const int ks = (int)std::min<size_t>((size_t)gram_ksplit(m, n), scratch_doubles / per);
    int kchunk = (m + ks - 1) / ks;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    TT_TRY(launch_gemm(s, true, false, n, n, m, 1.0, A, lda, 0, A, lda, 0, 0.0, scratch, n, 0, 1,
                       ks, kchunk, (long)n * n, 1));
    note_launch();
    gram_reduce_kernel<<<grid_for((long)n * n), 256, 0, s>>>(n, ks, scratch, G, ldg);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

long gram_resident() { return resident_gram_ctas(); }

// The most (split, tile) items a split-mode product of sizes up to the
// capacity can take (the split rules grow with K, so K = Kcap bounds them
// per tile count; mode 1's tuned table is indexed by log2 K, so every K
// bucket up to Kcap is tried).
long dyn_items(int mode, int Mcap, int Ncap, int Kcap, long resident) {
    long most = 1;
    if (mode == 2) {
        for (int n = 1; n <= Ncap; ++n) {
            const long T = (n + BN - 1) / BN;
            most = std::max(most, T * (T + 1) / 2 * (long)gram_split_rule(Kcap, n, resident));
        }
        return most;
    }
    // mode 1: sk_split's split is not monotone in K (the chunk is rounded to
    // BK), so bound it instead: no split below 152 tiles exceeds the built-in
    // ceil(304 / tiles), the tuned entries of every K bucket up to Kcap, 64,
    // or ceil(Kcap / BK)
    const int TMc = (Mcap + BM - 1) / BM, TNc = (Ncap + BN - 1) / BN;
    const int kbmax = floor_log2(std::max(Kcap, 1));
    for (int tm = 1; tm <= TMc; ++tm)
        for (int tn = 1; tn <= TNc; ++tn) {
            const long tiles = (long)tm * tn;
            long ks = 1;
            if (tiles < 152 && Kcap >= 4 * BK) {
                ks = (304 + tiles - 1) / tiles;
                const int tb = floor_log2((int)tiles);
                if (tb < AT_TILE_BUCKETS)
                    for (int kb = 0; kb <= kbmax && kb < AT_K_BUCKETS; ++kb)
                        ks = std::max<long>(ks, h_sk_table[tb * AT_K_BUCKETS + kb]);
                ks = std::min<long>(std::min<long>(ks, 64), (Kcap + BK - 1) / BK);
                ks = std::max<long>(ks, 1);
            }
            most = std::max(most, tiles * ks);
        }
    return most;
}

size_t dyn_partials_need(int mode, int Mcap, int Ncap, int Kcap) {
    if (mode == 0 || Mcap <= 0 || Ncap <= 0) return 0;
    const long resident = resident_gram_ctas();
    if (mode == 2) {  // ks(n) n^2 partial Grams for the most demanding n <= Ncap
        size_t most = 0;
        for (int n = 1; n <= Ncap; ++n)
            most = std::max(most, (size_t)gram_split_rule(Kcap, n, resident) * (size_t)n * (size_t)n);
        return most;
    }
    // ks M N <= ks tiles BM BN
    return (size_t)dyn_items(1, Mcap, Ncap, Kcap, resident) * BM * BN;
}

tt_status dgemm_dyn(cudaStream_t s, bool ta, bool tb, const int* desc, int Mcap, int Ncap, int Kcap,
                    double alpha, const double* A, const double* B, double* C, double* P, size_t pcap, int mode) {
    if (Mcap <= 0 || Ncap <= 0) return TT_OK;
    if (dyn_partials_need(mode, Mcap, Ncap, Kcap) > pcap) {
        set_error("dgemm: the partials buffer of a captured product is smaller than its split needs");
        return TT_ERR_TOO_LARGE;
    }
    const long resident = resident_gram_ctas();
    dim3 grid((Ncap + BN - 1) / BN, (Mcap + BM - 1) / BM, 1);
    if (mode != 0) {
        const long items = dyn_items(mode, Mcap, Ncap, Kcap, resident);
        if (items > 0x7fffffffL) {
            set_error("dgemm: problem too large for the item grid");
            return TT_ERR_TOO_LARGE;
        }
        grid = dim3((unsigned)items, 1, 1);
    }
    if (grid.y > 65535) {
        set_error("dgemm: problem too large for the tile grid");
        return TT_ERR_TOO_LARGE;
    }
    note_launch();
    if (ta && tb)
        dgemm_dyn_kernel<true, true><<<grid, THREADS, 0, s>>>(desc, alpha, A, B, C, P, mode, resident);
    else if (ta)
        dgemm_dyn_kernel<true, false><<<grid, THREADS, 0, s>>>(desc, alpha, A, B, C, P, mode, resident);
    else if (tb)
        dgemm_dyn_kernel<false, true><<<grid, THREADS, 0, s>>>(desc, alpha, A, B, C, P, mode, resident);
    else
        dgemm_dyn_kernel<false, false><<<grid, THREADS, 0, s>>>(desc, alpha, A, B, C, P, mode, resident);
    if (mode == 1) {
        note_launch();
        splitk_reduce_dyn_kernel<<<grid_for((long)Mcap * Ncap), 256, 0, s>>>(desc, P, alpha, C);
    } else if (mode == 2) {
        note_launch();
        gram_reduce_dyn_kernel<<<grid_for((long)Mcap * Ncap), 256, 0, s>>>(desc, P, resident, C);
    }
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

void scale_rows_dyn(cudaStream_t s, const int* desc, long total_cap, const double* in, const double* v, int mode,
                    double* out) {
    if (total_cap <= 0) return;
    note_launch();
    scale_rows_dyn_kernel<<<grid_for(total_cap), 256, 0, s>>>(desc, in, v, mode, out);
}

tt_status gram(cudaStream_t s, int m, int n, const double* A, long lda, double* G, long ldg,
               DevBuf& partials) {
    if (n <= 0) return TT_OK;
    const size_t need = gram_scratch_doubles(std::max(m, 1), n);
    TT_TRY(partials.ensure(need, s));
    return gram_with_scratch(s, m, n, A, lda, G, ldg, partials.p, partials.cap);
}

void scale_rows(cudaStream_t s, int rows, int cols, const double* in, long ldi, const double* v,
                int mode, double* out, long ldo) {
    if (rows <= 0 || cols <= 0) return;
    note_launch();
    scale_rows_kernel<<<grid_for((long)rows * cols), 256, 0, s>>>(rows, cols, in, ldi, v, mode,
                                                                 out, ldo);
}

tt_status gemv_t(cudaStream_t s, long m, int ncols, double alpha, const double* A, long lda,
                 const double* v, double* out, DevBuf& scratch) {
    if (ncols <= 0) return TT_OK;
    if (m <= 0) {
        fill(s, out, (size_t)ncols, 0.0);
        return TT_OK;
    }
    // about 4 blocks per SM, at least 64 rows each
    const long chunk = std::max<long>(64, (m + 152L * 4 - 1) / (152L * 4));
    const int nblk = (int)((m + chunk - 1) / chunk);
    TT_TRY(scratch.ensure((size_t)nblk * ncols, s));
    note_launch();
    gemv_t_partial_kernel<<<nblk, GEMV_THREADS, 0, s>>>(m, ncols, A, lda, v, chunk, scratch.p);
    note_launch();
    gemv_t_final_kernel<<<std::max(1, std::min(152, (ncols + 127) / 128)), 128, 0, s>>>(
        nblk, ncols, alpha, scratch.p, out);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

void fill(cudaStream_t s, double* p, size_t n, double value) {
    if (n == 0) return;
    note_launch();
    fill_kernel<<<grid_for((long)n), 256, 0, s>>>(p, n, value);
}

void copy2d(cudaStream_t s, int rows, int cols, const double* in, long ldi, double* out,
            long ldo) {
    if (rows <= 0 || cols <= 0) return;
    note_launch();
    copy2d_kernel<<<grid_for((long)rows * cols), 256, 0, s>>>(rows, cols, in, ldi, out, ldo);
}

namespace {
constexpr int PEAK_ITERS = 2048;
__global__ void __launch_bounds__(256) fp64_mma_peak_kernel(double* out, double seed) {
    const double a = seed * (threadIdx.x + 1), b = 1.0 + 1e-3 * threadIdx.x;
    double c[8][2];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = 0.0;
    for (int i = 0; i < PEAK_ITERS; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) dmma(c[j], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1];
    if (s == 1234.5) out[threadIdx.x] = s;  // keeps the chains live; never true in practice
}
}  // namespace

tt_status autotune_install(const int* table, int n) {
    if (n != AT_TILE_BUCKETS * AT_K_BUCKETS) {
        set_error("autotune: the table has " + std::to_string(AT_TILE_BUCKETS * AT_K_BUCKETS) + " entries");
        return TT_ERR_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (table[i] < 0 || table[i] > 64) {
            set_error("autotune: splits are 0 (the rule) or 1 .. 64");
            return TT_ERR_ARG;
        }
    TT_CUDA_TRY(cudaMemcpyToSymbol(d_sk_table, table, n * sizeof(int)));
    for (int i = 0; i < n; ++i) h_sk_table[i] = table[i];
    return TT_OK;
}

void autotune_read(int* table) {
    for (int i = 0; i < AT_TILE_BUCKETS * AT_K_BUCKETS; ++i) table[i] = h_sk_table[i];
}

// Measure, for every (tile-count, depth) bucket up to 2^14 deep, the products'
// time at each split of K the rule allows (1, 2, 4, ..., 64, capped at K / 32)
// on a representative product of that bucket (M x N tiles of 64, the
// bucket's smallest K), and keep the fastest (best of three runs each).
tt_status autotune(cudaStream_t s, int* table_out) {
    constexpr int KB_MAX = 14;
    const long Mmax = 64L << ((AT_TILE_BUCKETS - 1) / 2), Nmax = 64L << (AT_TILE_BUCKETS - 1 - (AT_TILE_BUCKETS - 1) / 2);
    const long Kmax = 1L << KB_MAX;
    double *A = nullptr, *B = nullptr, *C = nullptr, *P = nullptr;
    const size_t pdbl = (size_t)64 * Mmax * Nmax;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tt_status st = TT_OK;
    int table[AT_TILE_BUCKETS * AT_K_BUCKETS] = {0};
    auto cleanup = [&]() {
        if (A) cudaFreeAsync(A, s);
        if (B) cudaFreeAsync(B, s);
        if (C) cudaFreeAsync(C, s);
        if (P) cudaFreeAsync(P, s);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMallocAsync((void**)&A, Mmax * Kmax * sizeof(double), s) != cudaSuccess ||
        cudaMallocAsync((void**)&B, Kmax * Nmax * sizeof(double), s) != cudaSuccess ||
        cudaMallocAsync((void**)&C, Mmax * Nmax * sizeof(double), s) != cudaSuccess ||
        cudaMallocAsync((void**)&P, pdbl * sizeof(double), s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        (void)cudaGetLastError();
        cleanup();
        set_error("autotune: device memory for the trial products");
        return TT_ERR_OOM;
    }
    fill(s, A, (size_t)(Mmax * Kmax), 0.5);
    fill(s, B, (size_t)(Kmax * Nmax), 0.25);
    for (int tb = 0; tb < AT_TILE_BUCKETS && st == TT_OK; ++tb) {
        const int M = 64 << (tb / 2), N = 64 << (tb - tb / 2);
        for (int kb = 6; kb <= KB_MAX && st == TT_OK; ++kb) {
            const int K = 1 << kb;
            float best = 1e30f;
            int best_ks = 0;
            for (int ks = 1; ks <= 64 && ks <= std::max(1, K / (2 * BK)); ks *= 2) {
                int kchunk = (K + ks - 1) / ks;
                kchunk = (kchunk + BK - 1) / BK * BK;
                const int kk = (K + kchunk - 1) / kchunk;
                float t = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    cudaEventRecord(e0, s);
                    if (kk == 1) {
                        st = launch_gemm(s, false, false, M, N, K, 1.0, A, K, 0, B, N, 0, 0.0, C, N, 0, 1, 1, K, 0, 0);
                    } else {
                        st = launch_gemm(s, false, false, M, N, K, 1.0, A, K, 0, B, N, 0, 0.0, P, N, 0, 1, kk, kchunk,
                                         (long)M * N, 0);
                        note_launch();
                        splitk_reduce_kernel<<<grid_for((long)M * N), 256, 0, s>>>(M, N, kk, P, 1.0, C, N);
                    }
                    cudaEventRecord(e1, s);
                    if (st < 0 || cudaEventSynchronize(e1) != cudaSuccess) {
                        if (st >= 0) st = TT_ERR_CUDA;
                        break;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    t = std::min(t, ms);
                }
                if (st < 0) break;
                if (t < best) {
                    best = t;
                    best_ks = ks;
                }
            }
            table[tb * AT_K_BUCKETS + kb] = best_ks;
        }
    }
    // deeper products keep the choice of the deepest measured bucket
    for (int tb = 0; tb < AT_TILE_BUCKETS; ++tb)
        for (int kb = KB_MAX + 1; kb < AT_K_BUCKETS; ++kb) table[tb * AT_K_BUCKETS + kb] = table[tb * AT_K_BUCKETS + KB_MAX];
    cleanup();
    if (st < 0) return st;
    TT_TRY(autotune_install(table, AT_TILE_BUCKETS * AT_K_BUCKETS));
    if (table_out)
        for (int i = 0; i < AT_TILE_BUCKETS * AT_K_BUCKETS; ++i) table_out[i] = table[i];
    return TT_OK;
}

tt_status bench_fp64_mma(cudaStream_t s, double* tflops) {
    int dev = 0, sms = 0;
    TT_CUDA_TRY(cudaGetDevice(&dev));
    TT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    double* out = nullptr;
    TT_CUDA_TRY(cudaMallocAsync((void**)&out, 256 * sizeof(double), s));
    cudaEvent_t e0, e1;
    TT_CUDA_TRY(cudaEventCreate(&e0));
    TT_CUDA_TRY(cudaEventCreate(&e1));
    const int blocks = sms * 8;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        TT_CUDA_TRY(cudaEventRecord(e0, s));
        note_launch();
        fp64_mma_peak_kernel<<<blocks, 256, 0, s>>>(out, 1e-3);
        TT_CUDA_TRY(cudaEventRecord(e1, s));
        TT_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        TT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, s);
    const double flops = 2.0 * 8 * 8 * 4 * 8.0 * PEAK_ITERS * blocks * (256 / 32);
    *tflops = flops / (best * 1e-3) / 1e12;
    return TT_OK;
}

}  // namespace ttsn
