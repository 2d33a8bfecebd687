// Element kernels of the QR-based TT rounding (TT-SVD, App. A.1 of arXiv
// 2503.18056).  The orchestration (backward QR sweep, forward truncated SVDs)
// is round_ttsvd in api.cu; it runs on the Gram, eigensolver and GEMM kernels
// of the Gram-SVD path plus these:
//
// * shifted_scale_rows: the first pass of a shifted eigen-form Cholesky QR.
//   For Y (m x l) with Gram G = Y^T Y = V diag(lambda) V^T, the columns of
//   Y V (diag(lambda) + s I)^(-1/2) span range(Y) with singular values
//   sigma / sqrt(sigma^2 + s) <= 1 for any s > 0, so the pass never divides by
//   a rounding-level eigenvalue.  Shifted Cholesky QR (Fukaya, Kannan,
//   Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 42, 2020) uses
//   the same shift with Cholesky factors; two unshifted passes then make the
//   basis orthonormal to working precision.
// * transpose: tiled out = in^T for the backward sweep's C_k^T.
// * the Jordan-Wielandt form of the SVD of the small factor Rf (q x l): the
//   symmetric (q + l) matrix [[c I, Rf], [Rf^T, c I]] has eigenvalues
//   c + sigma_i, c (|q - l| times), c - sigma_i and eigenvectors
//   [u_i; v_i] / sqrt(2) for c + sigma_i.  Its eigenpairs from the two-sided
//   Jacobi carry absolute errors eps_mach ||Rf||, so sigma is resolved down to
//   that level (a Gram matrix Rf^T Rf would resolve only sqrt(eps_mach) of
//   sigma_max).  The shift c = ||Rf||_F makes every diagonal entry positive,
//   so the Jacobi's relative skip test reads as an absolute one at
//   eps_mach ||Rf||.
#include "internal.h"

namespace ttsn {

namespace {

__global__ void shifted_scale_rows_kernel(int l, const double* __restrict__ Vt, long ldv,
                                          const double* __restrict__ lam, double* __restrict__ out, long ldo) {
    // lam is sorted descending: lam[0] the largest, lam[l - 1] the smallest
    const double lmax = fmax(lam[0], 0.0);
    const double shift = (double)l * 2.220446049250313e-16 * lmax + fmax(0.0, -lam[l - 1]);
    for (int i = blockIdx.x; i < l; i += gridDim.x) {
        const double den = lam[i] + shift;
        const double f = den > 0.0 ? 1.0 / sqrt(den) : 0.0;
        for (int j = threadIdx.x; j < l; j += blockDim.x) out[(long)i * ldo + j] = f * Vt[(long)i * ldv + j];
    }
}

constexpr int TB = 32;

__global__ void transpose_kernel(long rows, long cols, const double* __restrict__ in, long ldi,
                                 double* __restrict__ out, long ldo) {
    __shared__ double tile[TB][TB + 1];
    const long r0 = (long)blockIdx.y * TB, c0 = (long)blockIdx.x * TB;
    for (int i = threadIdx.y; i < TB; i += blockDim.y) {
        const long r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = in[r * ldi + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < TB; i += blockDim.y) {
        const long c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * ldo + r] = tile[threadIdx.x][i];
    }
}

// c = ||Rf||_F in one CTA (fixed summation order)
__global__ void fro_norm_kernel(long count, const double* __restrict__ x, double* __restrict__ c_out) {
    __shared__ double part[1024 / 32];
    double acc = 0.0;
    for (long i = threadIdx.x; i < count; i += blockDim.x) acc += x[i] * x[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *c_out = sqrt(t);
    }
}

__global__ void jw_build_kernel(int q, int l, const double* __restrict__ Rf, long ldr, const double* __restrict__ c_in,
                                double* __restrict__ J) {
    const int p = q + l;
    const double c = *c_in;
    const long total = (long)p * p;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / p), j = (int)(e % p);
        double v = 0.0;
        if (i == j)
            v = c;
        else if (i < q && j >= q)
            v = Rf[(long)i * ldr + (j - q)];
        else if (i >= q && j < q)
            v = Rf[(long)j * ldr + (i - q)];
        J[e] = v;
    }
}

__global__ void jw_sigma2_kernel(int pm, const double* __restrict__ lam, const double* __restrict__ c_in,
                                 double* __restrict__ sig2) {
    const double c = *c_in;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pm; i += gridDim.x * blockDim.x) {
        const double sg = fmax(lam[i] - c, 0.0);
        sig2[i] = sg * sg;
    }
}

__global__ void jw_split_kernel(int r, int q, int l, const double* __restrict__ lam, const double* __restrict__ c_in,
                                const double* __restrict__ Vt, long ldv, double* __restrict__ U,
                                double* __restrict__ M) {
    const double c = *c_in;
    const double rt2 = 1.4142135623730951;
    for (int i = blockIdx.x; i < r; i += gridDim.x) {
        const double sg = fmax(lam[i] - c, 0.0);
        const double* row = Vt + (long)i * ldv;
        for (int j = threadIdx.x; j < q; j += blockDim.x) U[(long)i * q + j] = rt2 * row[j];
        for (int j = threadIdx.x; j < l; j += blockDim.x) M[(long)i * l + j] = sg * rt2 * row[q + j];
    }
}

}  // namespace

void shifted_scale_rows(cudaStream_t s, int l, const double* Vt, long ldv, const double* lam, double* out,
                        long ldo) {
    if (l <= 0) return;
    note_launch();
    shifted_scale_rows_kernel<<<std::min(l, 152 * 8), 128, 0, s>>>(l, Vt, ldv, lam, out, ldo);
}

void transpose(cudaStream_t s, long rows, long cols, const double* in, long ldi, double* out, long ldo) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((unsigned)((cols + TB - 1) / TB), (unsigned)((rows + TB - 1) / TB));
    note_launch();
    transpose_kernel<<<grid, dim3(TB, 8), 0, s>>>(rows, cols, in, ldi, out, ldo);
}

void jw_build(cudaStream_t s, int q, int l, const double* Rf, double* c_dev, double* J) {
    note_launch();
    fro_norm_kernel<<<1, 1024, 0, s>>>((long)q * l, Rf, c_dev);
    const long total = (long)(q + l) * (q + l);
    note_launch();
    jw_build_kernel<<<(int)std::min<long>((total + 255) / 256, 152L * 16), 256, 0, s>>>(q, l, Rf, l, c_dev, J);
}

void jw_sigma2(cudaStream_t s, int pm, const double* lam, const double* c_dev, double* sig2) {
    if (pm <= 0) return;
    note_launch();
    jw_sigma2_kernel<<<(pm + 255) / 256, 256, 0, s>>>(pm, lam, c_dev, sig2);
}

void jw_split(cudaStream_t s, int r, int q, int l, const double* lam, const double* c_dev, const double* Vt,
              long ldv, double* U, double* M) {
    if (r <= 0) return;
    note_launch();
    jw_split_kernel<<<std::min(r, 152 * 4), 256, 0, s>>>(r, q, l, lam, c_dev, Vt, ldv, U, M);
}

}  // namespace ttsn
