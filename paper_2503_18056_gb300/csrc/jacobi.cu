// Symmetric eigensolver and rank decision of the Gram-SVD rounding
// (App. A.2 of arXiv 2503.18056: "G_A = V_A S_A^2 V_A^T, G_B = V_B S_B^2 V_B^T"
// and the truncation of App. A, note on rank truncation).
//
// Eigensolver: two-sided cyclic Jacobi with the parallel round-robin
// ("circle") ordering.  Each round applies n/2 disjoint plane rotations at
// once: G <- J^T G J, Vt <- J^T Vt.  The work unit is a row pair (p, q): the
// two rows are loaded with coalesced L2 reads, rotated on the left by their own
// J_k, then every column pair is rotated in shared memory, and the rows are
// written to the other buffer (the matrix is double-buffered so a round needs
// one grid-wide barrier).  The kernel is persistent: a cooperative launch
// guarantees co-residency and the grid barrier is a bounded spin that latches
// DEV_TIMEOUT in the status word instead of waiting forever.  Rotation angles
// follow Golub & Van Loan, Alg. 8.4.1 (symSchur2); a rotation is skipped when
// |g_pq| <= tol_rel sqrt(|g_pp g_qq|) or |g_pq| <= tol_abs, and the sweep loop
// stops after a sweep that skipped every rotation.
#include <algorithm>

#include "internal.h"

namespace ttsn {

namespace {

constexpr int JT = 256;
constexpr int MAX_SWEEPS = 40;
// control block (ints): [0] barrier count, [1] barrier generation, [2] sweeps,
// [4 .. 4+MAX_SWEEPS) rotations applied per sweep
constexpr int CTRL_INTS = 8 + MAX_SWEEPS;
constexpr long long SPIN_LIMIT = 1LL << 24;  // ~1-2 s with the 64 ns sleep

__device__ __forceinline__ void round_pair(int N, int r, int k, int& p, int& q) {
    const int m = N - 1;
    if (k == 0) {
        p = m;
        q = r;
    } else {
        p = (r + k) % m;
        q = (r - k + m) % m;
    }
    if (p > q) {
        const int t = p;
        p = q;
        q = t;
    }
}

// Grid-wide barrier with a bounded wait.  Returns false (and latches
// DEV_TIMEOUT) if the wait ran out or another CTA already latched a failure.
__device__ bool grid_barrier(int* ctrl, int* status, unsigned nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (nblocks > 1) {
            unsigned* count = reinterpret_cast<unsigned*>(ctrl);
            unsigned* gen = reinterpret_cast<unsigned*>(ctrl + 1);
            const unsigned g = atomicAdd(gen, 0u);
            __threadfence();
            const unsigned arrived = atomicAdd(count, 1u);
            if (arrived == nblocks - 1) {
                atomicExch(count, 0u);
                __threadfence();
                atomicAdd(gen, 1u);
            } else {
                long long it = 0;
                while (atomicAdd(gen, 0u) == g) {
                    if (++it > SPIN_LIMIT) {
                        ok = 0;
                        atomicOr(status, DEV_TIMEOUT);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        if (atomicAdd(status, 0) & DEV_TIMEOUT) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void jacobi_init_kernel(int n, const double* __restrict__ G, long ldg, double* g0,
                                   double* vt, long ld) {
    const long total = (long)n * n;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        g0[(long)i * ld + j] = G[(long)i * ldg + j];
        vt[(long)i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
}

__global__ void __launch_bounds__(JT)
jacobi_kernel(int n, int N, double* g0, double* g1, long ld, double* vt, double* lam_out,
              int* ctrl, int* status, double tol_rel, double tol_abs_rel) {
    extern __shared__ double sm[];
    const int npairs = N / 2;
    double* cs = sm;
    double* sn = cs + npairs;
    double* rp = sn + npairs;
    double* rq = rp + n;
    __shared__ int s_cnt;
    __shared__ int s_done;

    double* cur = g0;
    double* nxt = g1;
    // absolute skip threshold relative to the largest diagonal entry: keeps
    // rounding noise in a numerically null block from being chased forever
    __shared__ double s_dmax;
    if (threadIdx.x == 0) {
        double dm = 0.0;
        for (int i = 0; i < n; ++i) dm = fmax(dm, fabs(__ldcg(g0 + (long)i * ld + i)));
        s_dmax = dm;
    }
    __syncthreads();
    const double tol_abs = tol_abs_rel * s_dmax;
    int sweep = 0;
    for (; sweep < MAX_SWEEPS; ++sweep) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (int r = 0; r < N - 1; ++r) {
            // 1. every CTA computes all rotation angles of this round
            for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
                int p, q;
                round_pair(N, r, k, p, q);
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double a = __ldcg(cur + (long)p * ld + p);
                    const double b = __ldcg(cur + (long)q * ld + q);
                    const double o =
                        0.5 * (__ldcg(cur + (long)p * ld + q) + __ldcg(cur + (long)q * ld + p));
                    const double ao = fabs(o);
                    if (ao > tol_abs && ao > tol_rel * sqrt(fabs(a) * fabs(b))) {
                        const double tau = (b - a) / (2.0 * o);
                        const double t =
                            (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        if (k % gridDim.x == blockIdx.x) atomicAdd(&s_cnt, 1);
                    }
                }
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // 2. row-pair work items
            for (int k = blockIdx.x; k < npairs; k += gridDim.x) {
                int p, q;
                round_pair(N, r, k, p, q);
                const bool hq = q < n;  // p < q always, so p < n whenever q < n
                const bool hp = p < n;
                const double c = cs[k], s = sn[k];
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    const double xp = hp ? __ldcg(cur + (long)p * ld + j) : 0.0;
                    const double xq = hq ? __ldcg(cur + (long)q * ld + j) : 0.0;
                    rp[j] = c * xp - s * xq;
                    rq[j] = s * xp + c * xq;
                }
                __syncthreads();
                for (int kk = threadIdx.x; kk < npairs; kk += blockDim.x) {
                    int pp, qq;
                    round_pair(N, r, kk, pp, qq);
                    if (qq < n) {
                        const double c2 = cs[kk], s2 = sn[kk];
                        double a0 = rp[pp], b0 = rp[qq];
                        rp[pp] = c2 * a0 - s2 * b0;
                        rp[qq] = s2 * a0 + c2 * b0;
                        a0 = rq[pp];
                        b0 = rq[qq];
                        rq[pp] = c2 * a0 - s2 * b0;
                        rq[qq] = s2 * a0 + c2 * b0;
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0 && hq && s != 0.0) {
                    rp[q] = 0.0;
                    rq[p] = 0.0;
                }
                __syncthreads();
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    if (hp) __stcg(nxt + (long)p * ld + j, rp[j]);
                    if (hq) __stcg(nxt + (long)q * ld + j, rq[j]);
                }
                if (hq && s != 0.0) {
                    for (int j = threadIdx.x; j < n; j += blockDim.x) {
                        const double vp = __ldcg(vt + (long)p * ld + j);
                        const double vq = __ldcg(vt + (long)q * ld + j);
                        __stcg(vt + (long)p * ld + j, c * vp - s * vq);
                        __stcg(vt + (long)q * ld + j, s * vp + c * vq);
                    }
                }
                __syncthreads();
            }
            if (r == N - 2 && threadIdx.x == 0) atomicAdd(ctrl + 4 + sweep, s_cnt);
            if (!grid_barrier(ctrl, status, gridDim.x)) return;
            double* t = cur;
            cur = nxt;
            nxt = t;
        }
        if (threadIdx.x == 0) s_done = (atomicAdd(ctrl + 4 + sweep, 0) == 0);
        __syncthreads();
        if (s_done) break;
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            ctrl[2] = min(sweep + 1, MAX_SWEEPS);
            if (sweep >= MAX_SWEEPS) atomicOr(status, DEV_NOT_CONVERGED);
        }
        // eigenvalues: the diagonal of the last written buffer
        for (int i = threadIdx.x; i < n; i += blockDim.x) lam_out[i] = __ldcg(cur + (long)i * ld + i);
    }
}

// One CTA per source row j: rank of lam_j among all (descending, ties by index),
// then copy eigenvector row j and eigenvalue to their sorted positions.
__global__ void __launch_bounds__(256)
jacobi_sort_kernel(int n, const double* __restrict__ d, long ld, const double* __restrict__ vt,
                   double* lam, double* Vt, long ldv, int* sweeps_out, const int* ctrl) {
    __shared__ int s_rank[256];
    const int j = blockIdx.x;
    const double lj = d[j];
    int cnt = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double li = d[i];
        if (li > lj || (li == lj && i < j)) ++cnt;
    }
    s_rank[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_rank[threadIdx.x] += s_rank[threadIdx.x + o];
        __syncthreads();
    }
    const int rank = s_rank[0];
    if (threadIdx.x == 0) lam[rank] = lj;
    for (int i = threadIdx.x; i < n; i += blockDim.x) Vt[(long)rank * ldv + i] = vt[(long)j * ld + i];
    if (j == 0 && threadIdx.x == 0 && sweeps_out) *sweeps_out = ctrl[2];
}

__global__ void trivial_eig_kernel(const double* G, double* lam, double* Vt, int* sweeps) {
    lam[0] = G[0];
    Vt[0] = 1.0;
    if (sweeps) *sweeps = 0;
}

__global__ void truncation_kernel(const double* lamK, int kB, double eps, int dm1, int forced,
                                  int max_rank, double* delta2_dev, int* dec_i, double* dec_d) {
    const double eps_mach = 2.220446049250313e-16;
    double total = 0.0;
    for (int j = kB - 1; j >= 0; --j) total += fmax(lamK[j], 0.0);
    double delta2 = *delta2_dev;
    if (delta2 < 0.0) {
        delta2 = eps * eps * total / (double)(dm1 > 0 ? dm1 : 1);
        *delta2_dev = delta2;
    }
    int navail = 0;
    const double lmax = kB > 0 ? lamK[0] : 0.0;
    if (lmax > 0.0)
        for (int j = 0; j < kB; ++j)
            if (lamK[j] > (double)kB * eps_mach * lmax) ++navail;
    int r, capped = 0;
    if (navail == 0) {
        r = 0;
    } else if (forced > 0) {
        r = min(forced, navail);
    } else {
        // smallest r >= 1 with sum_{j >= r} sigma_j^2 <= delta^2 (summed from the tail)
        double t = 0.0;
        int rstar = 0;
        for (int j = kB - 1; j >= 0; --j) {
            const double tn = t + fmax(lamK[j], 0.0);
            if (tn > delta2) {
                rstar = j + 1;
                break;
            }
            t = tn;
        }
        r = max(1, rstar);
        if (max_rank > 0 && r > max_rank) {
            r = max_rank;
            capped = 1;
        }
        r = min(r, navail);
    }
    double tail = 0.0;
    for (int j = kB - 1; j >= r && j >= 0; --j) tail += fmax(lamK[j], 0.0);
    dec_i[0] = r;
    dec_i[1] = capped;
    dec_d[0] = delta2;
    dec_d[1] = tail;
    dec_d[2] = total;
}

__global__ void count_floor_kernel(const double* lam, int n, int* out) {
    const double eps_mach = 2.220446049250313e-16;
    int cnt = 0;
    const double lmax = n > 0 ? lam[0] : 0.0;
    if (lmax > 0.0)
        for (int j = 0; j < n; ++j)
            if (lam[j] > (double)n * eps_mach * lmax) ++cnt;
    *out = cnt;
}

int g_coop_blocks = 0;  // co-resident CTAs of jacobi_kernel at the smem size last queried

}  // namespace

void EigWork::release() {
    g0.release();
    g1.release();
    lam_unsorted.release();
    vt_unsorted.release();
    if (d_ctrl) cudaFree(d_ctrl);
    d_ctrl = nullptr;
    ctrl_cap = 0;
}

tt_status syev(cudaStream_t s, int n, const double* G, long ldg, double* lam, double* Vt, long ldv,
               EigWork& w, int* status_dev, int* sweeps_dev) {
    if (n < 0) {
        set_error("syev: negative size");
        return TT_ERR_ARG;
    }
    if (n == 0) return TT_OK;
    if (n == 1) {
        note_launch();
        trivial_eig_kernel<<<1, 1, 0, s>>>(G, lam, Vt, sweeps_dev);
        TT_CUDA_TRY(cudaGetLastError());
        return TT_OK;
    }
    const int N = n + (n & 1);
    const long ld = n;
    TT_TRY(w.g0.ensure((size_t)n * n, s));
    TT_TRY(w.g1.ensure((size_t)n * n, s));
    TT_TRY(w.vt_unsorted.ensure((size_t)n * n, s));
    if (!w.d_ctrl) {
        TT_CUDA_TRY(cudaMalloc(&w.d_ctrl, CTRL_INTS * sizeof(int)));
        w.ctrl_cap = CTRL_INTS;
    }
    TT_CUDA_TRY(cudaMemsetAsync(w.d_ctrl, 0, CTRL_INTS * sizeof(int), s));
    {
        const long total = (long)n * n;
        const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
        note_launch();
        jacobi_init_kernel<<<blocks, 256, 0, s>>>(n, G, ldg, w.g0.p, w.vt_unsorted.p, ld);
        TT_CUDA_TRY(cudaGetLastError());
    }
    const size_t smem = (size_t)(N + 2 * n) * sizeof(double);
    if (smem > 200 * 1024) {
        set_error("syev: matrix too large for the shared-memory row buffers");
        return TT_ERR_TOO_LARGE;
    }
    TT_CUDA_TRY(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    TT_CUDA_TRY(cudaGetDevice(&dev));
    TT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, JT, smem));
    if (per_sm < 1) {
        set_error("syev: jacobi kernel cannot be resident");
        return TT_ERR_CUDA;
    }
    g_coop_blocks = per_sm * sms;
    // about two row-pair items per CTA; one CTA for small matrices
    int blocks = std::max(1, std::min(N / 4, sms));
    blocks = std::min(blocks, g_coop_blocks);
    double* g0 = w.g0.p;
    double* g1 = w.g1.p;
    double* vt = w.vt_unsorted.p;
    int* ctrl = w.d_ctrl;
    TT_TRY(w.lam_unsorted.ensure((size_t)n, s));
    double* lamu = w.lam_unsorted.p;
    // relative skip test as in high-relative-accuracy Jacobi; the absolute one
    // (1e-24 of the largest diagonal entry) is far below the Gram floor
    // n eps_mach lambda_max that the rounding applies afterwards
    double tol_rel = 1e-15, tol_abs_rel = 1e-24;
    int nn = n, NN = N;
    long ldl = ld;
    void* args[] = {&nn, &NN, &g0, &g1, &ldl, &vt, &lamu, &ctrl, &status_dev, &tol_rel, &tol_abs_rel};
    note_launch();
    TT_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(blocks), dim3(JT), args,
                                            smem, s));
    note_launch();
    jacobi_sort_kernel<<<n, 256, 0, s>>>(n, w.lam_unsorted.p, ld, w.vt_unsorted.p, lam, Vt, ldv,
                                         sweeps_dev, w.d_ctrl);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

void truncation_decision(cudaStream_t s, const double* lamK, int kB, double eps, int dm1,
                         int forced, int max_rank, double* delta2_dev, int* dec_i,
                         double* dec_d) {
    note_launch();
    truncation_kernel<<<1, 1, 0, s>>>(lamK, kB, eps, dm1, forced, max_rank, delta2_dev, dec_i,
                                      dec_d);
}

void count_above_floor(cudaStream_t s, const double* lam, int n, int* out_dev) {
    note_launch();
    count_floor_kernel<<<1, 1, 0, s>>>(lam, n, out_dev);
}

}  // namespace ttsn
