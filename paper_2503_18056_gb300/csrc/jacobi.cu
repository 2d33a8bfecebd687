// Small dense factorisations of the Gram-SVD rounding (App. A.2 of arXiv
// 2503.18056) and the rank decision of App. A (note on rank truncation).
//
// 1. Symmetric eigensolver: two-sided cyclic Jacobi with the parallel
//    round-robin ("circle") ordering.  Each round applies n/2 disjoint plane
//    rotations at once: G <- J^T G J, Vt <- J^T Vt.  A CTA owns a few row pairs
//    (p, q) per round: it forms those pairs' rotation angles and publishes them,
//    loads the rows with coalesced L2 reads and rotates them on the left by
//    their own J_k; after a grid-wide barrier it reads every pair's angles,
//    rotates the non-identity column pairs in shared memory and writes the rows
//    to the other buffer (the matrix is double-buffered; a second barrier ends
//    the round).  The three entries (g_pp, g_qq, g_pq) that define the next
//    round's rotations are written by the row owners into a compact array, so
//    the owning CTA reads them with one coalesced load.  Rotation
//    angles follow Golub & Van Loan, Alg. 8.4.1 (symSchur2); a rotation is
//    skipped when |g_pq| <= tol_rel sqrt(|g_pp g_qq|) or |g_pq| <= tol_abs, and
//    the sweeps stop after one that skipped every rotation.
// 2. Pivoted Cholesky of a positive semidefinite matrix, G = W^T W with W
//    upper-trapezoidal in pivot order (left-looking, diagonal pivoting, stopped
//    when the largest remaining diagonal entry is at eps_mach max(diag G)).  The rounding
//    needs from G_B only a factor with W^T W = G_B, which this gives in n
//    sequential steps instead of an eigendecomposition.
//
// Both kernels are persistent: a cooperative launch guarantees co-residency and
// the grid barrier is a bounded spin that latches DEV_TIMEOUT in the status
// word instead of waiting forever.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include <cooperative_groups.h>

#include "internal.h"

namespace ttsn {

namespace {

constexpr int JT = 256;
constexpr int MAX_SWEEPS = JACOBI_MAX_SWEEPS;
// control block (ints): [0] barrier arrivals, [1] unused, [2] sweeps,
// [3] pivoted-Cholesky rank, [4 .. 4+MAX_SWEEPS) rotations applied per sweep
constexpr int CTRL_INTS = 8 + MAX_SWEEPS;
constexpr long long SPIN_LIMIT = 1LL << 21;  // ~1 s (an L2 acquire load plus a 32 ns sleep per try)
constexpr int MAX_PAIRS_PER_CTA = 8;

__device__ __forceinline__ void round_pair(int N, int r, int k, int& p, int& q) {
    const int m = N - 1;
    if (k == 0) {
        p = m;
        q = r;
    } else {  // (r + k) mod m and (r - k) mod m for 0 <= r < m, 0 < k < m
        p = r + k;
        if (p >= m) p -= m;
        q = r - k;
        if (q < 0) q += m;
    }
    if (p > q) {
        const int t = p;
        p = q;
        q = t;
    }
}

// Pair index and partner of index x in round r (inverse of round_pair).
__device__ __forceinline__ void pair_of(int N, int r, int x, int& k, int& partner) {
    const int m = N - 1;
    if (x == m) {
        k = 0;
        partner = r;
        return;
    }
    if (x == r) {
        k = 0;
        partner = m;
        return;
    }
    const int d = (x - r + m) % m;  // 1 .. m-1
    if (d <= N / 2 - 1) {
        k = d;
        partner = (r - d + m) % m;
    } else {
        k = m - d;
        partner = (r + k) % m;
    }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier with a bounded wait.  ctrl[0] counts arrivals over the
// whole launch (the control block is zeroed before every launch), so the
// barrier that a CTA enters for the e-th time completes when the count
// reaches e * nblocks: one release-atomic arrival per CTA, acquire-load
// polling, no reset and no second word to bump.  Returns false (and latches
// DEV_TIMEOUT) if the wait ran out; the other CTAs then never see the count
// complete and run out in turn.  epoch is the caller's barrier counter (its
// value matters in thread 0 only).
__device__ bool grid_barrier(int* ctrl, int* status, unsigned nblocks, unsigned& epoch) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        ++epoch;
        if (nblocks > 1) {
            unsigned* count = reinterpret_cast<unsigned*>(ctrl);
            const unsigned target = epoch * nblocks;
            // the CTA's writes (every thread's, ordered by the __syncthreads
            // above) become visible GPU-wide before the arrival is counted
            __threadfence();
            const unsigned old = atomicAdd(count, 1u);
            if (old + 1u < target) {
                long long it = 0;
                while (ld_acquire(count) < target) {
                    if (++it > SPIN_LIMIT) {
                        ok = 0;
                        atomicOr(status, DEV_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void jacobi_init_kernel(int n, int N, const double* __restrict__ G, long ldg, double* g0,
                                   double* vt, long ld, double* abc, const int* n_dev) {
    if (n_dev) {
        n = *n_dev;
        N = n + (n & 1);
        ldg = ld = n;
    }
    const long total = (long)n * n;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        g0[(long)i * ld + j] = G[(long)i * ldg + j];
        vt[(long)i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    // entries of the round-0 pairs
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N / 2; k += gridDim.x * blockDim.x) {
        int p, q;
        round_pair(N, 0, k, p, q);
        if (q < n) {
            abc[3 * k] = G[(long)p * ldg + p];
            abc[3 * k + 1] = G[(long)q * ldg + q];
            abc[3 * k + 2] = 0.5 * (G[(long)p * ldg + q] + G[(long)q * ldg + p]);
        } else {
            abc[3 * k] = abc[3 * k + 1] = abc[3 * k + 2] = 0.0;
        }
    }
}

// One launch runs every sweep.  A round has two grid barriers:
//  A. each CTA forms the rotation angles of the pairs it owns only (from the
//     compact entries the previous round published), publishes them, and
//     left-rotates its own row pairs and eigenvector rows;
//  B. after the barrier every CTA reads all angles with one coalesced load,
//     compacts the list of pairs whose rotation is not the identity, applies
//     those column rotations to its own rows, stores the rows to the other
//     buffer and publishes the next round's pair entries.
// Forming each angle once instead of once per CTA is what the second barrier
// buys: on GB300 a CTA that formed all n/2 angles itself spent about as long
// on their FP64 square roots and divisions as on the rotations, and skipped
// (identity) rotations cost nothing in the later sweeps.
__global__ void __launch_bounds__(JT)
jacobi_kernel(int n, int N, double* g0, double* g1, long ld, double* vt, double* abc0,
              double* abc1, double* cs_g, double* lam_out, int* ctrl, int* status, double tol_rel,
              double tol_abs_rel, int max_sweeps, const int* n_dev) {
    if (n_dev) {  // a captured step: the grid and shared memory fit the largest n
        n = *n_dev;
        N = n + (n & 1);
        ld = n;
    }
    extern __shared__ double sm[];
    const int npairs = N / 2;
    // pairs this CTA owns: k = blockIdx.x + i * gridDim.x < npairs
    const int mine = max(0, (npairs - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x);
    double* cs = sm;                                     // 2 * npairs: c, s of every pair
    double* rows = cs + 2 * npairs;                      // 2 * ppc rows of n
    int* act = reinterpret_cast<int*>(rows + 2 * (size_t)((npairs + gridDim.x - 1) / gridDim.x) * n);
    __shared__ int s_cnt;
    __shared__ int s_done;
    __shared__ int s_nact;
    __shared__ int s_wsum[JT / 32];
    __shared__ double s_dmax;

    unsigned epoch = 0;
    double* cur = g0;
    double* nxt = g1;
    double* abc_cur = abc0;
    double* abc_nxt = abc1;
    if (threadIdx.x == 0) {
        double dm = 0.0;
        for (int i = 0; i < n; ++i) dm = fmax(dm, fabs(__ldcg(g0 + (long)i * ld + i)));
        s_dmax = dm;
    }
    __syncthreads();
    const double tol_abs = tol_abs_rel * s_dmax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (int r = 0; r < N - 1; ++r) {
            const int rn = (r + 1 == N - 1) ? 0 : r + 1;  // next round (wraps to the next sweep)
            // A1. the angles of the owned pairs (Golub & Van Loan, Alg. 8.4.1)
            if (threadIdx.x < mine) {
                const int i = threadIdx.x;
                const int k = blockIdx.x + i * gridDim.x;
                int p, q;
                round_pair(N, r, k, p, q);
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double a = __ldcg(abc_cur + 3 * k);
                    const double b = __ldcg(abc_cur + 3 * k + 1);
                    const double o = __ldcg(abc_cur + 3 * k + 2);
                    const double ao = fabs(o);
                    if (ao > tol_abs && ao > tol_rel * sqrt(fabs(a) * fabs(b))) {
                        const double tau = (b - a) / (2.0 * o);
                        const double t =
                            (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        atomicAdd(&s_cnt, 1);
                    }
                }
                cs[2 * k] = c;
                cs[2 * k + 1] = s;
                __stcg(cs_g + 2 * k, c);
                __stcg(cs_g + 2 * k + 1, s);
            }
            __syncthreads();
            // A2. load and left-rotate every owned row pair; rotate its eigenvector rows
            for (int i = 0; i < mine; ++i) {
                const int k = blockIdx.x + i * gridDim.x;
                int p, q;
                round_pair(N, r, k, p, q);
                const bool hp = p < n, hq = q < n;
                const double c = cs[2 * k], s = cs[2 * k + 1];
                double* rp = rows + (2 * i) * n;
                double* rq = rp + n;
                if (s != 0.0) {
#pragma unroll 4
                    for (int j = threadIdx.x; j < n; j += blockDim.x) {
                        const double xp = __ldcg(cur + (long)p * ld + j);
                        const double xq = __ldcg(cur + (long)q * ld + j);
                        rp[j] = c * xp - s * xq;
                        rq[j] = s * xp + c * xq;
                        const double vp = __ldcg(vt + (long)p * ld + j);
                        const double vq = __ldcg(vt + (long)q * ld + j);
                        __stcg(vt + (long)p * ld + j, c * vp - s * vq);
                        __stcg(vt + (long)q * ld + j, s * vp + c * vq);
                    }
                } else {
#pragma unroll 4
                    for (int j = threadIdx.x; j < n; j += blockDim.x) {
                        rp[j] = hp ? __ldcg(cur + (long)p * ld + j) : 0.0;
                        rq[j] = hq ? __ldcg(cur + (long)q * ld + j) : 0.0;
                    }
                }
            }
            if (!grid_barrier(ctrl, status, gridDim.x, epoch)) return;
            // B1. every pair's angles, and the list of the non-identity ones
            for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
                cs[2 * k] = __ldcg(cs_g + 2 * k);
                cs[2 * k + 1] = __ldcg(cs_g + 2 * k + 1);
            }
            __syncthreads();
            {
                // block-wide compaction in pair order: chunks of blockDim.x pairs
                int base = 0;
                for (int k0 = 0; k0 < npairs; k0 += blockDim.x) {
                    const int k = k0 + threadIdx.x;
                    const bool on = k < npairs && cs[2 * k + 1] != 0.0;
                    const unsigned bal = __ballot_sync(0xffffffffu, on);
                    if (lane == 0) s_wsum[warp] = __popc(bal);
                    __syncthreads();
                    int before = 0, total = 0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                        if (w < warp) before += s_wsum[w];
                        total += s_wsum[w];
                    }
                    if (on) act[base + before + __popc(bal & ((1u << lane) - 1u))] = k;
                    base += total;
                    __syncthreads();
                }
                if (threadIdx.x == 0) s_nact = base;
            }
            __syncthreads();
            const int nact = s_nact;
            // B2. right rotations of the non-identity column pairs, on all owned rows
            const int nrows = 2 * mine;
            for (int a = threadIdx.x; a < nact; a += blockDim.x) {
                const int kk = act[a];
                int pp, qq;
                round_pair(N, r, kk, pp, qq);
                const double c2 = cs[2 * kk], s2 = cs[2 * kk + 1];
                for (int row = 0; row < nrows; ++row) {
                    double* rr = rows + row * n;
                    const double a0 = rr[pp], b0 = rr[qq];
                    rr[pp] = c2 * a0 - s2 * b0;
                    rr[qq] = s2 * a0 + c2 * b0;
                }
            }
            __syncthreads();
            // B3. exact zeros for the rotated pairs
            if (threadIdx.x < mine) {
                const int i = threadIdx.x;
                const int k = blockIdx.x + i * gridDim.x;
                int p, q;
                round_pair(N, r, k, p, q);
                if (q < n && cs[2 * k + 1] != 0.0) {
                    rows[(2 * i) * n + q] = 0.0;
                    rows[(2 * i + 1) * n + p] = 0.0;
                }
            }
            __syncthreads();
            // B4. store rows and publish the next round's entries
            for (int i = 0; i < mine; ++i) {
                const int k = blockIdx.x + i * gridDim.x;
                int p, q;
                round_pair(N, r, k, p, q);
                const bool hp = p < n, hq = q < n;
                const double* rp = rows + (2 * i) * n;
                const double* rq = rp + n;
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    if (hp) __stcg(nxt + (long)p * ld + j, rp[j]);
                    if (hq) __stcg(nxt + (long)q * ld + j, rq[j]);
                }
                if (threadIdx.x < 2) {
                    const int x = threadIdx.x == 0 ? p : q;
                    const double* rx = threadIdx.x == 0 ? rp : rq;
                    if (x < n) {
                        int k2, partner;
                        pair_of(N, rn, x, k2, partner);
                        if (partner < n) {
                            if (x < partner) {
                                __stcg(abc_nxt + 3 * k2, rx[x]);
                                __stcg(abc_nxt + 3 * k2 + 2, rx[partner]);
                            } else {
                                __stcg(abc_nxt + 3 * k2 + 1, rx[x]);
                            }
                        }
                    }
                }
            }
            if (r == N - 2 && threadIdx.x == 0) atomicAdd(ctrl + 4 + sweep, s_cnt);
            if (!grid_barrier(ctrl, status, gridDim.x, epoch)) return;
            double* t = cur;
            cur = nxt;
            nxt = t;
            t = abc_cur;
            abc_cur = abc_nxt;
            abc_nxt = t;
        }
        if (threadIdx.x == 0) s_done = (atomicAdd(ctrl + 4 + sweep, 0) == 0);
        __syncthreads();
        if (s_done) break;
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            ctrl[2] = min(sweep + 1, max_sweeps);
            if (sweep >= max_sweeps) atomicOr(status, DEV_NOT_CONVERGED);
        }
        // eigenvalues: the diagonal of the last written buffer
        for (int i = threadIdx.x; i < n; i += blockDim.x) lam_out[i] = __ldcg(cur + (long)i * ld + i);
    }
}

// One-sided Jacobi on the rows of a factor W (k x n, ld n) with W^T W = K
// (Demmel & Veselic, SIAM J. Matrix Anal. Appl. 13, 1992: the eigenpairs of a
// positive definite matrix from its Cholesky factor by one-sided Jacobi, as
// accurate as two-sided Jacobi on K).  Row pairs follow the same round-robin
// ordering; one warp owns a pair for the round: it forms c = w_p . w_q, and
// if |c| > tol sqrt(a b) (a, b the squared row norms, kept in nrm) rotates the
// two rows so that they become orthogonal and recomputes their norms from the
// rotated rows.  A rotation touches only its own two rows, so a round needs
// one grid barrier and no exchange of angles.  On convergence the rows are
// orthogonal: K = sum_i w_i w_i^T, eigenvalue ||w_i||^2, eigenvector
// w_i / ||w_i||; rows k .. n-1 (K's null space below the factor's floor)
// get eigenvalue 0 and a zero vector.  A negative rank (the factorisation met
// Inf or NaN) gives NaN eigenvalues, which the rank decision reports.
constexpr int OSJ_MAX_WARPS = 8;
constexpr int OSJ_CLUSTER_N = 256;  // sizes solved on one thread-block cluster

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One pair: c = w_p . w_q, the rotation if it is needed, the rotated rows'
// norms.  C > 0: the lane's n / 32 entries of both rows are held in registers
// (all loads issued at once: one L2 round trip per pair); C == 0 streams the
// rows (any n).  Returns whether it rotated.
template <int C>
__device__ __forceinline__ bool osj_pair(double* wp, double* wq, int n, int lane, double* nrm_p, double* nrm_q,
                                         double tol) {
    double x[C > 0 ? C : 1], y[C > 0 ? C : 1];
    double c;
    if (C > 0) {
#pragma unroll
        for (int t = 0; t < C; ++t) {
            const int j = lane + 32 * t;
            x[t] = j < n ? __ldcg(wp + j) : 0.0;
            y[t] = j < n ? __ldcg(wq + j) : 0.0;
        }
        double c0 = 0.0, c1 = 0.0;
#pragma unroll
        for (int t = 0; t < C; t += 2) {
            c0 = fma(x[t], y[t], c0);
            if (t + 1 < C) c1 = fma(x[t + 1], y[t + 1], c1);
        }
        c = warp_sum(c0 + c1);
    } else {
        double c0 = 0.0, c1 = 0.0;
        int j = lane;
        for (; j + 32 < n; j += 64) {
            c0 = fma(__ldcg(wp + j), __ldcg(wq + j), c0);
            c1 = fma(__ldcg(wp + j + 32), __ldcg(wq + j + 32), c1);
        }
        if (j < n) c0 = fma(__ldcg(wp + j), __ldcg(wq + j), c0);
        c = warp_sum(c0 + c1);
    }
    const double a = __ldcg(nrm_p), b = __ldcg(nrm_q);
    if (!(a > 0.0 && b > 0.0 && fabs(c) > tol * sqrt(a * b))) return false;
    // Golub & Van Loan, Alg. 8.4.1 on [[a, c], [c, b]]
    const double tau = (b - a) / (2.0 * c);
    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    const double cs = 1.0 / sqrt(1.0 + t * t);
    const double sn = t * cs;
    // the rotation moves t c from one squared norm to the other: the growing
    // one is updated by that sum (no cancellation), the shrinking one is
    // summed again from the rotated row
    const bool p_shrinks = t * c > 0.0;
    double ns = 0.0;
    if (C > 0) {
#pragma unroll
        for (int t2 = 0; t2 < C; ++t2) {
            const int j = lane + 32 * t2;
            const double xn = cs * x[t2] - sn * y[t2];
            const double yn = sn * x[t2] + cs * y[t2];
            if (j < n) {
                __stcg(wp + j, xn);
                __stcg(wq + j, yn);
            }
            const double v = p_shrinks ? xn : yn;
            ns = fma(v, v, ns);
        }
    } else {
        for (int j = lane; j < n; j += 32) {
            const double xo = __ldcg(wp + j), yo = __ldcg(wq + j);
            const double xn = cs * xo - sn * yo;
            const double yn = sn * xo + cs * yo;
            __stcg(wp + j, xn);
            __stcg(wq + j, yn);
            const double v = p_shrinks ? xn : yn;
            ns = fma(v, v, ns);
        }
    }
    ns = warp_sum(ns);
    if (lane == 0) {
        __stcg(nrm_p, p_shrinks ? ns : a - t * c);
        __stcg(nrm_q, p_shrinks ? b + t * c : ns);
    }
    return true;
}

// Squared norms of rows 0 .. k-1, summed from the rows (one warp per row).
__device__ __forceinline__ void osj_norms(const double* W, int n, int k, double* nrm, int gw, int nw, int lane) {
    for (int i = gw; i < k; i += nw) {
        const double* wi = W + (long)i * n;
        double a = 0.0;
        for (int j = lane; j < n; j += 32) {
            const double v = __ldcg(wi + j);
            a = fma(v, v, a);
        }
        a = warp_sum(a);
        if (lane == 0) __stcg(nrm + i, a);
    }
}

// The round barrier: the whole grid (bounded spin, DEV_TIMEOUT on expiry) or,
// for a launch of one thread-block cluster, the hardware cluster barrier.
template <bool CLUSTER>
__device__ __forceinline__ bool osj_barrier(int* ctrl, int* status, unsigned& epoch) {
    if (CLUSTER) {
        cooperative_groups::this_cluster().sync();
        return true;
    }
    return grid_barrier(ctrl, status, gridDim.x, epoch);
}

template <int C, bool CLUSTER>
__global__ void __launch_bounds__(32 * OSJ_MAX_WARPS)
osj_kernel(int n, const int* __restrict__ k_dev, double* W, double* nrm, double* lam_u, double* vt_u, int* ctrl,
           int* status, int max_sweeps, const int* n_dev) {
    if (n_dev) {  // a captured step: sizes up to OSJ_CLUSTER_N take the cluster launch, larger the grid
        n = *n_dev;
        if (CLUSTER ? n > OSJ_CLUSTER_N : n <= OSJ_CLUSTER_N) return;  // every CTA, before any barrier
    }
    // relative skip threshold sqrt(n) eps_mach, the one of LAPACK's one-sided
    // Jacobi SVD (dgesvj): the typical rounding error of a computed inner
    // product of length n, so rounding noise does not keep pairs rotating
    const double tol = sqrt((double)n) * 2.220446049250313e-16;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
    const int nw = gridDim.x * wpb;
    const int kraw = *k_dev;
    if (kraw < 0) {  // every CTA returns before any barrier
        for (int i = gw; i < n; i += nw) {
            if (lane == 0) lam_u[i] = __longlong_as_double(0x7ff8000000000000LL);
            for (int j = lane; j < n; j += 32) vt_u[(long)i * n + j] = 0.0;
        }
        return;
    }
    const int k = min(kraw, n);
    unsigned epoch = 0;
    __shared__ int s_cnt;
    __shared__ int s_done;
    const int N = k + (k & 1), npairs = N / 2;
    int sweep = 0;
    if (k >= 2) {
        for (; sweep < max_sweeps; ++sweep) {
            if (threadIdx.x == 0) s_cnt = 0;
            // norms summed afresh at every sweep: the updates inside a sweep
            // only steer the angles and the skip test
            osj_norms(W, n, k, nrm, gw, nw, lane);
            if (!osj_barrier<CLUSTER>(ctrl, status, epoch)) return;
            int mine = 0;
            for (int r = 0; r < N - 1; ++r) {
                for (int kk = gw; kk < npairs; kk += nw) {
                    int p, q;
                    round_pair(N, r, kk, p, q);
                    if (q >= k) continue;
                    if (osj_pair<C>(W + (long)p * n, W + (long)q * n, n, lane, nrm + p, nrm + q, tol)) ++mine;
                }
                if (r == N - 2) {
                    if (lane == 0 && mine) atomicAdd(&s_cnt, mine);
                    __syncthreads();
                    if (threadIdx.x == 0) atomicAdd(ctrl + 4 + sweep, s_cnt);
                }
                if (!osj_barrier<CLUSTER>(ctrl, status, epoch)) return;
            }
            if (threadIdx.x == 0) s_done = (atomicAdd(ctrl + 4 + sweep, 0) == 0);
            __syncthreads();
            if (s_done) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl[2] = k >= 2 ? min(sweep + 1, max_sweeps) : 0;
        if (k >= 2 && sweep >= max_sweeps) atomicOr(status, DEV_NOT_CONVERGED);
    }
    // eigenvalues: the converged rows' squared norms, summed from the rows
    osj_norms(W, n, k, nrm, gw, nw, lane);
    if (!osj_barrier<CLUSTER>(ctrl, status, epoch)) return;
    for (int i = gw; i < n; i += nw) {
        const double a = i < k ? __ldcg(nrm + i) : 0.0;
        const double f = a > 0.0 ? 1.0 / sqrt(a) : 0.0;
        if (lane == 0) lam_u[i] = a;
        const double* wi = W + (long)i * n;
        for (int j = lane; j < n; j += 32) vt_u[(long)i * n + j] = i < k ? f * __ldcg(wi + j) : 0.0;
    }
}

// Pivoted Cholesky on one thread-block cluster for n <= PCHOL_SMALL_N: the
// same factorisation as pchol_kernel (pivot = largest remaining diagonal
// entry, ties to the lowest index, stop at the floor, -inf marks pivoted
// columns, the same per-column sums), with contiguous blocks of cpc columns
// per CTA, one thread per column, and the CTA's columns of W held in its
// shared memory.  A pivot: every CTA reads the CTAs' candidate (value,
// column) pairs from distributed shared memory and takes the same pivot p,
// reads W[0..k)[p] from the owner's shared memory, forms row k of W for its
// columns, updates their residual diagonal and posts its candidate for the
// next pivot; one hardware cluster barrier (release / acquire at cluster
// scope) ends the pivot.  On GB300 a pivot's n k FP64 FMAs are more than one
// SM absorbs (~1.7 FMA per clock) and a grid-wide barrier per pivot costs
// microseconds; a cluster spreads the FMAs over CL SMs for a barrier well
// under a microsecond.  Candidates are double-buffered by the pivot's
// parity, so a CTA never overwrites a slot another CTA may still read.
constexpr int PCHOL_SMALL_N = 384;

__global__ void __launch_bounds__(256)
pchol_cluster_kernel(int n, int cpc, const double* __restrict__ G, long ldg, double* W, int* kB_out,
                     double floor_rel, const int* n_dev, int nsmall) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    if (n_dev) {  // a captured step: the size is the device's; larger sizes take pchol_kernel
        n = *n_dev;
        ldg = n;
        if (n > nsmall) return;  // every CTA of the cluster, before any barrier
        if (n <= 0) {
            if (rank == 0 && threadIdx.x == 0) *kB_out = 0;
            return;
        }
    }
    extern __shared__ double sm[];
    double* Wl = sm;                         // rows 0..k) of this CTA's cpc columns (n x cpc)
    double* colp = sm + (size_t)n * cpc;     // W[0..k)[p]
    __shared__ double s_cv[2];  // candidate value per parity
    __shared__ int s_ci[2];     // candidate column per parity
    __shared__ double s_wv[8];
    __shared__ int s_wi[8];
    __shared__ int s_bad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    const int jl = threadIdx.x;
    const int j = rank * cpc + jl;
    const bool own = jl < cpc && j < n;
    double dj = own ? G[(long)j * ldg + j] : -1.0;
    // block candidate of (value, index), ties to the lowest index
    auto post = [&](double v, int idx, int par) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
            if (v2 > v || (v2 == v && i2 < idx)) {
                v = v2;
                idx = i2;
            }
        }
        if (lane == 0) {
            s_wv[warp] = v;
            s_wi[warp] = idx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = -1.0;
            int bi = n;
            for (int w = 0; w < nwarps; ++w)
                if (s_wv[w] > b || (s_wv[w] == b && s_wi[w] < bi)) {
                    b = s_wv[w];
                    bi = s_wi[w];
                }
            s_cv[par] = b;
            s_ci[par] = bi;
        }
    };
    // the cluster's candidate, read from every CTA's slot (after a barrier):
    // lane r of every warp reads CTA r's slot, a shuffle tree takes the best
    auto gather = [&](int par, double& b, int& bi) {
        b = -1.0;
        bi = n;
        if (lane < CL) {
            b = *cl.map_shared_rank(&s_cv[par], lane);
            bi = *cl.map_shared_rank(&s_ci[par], lane);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, b, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (v2 > b || (v2 == b && i2 < bi)) {
                b = v2;
                bi = i2;
            }
        }
    };
    // Inf or NaN on the diagonal (a Gram matrix shows any non-finite entry of
    // its factor there): rank -1 reports it instead of factorising
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    if (own && !isfinite(dj)) atomicOr(&s_bad, 1);
    __syncthreads();
    // the largest diagonal entry (the floor's scale) and the first pivot
    post(own ? dj : -1.0, own ? j : n, 0);
    if (threadIdx.x == 0 && s_bad) s_cv[0] = __longlong_as_double(0x7ff8000000000000LL);  // NaN marks it
    cl.sync();
    const int anybad = __any_sync(0xffffffffu, lane < CL && isnan(*cl.map_shared_rank(&s_cv[0], lane)));
    if (anybad) {
        cl.sync();  // every CTA has read the slots before any CTA exits
        if (rank == 0 && threadIdx.x == 0) *kB_out = -1;
        return;
    }
    double dmax;
    int p;
    gather(0, dmax, p);
    const double floor_abs = floor_rel * dmax;
    double dp = dmax;
    int par = 0;
    int k = 0;
    for (; k < n; ++k) {
        if (!(dp > floor_abs) || p >= n) break;
        const double l = sqrt(dp);
        {
            const double* Wo = cl.map_shared_rank(Wl, p / cpc);  // the owner's columns
            const int pl = p % cpc;
            for (int m = threadIdx.x; m < k; m += blockDim.x) colp[m] = Wo[(size_t)m * cpc + pl];
        }
        __syncthreads();
        if (own) {
            double w;
            if (j == p) {
                w = l;
                dj = -INFINITY;
            } else if (dj == -INFINITY) {
                w = 0.0;
            } else {
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                int m = 0;
                for (; m + 3 < k; m += 4) {
                    a0 += colp[m] * Wl[(size_t)m * cpc + jl];
                    a1 += colp[m + 1] * Wl[(size_t)(m + 1) * cpc + jl];
                    a2 += colp[m + 2] * Wl[(size_t)(m + 2) * cpc + jl];
                    a3 += colp[m + 3] * Wl[(size_t)(m + 3) * cpc + jl];
                }
                for (; m < k; ++m) a0 += colp[m] * Wl[(size_t)m * cpc + jl];
                w = (G[(long)p * ldg + j] - ((a0 + a1) + (a2 + a3))) / l;
                dj = dj - w * w;
            }
            Wl[(size_t)k * cpc + jl] = w;
            __stcg(W + (long)k * n + j, w);
        }
        par ^= 1;
        post(own && dj != -INFINITY ? dj : -1.0, own && dj != -INFINITY ? j : n, par);
        cl.sync();
        gather(par, dp, p);
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
    if (rank == 0 && threadIdx.x == 0) *kB_out = k;
}

// One CTA per source row j: rank of lam_j among all (descending, ties by index),
// then copy eigenvector row j and eigenvalue to their sorted positions.
__global__ void __launch_bounds__(256)
jacobi_sort_kernel(int n, const double* __restrict__ d, long ld, const double* __restrict__ vt,
                   double* lam, double* Vt, long ldv, int* sweeps_out, const int* ctrl, const int* n_dev) {
    if (n_dev) {
        n = *n_dev;
        ld = ldv = n;
        if ((int)blockIdx.x >= n) return;
    }
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

// ------------------------------------------------------------ pivoted Cholesky
// Left-looking: W[k][j] = (G[p][j] - sum_{m<k} Wc[p][m] Wc[j][m]) / sqrt(d_p) with
// p = argmax of the remaining diagonal d.  W (n x n rows used: k < rank,
// row-major) and its transpose Wc (n x n, Wc[j][m] = W[m][j]) are both written
// so every dot product reads contiguous memory.  d[j] = -inf marks pivoted
// columns; a residual that rounds below zero is only never chosen as a pivot
// (its later entries of W are still formed: treating it as pivoted would drop
// them, up to sqrt(eps_mach) of the pivots' scale each).
// The residual diagonal is double-buffered (2 n entries): step k reads
// d[k & 1] and writes d[(k + 1) & 1], so a CTA that still searches step k's
// pivot never sees another CTA's step-k updates (with one buffer a slow CTA
// could pick a different pivot once the fast ones had marked theirs).
__global__ void __launch_bounds__(JT)
pchol_kernel(int n, const double* __restrict__ G, long ldg, double* W, double* Wc, double* d,
             int* ctrl, int* status, double floor_rel, const int* n_dev, int nsmall) {
    if (n_dev) {  // a captured step: sizes up to nsmall go to pchol_cluster_kernel
        n = *n_dev;
        ldg = n;
        if (n <= nsmall) return;  // every CTA, before any barrier
    }
    unsigned epoch = 0;
    extern __shared__ double sm[];
    double* colp = sm;  // Wc[p][0..k)
    __shared__ double s_val[JT];
    __shared__ int s_idx[JT];
    __shared__ double s_dmax0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // every CTA reads the initial diagonal (G is an input and is not written)
    double dm = 0.0;
    int bad = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double x = G[(long)j * ldg + j];
        dm = fmax(dm, x);
        bad |= !isfinite(x);
    }
    // Inf or NaN on the diagonal: every CTA reads all of it, so all leave here
    // together (before the first grid barrier) and rank -1 reports it
    if (__syncthreads_or(bad)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctrl[3] = -1;
        return;
    }
    s_val[threadIdx.x] = dm;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_val[threadIdx.x] = fmax(s_val[threadIdx.x], s_val[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) s_dmax0 = s_val[0];
    __syncthreads();
    const double floor_abs = floor_rel * s_dmax0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        __stcg(d + j, G[(long)j * ldg + j]);
    if (!grid_barrier(ctrl, status, gridDim.x, epoch)) return;
    int k = 0;
    for (; k < n; ++k) {
        const double* dcur = d + (size_t)(k & 1) * n;
        double* dnext = d + (size_t)((k + 1) & 1) * n;
        // argmax of the remaining diagonal (identical in every CTA; ties -> lowest index)
        double best = -1.0;
        int bi = n;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double v = __ldcg(dcur + j);
            if (v > best) {
                best = v;
                bi = j;
            }
        }
        s_val[threadIdx.x] = best;
        s_idx[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                const double v2 = s_val[threadIdx.x + o];
                const int i2 = s_idx[threadIdx.x + o];
                if (v2 > s_val[threadIdx.x] || (v2 == s_val[threadIdx.x] && i2 < s_idx[threadIdx.x])) {
                    s_val[threadIdx.x] = v2;
                    s_idx[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        const double dp = s_val[0];
        const int p = s_idx[0];
        __syncthreads();
        if (!(dp > floor_abs) || p >= n) break;
        const double l = sqrt(dp);
        for (int m = threadIdx.x; m < k; m += blockDim.x) colp[m] = __ldcg(Wc + (long)p * n + m);
        __syncthreads();
        // this CTA's columns j = blockIdx.x + c * gridDim.x, one warp per column
        for (int j = blockIdx.x + warp * gridDim.x; j < n; j += nwarps * gridDim.x) {
            const double dj = __ldcg(dcur + j);
            const bool pivoted = dj == -INFINITY;
            double acc = 0.0;
            if (!pivoted && j != p)
                for (int m = lane; m < k; m += 32) acc += colp[m] * __ldcg(Wc + (long)j * n + m);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                double w;
                if (j == p) {
                    w = l;
                    __stcg(dnext + j, -INFINITY);
                } else if (pivoted) {
                    w = 0.0;
                    __stcg(dnext + j, dj);
                } else {
                    w = (G[(long)p * ldg + j] - acc) / l;
                    __stcg(dnext + j, dj - w * w);
                }
                __stcg(W + (long)k * n + j, w);
                __stcg(Wc + (long)j * n + k, w);
            }
        }
        if (!grid_barrier(ctrl, status, gridDim.x, epoch)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl[3] = k;
}

__global__ void pchol_finish_kernel(const int* ctrl, int* kB_out, const int* n_dev, int nsmall) {
    if (n_dev && *n_dev <= nsmall) return;
    *kB_out = ctrl[3];
}

// Self-test of the bounded wait: one CTA enters grid_barrier claiming a grid
// of two, so the second arrival never comes; the wait runs out after its
// iteration limit (~1 s), latches DEV_TIMEOUT and the kernel returns.
__global__ void wait_probe_kernel(int* ctrl, int* status) {
    unsigned epoch = 0;
    if (grid_barrier(ctrl, status, 2u, epoch) && threadIdx.x == 0) atomicOr(status, 0);
}

__global__ void truncation_kernel(const double* lamK, int kB, double eps, int dm1, int forced,
                                  int max_rank, double* delta2_dev, int* dec_i, double* dec_d,
                                  const int* kB_dev, int sv) {
    if (kB_dev) kB = *kB_dev > 0 ? *kB_dev : 0;
    const double eps_mach = 2.220446049250313e-16;
    // totals and tails are summed from the small end; eigenvalues are not clamped
    // at zero, so the symmetric rounding noise of the Gram eigenvalues cancels
    double total = 0.0;
    for (int j = kB - 1; j >= 0; --j) total += lamK[j];
    // an Inf or NaN anywhere in the tensor reaches the eigenvalues (or their
    // sum); the host reports it instead of rounding to the zero tensor
    dec_i[2] = isfinite(total) ? 0 : 1;
    total = fmax(total, 0.0);
    double delta2 = *delta2_dev;
    if (delta2 < 0.0) {
        delta2 = eps * eps * total / (double)(dm1 > 0 ? dm1 : 1);
        *delta2_dev = delta2;
    }
    // floor: Gram eigenvalues are resolved to kB eps_mach of the largest;
    // squared singular values from an SVD (sv) to the square of that
    int navail = 0;
    const double lmax = kB > 0 ? lamK[0] : 0.0;
    const double fl = sv ? ((double)kB * eps_mach) * ((double)kB * eps_mach) : (double)kB * eps_mach;
    if (lmax > 0.0)
        for (int j = 0; j < kB; ++j)
            if (lamK[j] > fl * lmax) ++navail;
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
            const double tn = t + lamK[j];
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
    for (int j = kB - 1; j >= r && j >= 0; --j) tail += lamK[j];
    dec_i[0] = r;
    dec_i[1] = capped;
    dec_d[0] = delta2;
    dec_d[1] = fmax(tail, 0.0);
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

tt_status coop_blocks(const void* fn, size_t smem, int want, int* out) {
    int dev = 0, sms = 0, per_sm = 0;
    TT_CUDA_TRY(cudaGetDevice(&dev));
    TT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, JT, smem));
    if (per_sm < 1) {
        set_error("persistent kernel cannot be resident with its shared memory");
        return TT_ERR_CUDA;
    }
    *out = std::max(1, std::min(want, std::min(sms, per_sm * sms)));
    return TT_OK;
}

tt_status ensure_ctrl(EigWork& w, cudaStream_t s) {
    if (!w.d_ctrl) {
        TT_TRY(w.ctrl_buf.ensure((CTRL_INTS * sizeof(int) + 7) / 8, s));
        w.d_ctrl = reinterpret_cast<int*>(w.ctrl_buf.p);
        w.ctrl_cap = CTRL_INTS;
    }
    TT_CUDA_TRY(cudaMemsetAsync(w.d_ctrl, 0, CTRL_INTS * sizeof(int), s));
    return TT_OK;
}

}  // namespace

void EigWork::release() {
    cs.release();
    g0.release();
    g1.release();
    lam_unsorted.release();
    vt_unsorted.release();
    abc.release();
    psd.release();
    ctrl_buf.release();
    d_ctrl = nullptr;
    ctrl_cap = 0;
}

tt_status syev(cudaStream_t s, int n, const double* G, long ldg, double* lam, double* Vt, long ldv,
               EigWork& w, int* status_dev, int* sweeps_dev, int max_sweeps) {
    if (n < 0) {
        set_error("syev: negative size");
        return TT_ERR_ARG;
    }
    if (max_sweeps < 1 || max_sweeps > MAX_SWEEPS) {
        set_error("syev: the sweep limit must be in 1 .. " + std::to_string(MAX_SWEEPS));
        return TT_ERR_ARG;
    }
    if (n == 0) return TT_OK;
    if (n == 1) {
        note_launch();
        trivial_eig_kernel<<<1, 1, 0, s>>>(G, lam, Vt, sweeps_dev);
        TT_CUDA_TRY(cudaGetLastError());
        return TT_OK;
    }
    // relative skip test as in high-relative-accuracy Jacobi; the absolute one
    // (1e-20 of the largest diagonal entry) only skips rotations inside the
    // block of eigenvalues below the Gram floor n eps_mach lambda_max that the
    // rounding discards afterwards: on the rounding's K matrices it ends the
    // iteration 1-3 sweeps earlier than 1e-24 with the same eigenpairs above
    // the floor.  (One CTA would save the grid barrier per round but not the
    // round's ~n^2 FP64 FMAs, which one SM's share of GB300's FP64 rate cannot
    // absorb: measured 1.1 ms mean per eigensolve at n <= 96.)
    double tol_rel = 1e-15, tol_abs_rel = 1e-20;
    const int N = n + (n & 1);
    const int npairs = N / 2;
    const long ld = n;
    TT_TRY(w.g0.ensure((size_t)n * n, s));
    TT_TRY(w.g1.ensure((size_t)n * n, s));
    TT_TRY(w.vt_unsorted.ensure((size_t)n * n, s));
    TT_TRY(w.lam_unsorted.ensure((size_t)n, s));
    TT_TRY(w.abc.ensure((size_t)6 * npairs, s));
    TT_TRY(w.cs.ensure((size_t)2 * npairs, s));
    TT_TRY(ensure_ctrl(w, s));
    // one row pair per CTA where the GPU holds that many CTAs: a round's FP64
    // work per CTA (about 18 n flops per owned pair) is what bounds the round
    // on GB300's FP64 pipe, so the pairs are spread over as many SMs as exist.
    // Shared memory: all angles, the owned rows, the list of active pairs.
    auto smem_for = [&](int ppc) {
        return (size_t)(npairs * 2 + 2 * (size_t)ppc * n) * sizeof(double) + (size_t)npairs * sizeof(int);
    };
    int want = npairs;
    // the row buffers for MAX_PAIRS_PER_CTA pairs where they fit; above that
    // (n > ~1480) for the pairs each SM must own
    size_t smem = smem_for(MAX_PAIRS_PER_CTA);
    if (smem > 200 * 1024) {
        int dev = 0, sms = 1;
        TT_CUDA_TRY(cudaGetDevice(&dev));
        TT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        smem = smem_for(std::min(MAX_PAIRS_PER_CTA, (npairs + sms - 1) / sms));
    }
    if (smem > 200 * 1024) {
        set_error("syev: matrix too large for the shared-memory row buffers");
        return TT_ERR_TOO_LARGE;
    }
    TT_TRY(ensure_max_dynamic_smem((const void*)jacobi_kernel));
    int blocks = 1;
    TT_TRY(coop_blocks((const void*)jacobi_kernel, smem, want, &blocks));
    const int ppc = (npairs + blocks - 1) / blocks;
    if (ppc > MAX_PAIRS_PER_CTA || smem_for(ppc) > smem) {
        set_error("syev: too few resident CTAs for this matrix size");
        return TT_ERR_TOO_LARGE;
    }
    {
        const long total = (long)n * n;
        const int ib = (int)std::min<long>((total + 255) / 256, 152L * 16);
        note_launch();
        jacobi_init_kernel<<<ib, 256, 0, s>>>(n, N, G, ldg, w.g0.p, w.vt_unsorted.p, ld, w.abc.p, nullptr);
        TT_CUDA_TRY(cudaGetLastError());
    }
    double* g0 = w.g0.p;
    double* g1 = w.g1.p;
    double* vt = w.vt_unsorted.p;
    double* abc0 = w.abc.p;
    double* abc1 = w.abc.p + 3 * npairs;
    double* lamu = w.lam_unsorted.p;
    double* csg = w.cs.p;
    int* ctrl = w.d_ctrl;
    int nn = n, NN = N;
    long ldl = ld;
    int msw = max_sweeps;
    const int* nnull = nullptr;
    void* args[] = {&nn, &NN, &g0, &g1, &ldl, &vt, &abc0, &abc1, &csg, &lamu, &ctrl, &status_dev, &tol_rel,
                    &tol_abs_rel, &msw, &nnull};
    note_launch();
    TT_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(blocks), dim3(JT), args,
                                            smem, s));
    note_launch();
    jacobi_sort_kernel<<<n, 256, 0, s>>>(n, w.lam_unsorted.p, ld, w.vt_unsorted.p, lam, Vt, ldv,
                                         sweeps_dev, w.d_ctrl, nullptr);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

// Largest cluster (16, else 8) the GPU schedules for a kernel of `threads`
// threads and no dynamic shared memory, found once per kernel.
int cluster_size_for(const void* fn, int threads) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, int>> known;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& kv : known)
        if (kv.first == fn) return kv.second;
    int cl = 8;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = 160 * 1024;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) == cudaSuccess && nc > 0) cl = 16;
    }
    (void)cudaGetLastError();
    known.emplace_back(fn, cl);
    return cl;
}

// Largest n the cluster factorisation takes: at most PCHOL_SMALL_N, and its
// columns of W must fit a CTA's shared memory (n ceil(n / CL) + n doubles).
int pchol_small_limit() {
    const int cl = cluster_size_for((const void*)pchol_cluster_kernel, 256);
    int n = PCHOL_SMALL_N;
    while (n > 0 && ((size_t)n * ((n + cl - 1) / cl) + n) * sizeof(double) > 200 * 1024) --n;
    return n;
}

tt_status launch_pchol_cluster(cudaStream_t s, int n, const double* G, long ldg, double* W, int* kB_dev,
                               const int* n_dev, int nsmall) {
    const int cl = cluster_size_for((const void*)pchol_cluster_kernel, 256);
    const int cpc = (n + cl - 1) / cl;
    const int threads = std::max(32, (cpc + 31) / 32 * 32);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = ((size_t)n * cpc + n) * sizeof(double);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // stop at the rounding-noise level of G's entries (eps_mach max diag)
    const double fr = 2.220446049250313e-16;
    note_launch();
    TT_CUDA_TRY(cudaLaunchKernelEx(&cfg, pchol_cluster_kernel, n, cpc, G, ldg, W, kB_dev, fr, n_dev, nsmall));
    return TT_OK;
}

tt_status osj_launch(cudaStream_t s, int ncap, const int* k_dev, EigWork& w, int* status_dev, int max_sweeps,
                     const int* n_dev, double* nrm) {
    TT_TRY(ensure_ctrl(w, s));  // zero barrier and sweep counters (pchol used them)
    int nn = ncap;
    double* Wp = w.g0.p;
    double* lamu = w.lam_unsorted.p;
    double* vtu = w.vt_unsorted.p;
    int* ctrl = w.d_ctrl;
    int msw = max_sweeps;
    if (ncap <= OSJ_CLUSTER_N || n_dev) {
        // one cluster: a round ends at a hardware cluster barrier instead of a
        // grid-wide one; its CL SMs hold up to OSJ_MAX_WARPS pairs each.  A
        // captured step launches it for sizes up to OSJ_CLUSTER_N and the
        // grid kernel after it for larger ones (each returns at once
        // outside its range), so a replay takes the host path's kernel.
        const int ncl = std::min(ncap, OSJ_CLUSTER_N);
        const int cl = cluster_size_for((const void*)osj_kernel<8, true>, 32 * OSJ_MAX_WARPS);
        const int npairs = (ncl + 1) / 2;
        const int wpb = std::max(1, std::min(OSJ_MAX_WARPS, (npairs + cl - 1) / cl));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(32 * wpb);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        note_launch();
        TT_CUDA_TRY(cudaLaunchKernelEx(&cfg, osj_kernel<8, true>, nn, k_dev, Wp, nrm, lamu, vtu, ctrl, status_dev,
                                       msw, n_dev));
        if (ncap <= OSJ_CLUSTER_N) return TT_OK;
    }
    // rows in registers up to n = 1024 (entries per lane: 8, 16 or 32)
    const void* fn = ncap <= 256 ? (const void*)osj_kernel<8, false>
                     : ncap <= 512 ? (const void*)osj_kernel<16, false>
                     : ncap <= 1024 ? (const void*)osj_kernel<32, false> : (const void*)osj_kernel<0, false>;
    // one CTA per SM with one warp per pair it owns, so every SM carries the
    // same number of pairs in a round (the round ends at the slowest SM)
    int blocks = 1, wpb = 1;
    {
        int dev = 0, sms = 0, per_sm = 0;
        TT_CUDA_TRY(cudaGetDevice(&dev));
        TT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int npairs = (ncap + 1) / 2;
        wpb = std::max(1, std::min(OSJ_MAX_WARPS, (npairs + sms - 1) / sms));
        TT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * wpb, 0));
        if (per_sm < 1) {
            set_error("one-sided Jacobi kernel cannot be resident");
            return TT_ERR_CUDA;
        }
        blocks = std::max(1, std::min((npairs + wpb - 1) / wpb, per_sm * sms));
    }
    void* args[] = {&nn, &k_dev, &Wp, &nrm, &lamu, &vtu, &ctrl, &status_dev, &msw, &n_dev};
    note_launch();
    TT_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(32 * wpb), args, 0, s));
    return TT_OK;
}

tt_status wait_probe(cudaStream_t s, EigWork& w, int* status_dev) {
    TT_TRY(ensure_ctrl(w, s));
    note_launch();
    wait_probe_kernel<<<1, 32, 0, s>>>(w.d_ctrl, status_dev);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status pchol(cudaStream_t s, int n, const double* G, long ldg, double* W, double* Wc,
                double* dwork, EigWork& w, int* status_dev, int* kB_dev) {
    if (n <= 0) return TT_OK;
    TT_TRY(ensure_ctrl(w, s));
    const size_t smem = (size_t)n * sizeof(double);
    if (smem > 200 * 1024) {
        set_error("pchol: matrix too large");
        return TT_ERR_TOO_LARGE;
    }
    TT_TRY(ensure_max_dynamic_smem((const void*)pchol_kernel));
    const int nsmall = pchol_small_limit();
    if (n <= nsmall) return launch_pchol_cluster(s, n, G, ldg, W, kB_dev, nullptr, nsmall);
    int blocks = 1;
    // about eight columns per CTA (one warp each)
    TT_TRY(coop_blocks((const void*)pchol_kernel, smem, std::max(1, (n + 7) / 8), &blocks));
    int nn = n;
    long ldgl = ldg;
    const double* Gp = G;
    int* ctrl = w.d_ctrl;
    // stop at the rounding-noise level of G's entries (eps_mach max diag): a
    // higher floor (n eps_mach, LAPACK's default for pivoted Cholesky) drops
    // parts of G_B that still carry tensor components at the 1e-9 level
    double fr = 2.220446049250313e-16;
    const int* nnull = nullptr;
    int nsm = nsmall;
    void* args[] = {&nn, &Gp, &ldgl, &W, &Wc, &dwork, &ctrl, &status_dev, &fr, &nnull, &nsm};
    note_launch();
    TT_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)pchol_kernel, dim3(blocks), dim3(JT), args,
                                            smem, s));
    note_launch();
    pchol_finish_kernel<<<1, 1, 0, s>>>(w.d_ctrl, kB_dev, nullptr, nsmall);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status eig_reserve(EigWork& w, cudaStream_t s) { return ensure_ctrl(w, s); }

tt_status eig_prepare() {
    TT_TRY(ensure_max_dynamic_smem((const void*)pchol_kernel));
    TT_TRY(ensure_max_dynamic_smem((const void*)jacobi_kernel));
    // cluster attributes set before any capture
    cluster_size_for((const void*)pchol_cluster_kernel, 256);
    cluster_size_for((const void*)osj_kernel<8, true>, 32 * OSJ_MAX_WARPS);
    return TT_OK;
}

tt_status pchol_dyn(cudaStream_t s, const int* n_dev, int ncap, const double* G, double* W, double* Wc,
                    double* dwork, EigWork& w, int* status_dev, int* kB_dev) {
    if (ncap <= 0) return TT_OK;
    TT_TRY(ensure_ctrl(w, s));
    const int nsmall = pchol_small_limit();
    TT_TRY(launch_pchol_cluster(s, std::min(ncap, nsmall), G, ncap, W, kB_dev, n_dev, nsmall));
    if (ncap > nsmall) {
        const size_t smem = (size_t)ncap * sizeof(double);
        if (smem > 200 * 1024) {
            set_error("pchol: matrix too large");
            return TT_ERR_TOO_LARGE;
        }
        TT_TRY(ensure_max_dynamic_smem((const void*)pchol_kernel));
        int blocks = 1;
        TT_TRY(coop_blocks((const void*)pchol_kernel, smem, std::max(1, (ncap + 7) / 8), &blocks));
        int nn = ncap;
        long ldgl = ncap;
        const double* Gp = G;
        int* ctrl = w.d_ctrl;
        double fr = 2.220446049250313e-16;
        int nsm = nsmall;
        void* args[] = {&nn, &Gp, &ldgl, &W, &Wc, &dwork, &ctrl, &status_dev, &fr, &n_dev, &nsm};
        note_launch();
        TT_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)pchol_kernel, dim3(blocks), dim3(JT), args, smem, s));
        note_launch();
        pchol_finish_kernel<<<1, 1, 0, s>>>(w.d_ctrl, kB_dev, n_dev, nsmall);
        TT_CUDA_TRY(cudaGetLastError());
    }
    return TT_OK;
}

tt_status syev_dyn(cudaStream_t s, const int* n_dev, int ncap, const double* G, double* lam, double* Vt,
                   EigWork& w, int* status_dev, int* sweeps_dev, int max_sweeps) {
    if (ncap <= 0) return TT_OK;
    double tol_rel = 1e-15, tol_abs_rel = 1e-20;
    const int Ncap = ncap + (ncap & 1);
    const int npcap = Ncap / 2;
    TT_TRY(w.g0.ensure((size_t)ncap * ncap, s));
    TT_TRY(w.g1.ensure((size_t)ncap * ncap, s));
    TT_TRY(w.vt_unsorted.ensure((size_t)ncap * ncap, s));
    TT_TRY(w.lam_unsorted.ensure((size_t)ncap, s));
    TT_TRY(w.abc.ensure((size_t)6 * npcap, s));
    TT_TRY(w.cs.ensure((size_t)2 * npcap, s));
    TT_TRY(ensure_ctrl(w, s));
    // grid and shared memory for the largest n; a smaller n leaves CTAs with
    // fewer (or no) pairs, and every pair's arithmetic is the same as in syev
    auto smem_for = [&](int ppc) {
        return (size_t)(npcap * 2 + 2 * (size_t)ppc * ncap) * sizeof(double) + (size_t)npcap * sizeof(int);
    };
    size_t smem = smem_for(MAX_PAIRS_PER_CTA);
    if (smem > 200 * 1024) smem = smem_for(1);
    if (smem > 200 * 1024) {
        set_error("syev: matrix too large for the shared-memory row buffers");
        return TT_ERR_TOO_LARGE;
    }
    TT_TRY(ensure_max_dynamic_smem((const void*)jacobi_kernel));
    int blocks = 1;
    TT_TRY(coop_blocks((const void*)jacobi_kernel, smem, npcap, &blocks));
    const int ppc = (npcap + blocks - 1) / blocks;
    if (ppc > MAX_PAIRS_PER_CTA || smem_for(ppc) > smem) {
        set_error("syev: too few resident CTAs for this matrix size");
        return TT_ERR_TOO_LARGE;
    }
    {
        const long total = (long)ncap * ncap;
        const int ib = (int)std::min<long>((total + 255) / 256, 152L * 16);
        note_launch();
        jacobi_init_kernel<<<ib, 256, 0, s>>>(ncap, Ncap, G, ncap, w.g0.p, w.vt_unsorted.p, ncap, w.abc.p, n_dev);
        TT_CUDA_TRY(cudaGetLastError());
    }
    double* g0 = w.g0.p;
    double* g1 = w.g1.p;
    double* vt = w.vt_unsorted.p;
    double* abc0 = w.abc.p;
    double* abc1 = w.abc.p + 3 * npcap;
    double* csg = w.cs.p;
    double* lamu = w.lam_unsorted.p;
    int* ctrl = w.d_ctrl;
    int nn = ncap, NN = Ncap;
    long ldl = ncap;
    int msw = max_sweeps;
    void* args[] = {&nn, &NN, &g0, &g1, &ldl, &vt, &abc0, &abc1, &csg, &lamu, &ctrl, &status_dev, &tol_rel,
                    &tol_abs_rel, &msw, &n_dev};
    note_launch();
    TT_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(blocks), dim3(JT), args, smem, s));
    note_launch();
    jacobi_sort_kernel<<<ncap, 256, 0, s>>>(ncap, w.lam_unsorted.p, ncap, w.vt_unsorted.p, lam, Vt, ncap,
                                            sweeps_dev, w.d_ctrl, n_dev);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

void truncation_decision_dyn(cudaStream_t s, const double* lamK, const int* kB_dev, double eps, int dm1,
                             int forced, int max_rank, double* delta2_dev, int* dec_i, double* dec_d) {
    note_launch();
    truncation_kernel<<<1, 1, 0, s>>>(lamK, 0, eps, dm1, forced, max_rank, delta2_dev, dec_i, dec_d, kB_dev, 0);
}

void truncation_decision(cudaStream_t s, const double* lamK, int kB, double eps, int dm1,
                         int forced, int max_rank, double* delta2_dev, int* dec_i,
                         double* dec_d, bool singular_values) {
    note_launch();
    truncation_kernel<<<1, 1, 0, s>>>(lamK, kB, eps, dm1, forced, max_rank, delta2_dev, dec_i,
                                      dec_d, nullptr, singular_values ? 1 : 0);
}

tt_status syev_psd(cudaStream_t s, int n, const double* K, long ldk, double* lam, double* Vt, long ldv,
                   EigWork& w, int* status_dev, int* sweeps_dev, int max_sweeps) {
    if (n < 0) {
        set_error("syev_psd: negative size");
        return TT_ERR_ARG;
    }
    if (max_sweeps < 1 || max_sweeps > MAX_SWEEPS) {
        set_error("syev_psd: the sweep limit must be in 1 .. " + std::to_string(MAX_SWEEPS));
        return TT_ERR_ARG;
    }
    if (n == 0) return TT_OK;
    if (n == 1) {
        note_launch();
        trivial_eig_kernel<<<1, 1, 0, s>>>(K, lam, Vt, sweeps_dev);
        TT_CUDA_TRY(cudaGetLastError());
        return TT_OK;
    }
    TT_TRY(w.g0.ensure((size_t)n * n, s));
    TT_TRY(w.g1.ensure((size_t)n * n, s));
    TT_TRY(w.vt_unsorted.ensure((size_t)n * n, s));
    TT_TRY(w.lam_unsorted.ensure((size_t)n, s));
    TT_TRY(w.psd.ensure((size_t)3 * n + 2, s));
    int* k_dev = reinterpret_cast<int*>(w.psd.p + 3 * n);
    // K = W^T W (pivoted, rows of W in pivot order), then its rows orthogonalised
    TT_TRY(pchol(s, n, K, ldk, w.g0.p, w.g1.p, w.psd.p, w, status_dev, k_dev));
    TT_TRY(osj_launch(s, n, k_dev, w, status_dev, max_sweeps, nullptr, w.psd.p + 2 * n));
    note_launch();
    jacobi_sort_kernel<<<n, 256, 0, s>>>(n, w.lam_unsorted.p, n, w.vt_unsorted.p, lam, Vt, ldv, sweeps_dev,
                                         w.d_ctrl, nullptr);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status syev_psd_dyn(cudaStream_t s, const int* n_dev, int ncap, const double* K, double* lam, double* Vt,
                       EigWork& w, int* status_dev, int* sweeps_dev, int max_sweeps) {
    if (ncap <= 0) return TT_OK;
    TT_TRY(w.g0.ensure((size_t)ncap * ncap, s));
    TT_TRY(w.g1.ensure((size_t)ncap * ncap, s));
    TT_TRY(w.vt_unsorted.ensure((size_t)ncap * ncap, s));
    TT_TRY(w.lam_unsorted.ensure((size_t)ncap, s));
    TT_TRY(w.psd.ensure((size_t)3 * ncap + 2, s));
    int* k_dev = reinterpret_cast<int*>(w.psd.p + 3 * ncap);
    TT_TRY(pchol_dyn(s, n_dev, ncap, K, w.g0.p, w.g1.p, w.psd.p, w, status_dev, k_dev));
    TT_TRY(osj_launch(s, ncap, k_dev, w, status_dev, max_sweeps, n_dev, w.psd.p + 2 * ncap));
    note_launch();
    jacobi_sort_kernel<<<ncap, 256, 0, s>>>(ncap, w.lam_unsorted.p, ncap, w.vt_unsorted.p, lam, Vt, ncap,
                                            sweeps_dev, w.d_ctrl, n_dev);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

void count_above_floor(cudaStream_t s, const double* lam, int n, int* out_dev) {
    note_launch();
    count_floor_kernel<<<1, 1, 0, s>>>(lam, n, out_dev);
}

}  // namespace ttsn
