// Transport, source and quadrature kernels of the TT-S_N step (arXiv
// 2503.18056, Sec. 3-4) on the paper's three-core layout (Eq. tensor_decomp):
// I_ilp = X_i Theta_l Phi_p, all spatial axes grouped in X (N_c x r1).
//
// Transport (Sec. 4.3): the upwind update of Eq. lhs / Eq. upwind is the TT sum
//   I* = I - sum_a nu_a [ (D^-_a X) (x) (thfac Theta) (x) (phfac Phi)
//                       + (D^+_a X) (x) (thfac' Theta) (x) (phfac' Phi) ],
// nu_a = c dt / dx_a, D^-_a X_i = X_i - X_{i-1}, D^+_a X_i = X_{i+1} - X_i with
// ghost rows per Sec. 4.5 (zero rows for vacuum, wrapped rows for periodic)
// and rank-one masked direction cosines (sin(theta), max/min(cos(phi), 0)) for
// x, (sin(theta), max/min(sin(phi), 0)) for y, (max/min(cos(theta), 0), 1) for
// z.  Terms are summed by TT addition (Sec. 4.1) in the order
// [I, x+, x-, y+, y-, z+, z-]: the spatial core is the concatenation of the
// term cores, the angular cores are block-diagonal / stacked.
//
// Source (Sec. 3.2, 4.4): per cell k_a = c dt sigma_a, k_s = c dt sigma_s,
// E* = X*_i . thbar / c (Eq. tt_energy_density), T-dagger from
// gamma a_r T^4 + T = T^m + gamma E*, gamma = k_a / ((1 + k_a) C_v), then
// I^{m+1} = s I* + e (x) 1 (x) 1 with s = 1/(1 + k_a + k_s) and
// e = s (k_s J^{m+1} + k_a c a_r T-dagger^4 / 4 pi),
// J^{m+1} = (c E*/4 pi + k_a c a_r T-dagger^4 / 4 pi)/(1 + k_a): a row scaling
// of the spatial core plus one appended column (angular cores get a unit
// block), fused into the same pass as transport so the grown spatial core is
// written once.
#include <algorithm>

#include "internal.h"

namespace ttsn {

namespace {

constexpr double FOUR_PI = 12.566370614359172953850573533118;

struct TermFactors {
    // thfac/phfac for term j at ordinate (l) / (p)
    __device__ static double th(int j, int l, const double* mu, const double* sint) {
        if (j == 0) return 1.0;
        const int axis = (j - 1) >> 1;
        const bool plus = ((j - 1) & 1) == 0;
        if (axis < 2) return sint[l];
        return plus ? fmax(mu[l], 0.0) : fmin(mu[l], 0.0);
    }
    __device__ static double ph(int j, int p, const double* cphi, const double* sphi) {
        if (j == 0) return 1.0;
        const int axis = (j - 1) >> 1;
        const bool plus = ((j - 1) & 1) == 0;
        if (axis == 0) return plus ? fmax(cphi[p], 0.0) : fmin(cphi[p], 0.0);
        if (axis == 1) return plus ? fmax(sphi[p], 0.0) : fmin(sphi[p], 0.0);
        return 1.0;
    }
};

// Thg: (R1, nt, R2) with R1 >= nterms r1 (+1 if src), R2 >= nterms r2 (+1 if src)
__global__ void grown_theta_kernel(int nterms, int src, int r1, int r2, int nt, const double* Th,
                                   const double* mu, const double* sint, double* Thg, int R1,
                                   int R2) {
    const long total = (long)R1 * nt * R2;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int b = (int)(t % R2);
        const long t2 = t / R2;
        const int l = (int)(t2 % nt);
        const int a = (int)(t2 / nt);
        double v = 0.0;
        const int ja = a / r1, jb = b / r2;
        if (ja == jb && ja < nterms) {
            v = TermFactors::th(ja, l, mu, sint) *
                Th[((long)(a - ja * r1) * nt + l) * r2 + (b - jb * r2)];
        } else if (src && a == R1 - 1 && b == R2 - 1) {
            v = 1.0;
        }
        Thg[t] = v;
    }
}

// Phg: (R2, np)
__global__ void grown_phi_kernel(int nterms, int src, int r2, int np, const double* Ph,
                                 const double* cphi, const double* sphi, double* Phg, int R2) {
    const long total = (long)R2 * np;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int p = (int)(t % np);
        const int b = (int)(t / np);
        double v = 0.0;
        const int jb = b / r2;
        if (jb < nterms) {
            v = TermFactors::ph(jb, p, cphi, sphi) * Ph[(long)(b - jb * r2) * np + p];
        } else if (src && b == R2 - 1) {
            v = 1.0;
        }
        Phg[t] = v;
    }
}

// phibar[j][b] = sum_p v phfac_j[p] Ph[b][p]
__global__ void phibar_kernel(int nterms, int r2, int np, const double* Ph, const double* cphi,
                              const double* sphi, double v, double* phibar) {
    const int total = nterms * r2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int j = t / r2, b = t % r2;
        double acc = 0.0;
        for (int p = 0; p < np; ++p) acc += TermFactors::ph(j, p, cphi, sphi) * Ph[(long)b * np + p];
        phibar[t] = v * acc;
    }
}

// thbar[j r1 + a] = sum_l w thfac_j[l] sum_b Th[a][l][b] phibar[j][b]
__global__ void thbar_kernel(int nterms, int r1, int r2, int nt, const double* Th,
                             const double* mu, const double* sint, double w, const double* phibar,
                             double* thbar) {
    const int total = nterms * r1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int j = t / r1, a = t % r1;
        double acc = 0.0;
        for (int l = 0; l < nt; ++l) {
            double inner = 0.0;
            const double* row = Th + ((long)a * nt + l) * r2;
            for (int b = 0; b < r2; ++b) inner += row[b] * phibar[j * r2 + b];
            acc += TermFactors::th(j, l, mu, sint) * inner;
        }
        thbar[t] = w * acc;
    }
}

// Quartic of Sec. 3.2 on the increasing branch T >= T_b = -(4 gamma a_r)^(-1/3):
// gamma a_r T^4 + T = rhs.  Newton from the upper bracket end; f is convex and
// increasing there, so the iterates decrease monotonically onto the root.
__device__ double t_dagger(double Tm, double Estar, double ka, double Cv, double a_r) {
    const double gamma = ka / ((1.0 + ka) * Cv);
    const double rhs = Tm + gamma * Estar;
    const double ga = gamma * a_r;
    if (ga == 0.0) return rhs;
    double T;
    if (rhs >= 0.0) {
        T = fmin(rhs, sqrt(sqrt(rhs / ga)));
    } else {
        const double Tb = -cbrt(1.0 / (4.0 * ga));
        if (rhs < 0.75 * Tb) return Tb;
        T = rhs;
    }
    for (int it = 0; it < 200; ++it) {
        const double T3 = T * T * T;
        const double f = ga * T3 * T + T - rhs;
        const double fp = 4.0 * ga * T3 + 1.0;
        const double Tn = T - f / fp;
        if (Tn == T) break;
        if (it > 0 && Tn > T) break;  // rounding floor reached (iterates stopped decreasing)
        T = Tn;
    }
    return T;
}

// One warp per cell.  Pass 1 computes the transport block values for the
// quadrature dot product (E*), the source scalars follow, pass 2 recomputes and
// writes the scaled values.
__global__ void __launch_bounds__(256)
transport_source_kernel(Grid g, Fields f, int transport, int source, int r1,
                        const double* __restrict__ X, long ldx, const double* __restrict__ thbar,
                        double* __restrict__ Xg, long ldg) {
    const int lane = threadIdx.x & 31;
    const long warps = (long)gridDim.x * (blockDim.x >> 5);
    const int nterms = transport ? 1 + 2 * g.ndim : 1;
    for (long i = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < g.nc; i += warps) {
        // cell coordinates (C order, axis 0 slowest) and neighbour rows (-1 = zero ghost)
        long nb[3][2];
        long rem = i, stride = 1;
        int coord[3] = {0, 0, 0};
        for (int a = g.ndim - 1; a >= 0; --a) {
            coord[a] = (int)(rem % g.n[a]);
            rem /= g.n[a];
        }
        for (int a = g.ndim - 1; a >= 0; --a) {
            const int ca = coord[a];
            const int na = g.n[a];
            long lo, hi;
            if (g.bc[a] == TT_BC_PERIODIC) {
                lo = i + (long)((ca == 0) ? (na - 1) : -1) * stride;
                hi = i + (long)((ca == na - 1) ? -(na - 1) : 1) * stride;
            } else {
                lo = (ca == 0) ? -1 : i - stride;
                hi = (ca == na - 1) ? -1 : i + stride;
            }
            nb[a][0] = lo;
            nb[a][1] = hi;
            stride *= na;
        }
        double nu[3];
        for (int a = 0; a < g.ndim; ++a) nu[a] = f.c * f.dt / g.dx[a];

        double scale = 1.0, emit = 0.0;
        if (source) {
            double dot = 0.0;
            for (int col = lane; col < r1; col += 32) {
                const double x0 = X[i * ldx + col];
                dot += x0 * thbar[col];
                if (transport) {
                    for (int a = 0; a < g.ndim; ++a) {
                        const double xm = nb[a][0] >= 0 ? X[nb[a][0] * ldx + col] : 0.0;
                        const double xp = nb[a][1] >= 0 ? X[nb[a][1] * ldx + col] : 0.0;
                        dot += -nu[a] * (x0 - xm) * thbar[(1 + 2 * a) * r1 + col];
                        dot += -nu[a] * (xp - x0) * thbar[(2 + 2 * a) * r1 + col];
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
            const double Estar = dot / f.c;
            const double ka = f.c * f.dt * f.sigma_a[i];
            const double ks = f.sigma_s ? f.c * f.dt * f.sigma_s[i] : 0.0;
            const double Td = t_dagger(f.T[i], Estar, ka, f.cv[i], f.a_r);
            const double Td2 = Td * Td;
            const double B = f.c * f.a_r * Td2 * Td2 / FOUR_PI;
            const double Jnew = (f.c * Estar / FOUR_PI + ka * B) / (1.0 + ka);
            scale = 1.0 / (1.0 + ka + ks);
            emit = scale * (ks * Jnew + ka * B);
            if (lane == 0) f.E_star[i] = Estar;
        }
        double* out = Xg + i * ldg;
        for (int col = lane; col < r1; col += 32) {
            const double x0 = X[i * ldx + col];
            out[col] = scale * x0;
            if (transport) {
                for (int a = 0; a < g.ndim; ++a) {
                    const double xm = nb[a][0] >= 0 ? X[nb[a][0] * ldx + col] : 0.0;
                    const double xp = nb[a][1] >= 0 ? X[nb[a][1] * ldx + col] : 0.0;
                    out[(1 + 2 * a) * r1 + col] = scale * (-nu[a] * (x0 - xm));
                    out[(2 + 2 * a) * r1 + col] = scale * (-nu[a] * (xp - x0));
                }
            }
        }
        if (source && lane == 0) out[nterms * r1] = emit;
    }
}

__global__ void __launch_bounds__(256)
energy_rows_kernel(long nc, int r, const double* __restrict__ X, long ldx,
                   const double* __restrict__ thbar, double c, double* E_out,
                   const double* __restrict__ E_star, const double* __restrict__ cv, double* T,
                   int update_T) {
    const int lane = threadIdx.x & 31;
    const long warps = (long)gridDim.x * (blockDim.x >> 5);
    for (long i = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < nc; i += warps) {
        double dot = 0.0;
        for (int col = lane; col < r; col += 32) dot += X[i * ldx + col] * thbar[col];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) {
            const double E = dot / c;
            if (E_out) E_out[i] = E;
            if (update_T) T[i] = T[i] + (E_star[i] - E) / cv[i];
        }
    }
}

__global__ void init_iso_kernel(long nc, const double* Tr, double c, double a_r, double* X) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nc;
         i += (long)gridDim.x * blockDim.x) {
        const double t2 = Tr[i] * Tr[i];
        X[i] = c * a_r * t2 * t2 / FOUR_PI;
    }
}

constexpr int RED_BLOCKS = 1024;

__global__ void totals_partial_kernel(long nc, const double* E, const double* cv, const double* T,
                                      double* part) {
    __shared__ double s0[256], s1[256];
    double a = 0.0, b = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nc;
         i += (long)gridDim.x * blockDim.x) {
        a += E[i];
        b += cv[i] * T[i];
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s0[threadIdx.x] += s0[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s0[0];
        part[RED_BLOCKS + blockIdx.x] = s1[0];
    }
}

__global__ void totals_final_kernel(const double* part, double* totals) {
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < RED_BLOCKS; ++k) {
            a += part[k];
            b += part[RED_BLOCKS + k];
        }
        totals[0] = a;
        totals[1] = b;
    }
}

inline int blocks_for(long total, int threads = 256) {
    long b = (total + threads - 1) / threads;
    return (int)std::max<long>(1, std::min<long>(b, 152L * 32));
}

}  // namespace

void build_grown_angular(cudaStream_t s, const Angular& ang, int ndim, bool transport,
                         bool source, int r1, int r2, const double* Th, const double* Ph,
                         double* Thg, double* Phg, int R1, int R2) {
    const int nterms = transport ? 1 + 2 * ndim : 1;
    note_launch();
    grown_theta_kernel<<<blocks_for((long)R1 * ang.n_theta * R2), 256, 0, s>>>(
        nterms, source ? 1 : 0, r1, r2, ang.n_theta, Th, ang.mu, ang.sint, Thg, R1, R2);
    note_launch();
    grown_phi_kernel<<<blocks_for((long)R2 * ang.n_phi), 256, 0, s>>>(
        nterms, source ? 1 : 0, r2, ang.n_phi, Ph, ang.cphi, ang.sphi, Phg, R2);
}

// phibar scratch: thbar + nterms*r1 (caller allocates (nterms*(r1+r2)) doubles at thbar)
void grown_thbar(cudaStream_t s, const Angular& ang, int ndim, bool transport, int r1, int r2,
                 const double* Th, const double* Ph, double* thbar) {
    const int nterms = transport ? 1 + 2 * ndim : 1;
    double* phibar = thbar + nterms * r1;
    note_launch();
    phibar_kernel<<<blocks_for((long)nterms * r2), 256, 0, s>>>(nterms, r2, ang.n_phi, Ph,
                                                               ang.cphi, ang.sphi, ang.v, phibar);
    note_launch();
    thbar_kernel<<<blocks_for((long)nterms * r1, 64), 64, 0, s>>>(
        nterms, r1, r2, ang.n_theta, Th, ang.mu, ang.sint, ang.w, phibar, thbar);
}

void plain_thbar(cudaStream_t s, const Angular& ang, int r1, int r2, const double* Th,
                 const double* Ph, double* thbar) {
    grown_thbar(s, ang, 0, false, r1, r2, Th, Ph, thbar);
}

void transport_source_rows(cudaStream_t s, const Grid& g, const Fields& f, bool transport,
                           bool source, int r1, const double* X, long ldx, const double* thbar,
                           double* Xg, long ldg) {
    const long warps_needed = g.nc;
    const int blocks = (int)std::max<long>(1, std::min<long>((warps_needed + 7) / 8, 152L * 64));
    note_launch();
    transport_source_kernel<<<blocks, 256, 0, s>>>(g, f, transport ? 1 : 0, source ? 1 : 0, r1, X,
                                                   ldx, thbar, Xg, ldg);
}

void energy_rows(cudaStream_t s, long nc, int r, const double* X, long ldx, const double* thbar,
                 double c, double* E_out, const double* E_star, const double* cv, double* T,
                 bool update_T) {
    const int blocks = (int)std::max<long>(1, std::min<long>((nc + 7) / 8, 152L * 64));
    note_launch();
    energy_rows_kernel<<<blocks, 256, 0, s>>>(nc, r, X, ldx, thbar, c, E_out, E_star, cv, T,
                                              update_T ? 1 : 0);
}

void init_isotropic(cudaStream_t s, long nc, const double* Tr, double c, double a_r, double* X) {
    note_launch();
    init_iso_kernel<<<blocks_for(nc), 256, 0, s>>>(nc, Tr, c, a_r, X);
}

void energy_totals(cudaStream_t s, long nc, const double* E, const double* cv, const double* T,
                   double* totals_dev, double* scratch) {
    note_launch();
    totals_partial_kernel<<<RED_BLOCKS, 256, 0, s>>>(nc, E, cv, T, scratch);
    note_launch();
    totals_final_kernel<<<1, 32, 0, s>>>(scratch, totals_dev);
}

}  // namespace ttsn
