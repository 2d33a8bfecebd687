// Split-space layout: one TT core per spatial axis, then theta and phi
// (the alternative to the grouped spatial core that Sec. 4.1 and Sec. 7
// discuss).  This file builds the cores of the grown TT of a step:
//
//   transport (Sec. 4.3): the TT sum of the 1 + 2 ndim terms
//   I - sum_a nu_a [D^-_a I (.) n_a^+ + D^+_a I (.) n_a^-] by the addition of
//   Sec. 4.1 -- the first core concatenates the terms' cores, middle cores are
//   block diagonal, the last core stacks them.  Term (a, +/-) applies D^-/+
//   along the mode of spatial core a (ghost slices of Sec. 4.5: zero for
//   vacuum, wrapped for periodic; other fluxes: the face-weighted stencil
//   of the flux, uniform here since the layout takes uniform opacities); the
//   theta core carries -nu_a times the term's theta factor and the phi core
//   the term's phi factor;
//   emission (Sec. 3.2, 4.4): e (x) 1 (x) 1 with e a spatial field, appended as
//   one more TT term whose spatial cores hold e exactly: 1D a column e;
//   2D [I_{N_x}] [e as N_x x N_y x 1]; 3D [I_{N_x}] [e as N_x x N_y x N_z]
//   [I_{N_z}]; then unit angular cores.  The absorption factor s (uniform in
//   this layout) scales the transport blocks of the phi core.
//
// Every element of a grown core is written once (zeros included), one thread
// per element with the last rank index fastest, so reads of the input core
// and writes are coalesced; the kernel is bound by the write of the grown core.
#include <algorithm>

#include "internal.h"

namespace ttsn {

namespace {

__device__ __forceinline__ double split_term_value(const SplitCoreSpec& c, const double* __restrict__ G,
                                                   const double* __restrict__ fac, int j, int a, int i,
                                                   int b) {
    const long row = (long)a * c.n;
    const double g = G[(row + i) * c.rb + b];
    if (c.kind == SPLIT_SPATIAL) {
        if (j == 0) return g;
        const int axis = (j - 1) >> 1;
        if (axis != c.axis) return g;
        // term (axis, t): c0 I_i + cp I_{i+1} - cm I_{i-1} (upwinding: I_i - I_{i-1}
        // and I_{i+1} - I_i), ghost slices zero (vacuum), wrapped (periodic) or
        // a copy of the boundary slice (outflow)
        const int t = (j - 1) & 1;
        double gm = 0.0, gp = 0.0;
        if (i > 0)
            gm = G[(row + i - 1) * c.rb + b];
        else if (c.bc == TT_BC_PERIODIC)
            gm = G[(row + c.n - 1) * c.rb + b];
        else if (c.bc == TT_BC_OUTFLOW)
            gm = g;
        if (i + 1 < c.n)
            gp = G[(row + i + 1) * c.rb + b];
        else if (c.bc == TT_BC_PERIODIC)
            gp = G[row * c.rb + b];
        else if (c.bc == TT_BC_OUTFLOW)
            gp = g;
        return c.co[t][0] * g + c.co[t][1] * gp - c.co[t][2] * gm;
    }
    return fac[(long)j * c.n + i] * g * c.tscale;
}

__global__ void __launch_bounds__(256)
split_grow_kernel(SplitCoreSpec c, const double* __restrict__ G, const double* __restrict__ fac,
                  double* __restrict__ out) {
    const long total = (long)c.Ra * c.n * c.Rb;
    const int Ta = c.K * c.ra, Tb = c.K * c.rb;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
         t += (long)gridDim.x * blockDim.x) {
        const int bo = (int)(t % c.Rb);
        const long q = t / c.Rb;
        const int i = (int)(q % c.n);
        const int ao = (int)(q / c.n);
        const bool t_row = c.first || ao < Ta, t_col = c.last || bo < Tb;
        const bool e_row = c.first || ao >= Ta, e_col = c.last || bo >= Tb;
        double v = 0.0;
        if (t_row && t_col && c.K > 0) {
            int j, a, b;
            if (c.first) {
                j = bo / c.rb;
                b = bo - j * c.rb;
                a = 0;
            } else if (c.last) {
                j = ao / c.ra;
                a = ao - j * c.ra;
                b = 0;
            } else {
                j = ao / c.ra;
                a = ao - j * c.ra;
                const int j2 = bo / c.rb;
                b = bo - j2 * c.rb;
                if (j2 != j) j = -1;
            }
            if (j >= 0) v = split_term_value(c, G, fac, j, a, i, b);
        } else if (e_row && e_col && c.ekind != SPLIT_E_NONE) {
            const int ae = c.first ? 0 : ao - Ta, be = c.last ? 0 : bo - Tb;
            switch (c.ekind) {
                case SPLIT_E_IDENT_COL: v = (i == be) ? 1.0 : 0.0; break;
                case SPLIT_E_IDENT_ROW: v = (ae == i) ? 1.0 : 0.0; break;
                case SPLIT_E_ONES: v = 1.0; break;
                default: v = 0.0; break;  // SPLIT_E_FIELD: written by the source kernel
            }
        }
        out[t] = v;
    }
}

}  // namespace

void split_grow_core(cudaStream_t s, const SplitCoreSpec& c, const double* G, const double* fac,
                     double* out) {
    const long total = (long)c.Ra * c.n * c.Rb;
    if (total <= 0) return;
    const int blocks = (int)std::max<long>(1, std::min<long>((total + 255) / 256, 152L * 16));
    note_launch();
    split_grow_kernel<<<blocks, 256, 0, s>>>(c, G, fac, out);
}

}  // namespace ttsn
