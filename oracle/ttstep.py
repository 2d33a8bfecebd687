"""Step-then-truncate TT-S_N stepper (oracle; test infrastructure).

Layout: the paper's three cores (Eq. tensor_decomp), I_ilp = X_i Theta_l Phi_p,
with all spatial axes grouped into the first core (cell index in C order of
the (N_x[, N_y[, N_z]]) grid, x slowest).  One time step:

1. transport (Sec. 4.3): the upwind update of Eq. lhs / Eq. upwind written as
   a TT sum I - sum_a nu_a [D^-_a I (.) n_a^+ + D^+_a I (.) n_a^-], nu_a =
   c dt / dx_a, where D^-_a X_i = X_i - X_{i-1} and D^+_a X_i = X_{i+1} - X_i act
   on the spatial core with ghost rows (Sec. 4.5: zero rows for vacuum, copied
   rows for periodic) and the masked direction cosines are rank one:
   n_x^+- = sin(theta) * max/min(cos(phi), 0), n_y^+- = sin(theta) *
   max/min(sin(phi), 0), n_z^+- = max/min(cos(theta), 0) * 1.  Terms are summed
   with the addition of Sec. 4.1 in the order [I, x+, x-, y+, y-, z+, z-];
2. source (Sec. 3.2 and 4.4): E* by TT integration (Eq. tt_energy_density),
   T-dagger from the quartic, then I^{m+1} = s (.) I* + e (x) 1 (x) 1 with
   s = 1/(1 + k_a + k_s) a rank-one Hadamard factor and
   e = s (k_s J^{m+1} + k_a c a_r T-dagger^4 / 4 pi) a rank-one addition;
3. rounding (Sec. 4.2, App. A) to tolerance eps -- once per step after the
   source by default, or after transport and again after the source
   (``rounds_per_step=2``, the schedule Sec. 4.2 describes);
4. temperature: C_v (T^{m+1} - T^m) = E* - E^{m+1}, E^{m+1} integrated from the
   rounded TT, so that sum(E + C_v T) is conserved through the source stage
   and the rounding.

Fixed external sources S = sum_k x_k (x) theta_k (x) phi_k (optional) enter
the transport stage explicitly, I* = L I + c dt S: each is one more rank-one
term of the TT sum, after the streaming terms.

Interface fluxes (Sec. 3.1, Sec. 4.3): with piecewise-constant states every
flux of the paper is, per axis a and face, c times a sum of two rank-one
angular factors each multiplying a two-point combination w_L U_L + w_R U_R of
the face's states, so the transport stage stays a TT sum of 1 + 2 ndim terms:
term (a, 1) has angular factor g1 and face weights (w_L1, w_R1), term (a, 2)
g2 and (w_L2, w_R2), and its spatial core is
-nu_a [w_L(i+1/2) X_i + w_R(i+1/2) X_{i+1} - w_L(i-1/2) X_{i-1} - w_R(i-1/2) X_i]:
* upwind (Eq. upwind): g = (n_a^+, n_a^-), w = (1, 0) and (0, 1);
* Rusanov (Eq. rusanov_flux_toro, S+ = s c): g = (n_a, 1), w = (1/2, 1/2) and
  (s/2, -s/2);
* HLL (Eq. hll with Sec. 3.1's wave speeds): for n_a >= 0, S_R = c n_a A(tau),
  S_L = -c n_a B(tau), and mirrored for n_a < 0, so g = (n_a^+, n_a^-) and
  w = (A (1 + B), B (1 - A)) / (A + B) and (B (1 - A), A (1 + B)) / (A + B),
  with A = sqrt((1 - exp(-tau^2)) / tau^2) or sqrt(1 - tau^2 / 2) and
  B = sqrt((1 - exp(-tau^4)) / tau^2) or tau (tau >= or < tau_threshold),
  tau the face optical depth of Eq. tauc (ghost opacity: wrapped cell for
  periodic axes, the boundary cell for vacuum);
* Rusanov with the optical-depth speed S+ = c |n_a| min(1, 1/tau) (Sec. 3.1,
  the thick-limit speed of the expansion after Eq. hll): g = (n_a, |n_a|),
  w = (1/2, 1/2) and (m/2, -m/2) with m = min(1, 1/tau) per face; |n_a| is
  separable (sin(theta) |cos(phi)|, sin(theta) |sin(phi)|, |mu|).
"""
import numpy as np

from . import angles, tt
from .quartic import t_dagger
from .rounding import round_gram, round_randomized, round_ttsvd

PERIODIC = 0
VACUUM = 1
OUTFLOW = 2


class TTSN:
    def __init__(self, n, L, n_theta, n_phi, c, a_r, dt, bc, sigma_a, cv, T0,
                 cores, sigma_s=None, eps=0.0, max_rank=None,
                 rounds_per_step=1, rounding="gram", sources=None, flux="upwind",
                 rusanov_s=1.0, hll_beta=1.0, hll_tau_threshold=1.0, inflow=None, sketch=None):
        self.flux = flux
        # rounding="randomized": Gaussian sketch TT (cores (L_{k-1}, n_k, L_k));
        # a rounding to ranks l_k uses the leading l_{k-1} x n_k x l_k blocks
        self.sketch = sketch
        # inflow faces: the ghost intensity g theta phi of a vacuum face enters
        # the boundary cells' stencil as known values, i.e. as rank-one terms
        # -nu (-w_L(lo) g theta phi) on the low face and -nu w_R(hi) g theta phi
        # on the high face, times each term's angular factor
        self.inflow = {k: tuple(np.asarray(v, float) for v in vals) for k, vals in (inflow or {}).items()}
        self.rusanov_s = float(rusanov_s)
        self.hll_beta, self.hll_tau_threshold = float(hll_beta), float(hll_tau_threshold)
        self.ndim = len(n)
        self.n = tuple(n)
        self.nc = int(np.prod(n))
        self.dx = [L[a] / n[a] for a in range(self.ndim)]
        self.c, self.a_r, self.dt = float(c), float(a_r), float(dt)
        self.bc = list(bc)
        self.g = angles.grid(n_theta, n_phi)
        self.sigma_a = np.array(sigma_a, float).reshape(-1)
        self.sigma_s = (np.zeros(self.nc) if sigma_s is None
                        else np.array(sigma_s, float).reshape(-1))
        self.cv = np.array(cv, float).reshape(-1)
        self.T = np.array(T0, float).reshape(-1).copy()
        self.cores = [np.array(G, float) for G in cores]
        self.eps, self.max_rank = eps, max_rank
        self.rounds_per_step = rounds_per_step
        self.rounding = rounding
        self.sources = [(np.asarray(x, float).reshape(-1), np.asarray(th, float),
                         np.asarray(ph, float)) for x, th, ph in (sources or [])]
        self.last_sigmas = []
        self.last_ranks = []

    @staticmethod
    def isotropic_cores(I_field, n_theta, n_phi):
        """Rank-one TT of an isotropic intensity field I(x)."""
        return [np.asarray(I_field, float).reshape(1, -1, 1),
                np.ones((1, n_theta, 1)), np.ones((1, n_phi, 1))]

    # -- spatial difference operators on the grouped core (Sec. 4.5 ghosts)
    def _neighbour(self, X, axis, offset):
        """Row i of the result is X at cell i + offset along ``axis``
        (periodic wrap, a zero ghost row for vacuum, the edge row for outflow)."""
        r = X.shape[-1]
        Y = X.reshape(self.n + (r,))
        if self.bc[axis] == PERIODIC:
            Z = np.roll(Y, -offset, axis=axis)
        elif self.bc[axis] == OUTFLOW:
            idx = np.clip(np.arange(self.n[axis]) + offset, 0, self.n[axis] - 1)
            Z = np.take(Y, idx, axis=axis)
        else:
            Z = np.zeros_like(Y)
            N = self.n[axis]
            src = [slice(None)] * Y.ndim
            dst = [slice(None)] * Y.ndim
            if offset > 0:
                src[axis] = slice(offset, N)
                dst[axis] = slice(0, N - offset)
            else:
                src[axis] = slice(0, N + offset)
                dst[axis] = slice(-offset, N)
            Z[tuple(dst)] = Y[tuple(src)]
        return Z.reshape(X.shape)

    def _masks(self, axis):
        g = self.g
        if axis == 0:
            cphi = np.cos(g["phi"])
            return (g["sin_theta"], np.maximum(cphi, 0.0)), (g["sin_theta"], np.minimum(cphi, 0.0))
        if axis == 1:
            sphi = np.sin(g["phi"])
            return (g["sin_theta"], np.maximum(sphi, 0.0)), (g["sin_theta"], np.minimum(sphi, 0.0))
        one = np.ones_like(g["phi"])
        return (np.maximum(g["mu"], 0.0), one), (np.minimum(g["mu"], 0.0), one)

    def _face_weights(self, a):
        """(w_L1, w_R1, w_L2, w_R2) at the faces below (lo) and above (hi) every
        cell along axis a, each an (N_c,) array: returns ((lo1, hi1), (lo2, hi2))
        with lo/hi = (w_L, w_R)."""
        nc = int(np.prod(self.n))
        if self.flux == "upwind":
            w1, w2 = (1.0, 0.0), (0.0, 1.0)
            const = True
        elif self.flux == "rusanov":
            s = self.rusanov_s
            w1, w2 = (0.5, 0.5), (0.5 * s, -0.5 * s)
            const = True
        else:
            const = False
        if const:
            f = lambda v: np.full(nc, v)
            pair = lambda w: ((f(w[0]), f(w[1])), (f(w[0]), f(w[1])))
            return pair(w1), pair(w2)
        sig = (self.sigma_a + self.sigma_s).reshape(self.n)
        N = self.n[a]

        def shifted(off):
            if self.bc[a] == PERIODIC:
                return np.roll(sig, -off, axis=a)
            idx = np.clip(np.arange(N) + off, 0, N - 1)
            return np.take(sig, idx, axis=a)

        def tau_with(other):
            t = np.zeros_like(sig)
            ok = (sig > 0.0) & (other > 0.0)
            t[ok] = 2.0 * self.hll_beta * self.dx[a] / (1.0 / sig[ok] + 1.0 / other[ok])
            return t

        def AB(t):
            thr = self.hll_tau_threshold
            big = t >= thr
            tt = np.where(t > 0.0, t, 1.0)
            A = np.where(big, np.sqrt((1.0 - np.exp(-t ** 2)) / tt ** 2), np.sqrt(np.maximum(1.0 - t ** 2 / 2.0, 0.0)))
            B = np.where(big, np.sqrt((1.0 - np.exp(-t ** 4)) / tt ** 2), t)
            return A, B

        out = []
        if self.flux == "rusanov_tau":
            for t in (tau_with(shifted(-1)), tau_with(shifted(+1))):  # lo face, hi face
                t = t.reshape(-1)
                m = np.where(t > 1.0, 1.0 / np.where(t > 1.0, t, 1.0), 1.0)
                out.append(((np.full(nc, 0.5), np.full(nc, 0.5)), (0.5 * m, -0.5 * m)))
            (lo1, lo2), (hi1, hi2) = out
            return (lo1, hi1), (lo2, hi2)
        for t in (tau_with(shifted(-1)), tau_with(shifted(+1))):  # lo face, hi face
            A, B = AB(t.reshape(-1))
            out.append(((A * (1.0 + B) / (A + B), B * (1.0 - A) / (A + B)),
                        (B * (1.0 - A) / (A + B), A * (1.0 + B) / (A + B))))
        (lo1, lo2), (hi1, hi2) = out
        return (lo1, hi1), (lo2, hi2)

    def _angular(self, a):
        """Angular factors (theta, phi) of the two terms of axis a."""
        if self.flux not in ("rusanov", "rusanov_tau"):
            return self._masks(a)
        g = self.g
        one_t, one_p = np.ones_like(g["mu"]), np.ones_like(g["phi"])
        if a == 0:
            n1 = (g["sin_theta"], np.cos(g["phi"]))
        elif a == 1:
            n1 = (g["sin_theta"], np.sin(g["phi"]))
        else:
            n1 = (g["mu"], one_p)
        if self.flux == "rusanov":
            return n1, (one_t, one_p)
        return n1, (np.abs(n1[0]), np.abs(n1[1]))

    def transport(self, cores):
        X, Th, Ph = cores
        Xm = X[0]
        terms = [cores]
        for a in range(self.ndim):
            nu = self.c * self.dt / self.dx[a]
            Xlo = self._neighbour(Xm, a, -1)
            Xhi = self._neighbour(Xm, a, +1)
            for (lo, hi), (tf, pf) in zip(self._face_weights(a), self._angular(a)):
                (wLlo, wRlo), (wLhi, wRhi) = lo, hi
                D = ((wLhi - wRlo)[:, None] * Xm + wRhi[:, None] * Xhi - wLlo[:, None] * Xlo)
                terms.append([(-nu * D)[None], Th * tf[None, :, None], Ph * pf[None, :, None]])
        for x, th, ph in self.sources:
            terms.append(tt.rank_one([self.c * self.dt * x, th, ph]))
        for (a, side), (gf, th_f, ph_f) in sorted(self.inflow.items()):
            if self.bc[a] != VACUUM:
                continue
            nu = self.c * self.dt / self.dx[a]
            coord = np.indices(self.n)[a].reshape(-1)
            on = coord == (0 if side == 0 else self.n[a] - 1)
            g = np.where(on, gf.reshape(-1), 0.0)
            for (lo, hi), (tf, pf) in zip(self._face_weights(a), self._angular(a)):
                w = lo[0] if side == 0 else -hi[1]  # +w_L(i-1/2) or -w_R(i+1/2)
                if np.any(w * g != 0.0):  # upwinding has one such term per face
                    terms.append(tt.rank_one([nu * w * g, tf * th_f, pf * ph_f]))
        return tt.add_many(terms)

    def energy_density(self, cores=None):
        cores = self.cores if cores is None else cores
        return tt.energy_density_grouped(cores, self.g["w"], self.g["v"], self.c)

    def source(self, cores):
        c, a_r, dt = self.c, self.a_r, self.dt
        k_a = c * dt * self.sigma_a
        k_s = c * dt * self.sigma_s
        E_star = self.energy_density(cores)
        Td = t_dagger(self.T, E_star, k_a, self.cv, a_r)
        B = c * a_r * Td ** 4 / (4.0 * np.pi)
        J_new = (c * E_star / (4.0 * np.pi) + k_a * B) / (1.0 + k_a)
        s = 1.0 / (1.0 + k_a + k_s)
        e = s * (k_s * J_new + k_a * B)
        nt, npf = len(self.g["mu"]), len(self.g["phi"])
        ones_t, ones_p = np.ones(nt), np.ones(npf)
        scaled = tt.hadamard(cores, tt.rank_one([s, ones_t, ones_p]))
        return tt.add(scaled, tt.rank_one([e, ones_t, ones_p])), E_star, Td

    def round(self, cores, forced=None):
        if self.rounding is None:
            return cores
        if self.rounding == "randomized":
            R = tt.ranks(cores)
            ls = [min(forced[k] if forced else self.sketch[k].shape[2], R[k]) for k in range(len(R))]
            r = [1] + ls + [1]
            om = [self.sketch[k][: r[k], :, : r[k + 1]] for k in range(len(cores))]
            out = round_randomized(cores, om)
            self.last_sigmas.append([])
            self.last_ranks.append(tt.ranks(out))
            return out
        fn = round_gram if self.rounding == "gram" else round_ttsvd
        out, sig = fn(cores, self.eps, self.max_rank, forced)
        self.last_sigmas.append(sig)
        self.last_ranks.append(tt.ranks(out))
        return out

    def step(self, forced=None, forced2=None, with_source=True):
        """One time step.  ``forced``: ranks for the (last) rounding of the step;
        ``forced2``: ranks for the post-transport rounding when rounding twice."""
        self.last_sigmas = []
        self.last_ranks = []
        cur = self.transport(self.cores)
        if not with_source:
            self.cores = self.round(cur, forced)
            return self.cores
        if self.rounds_per_step == 2:
            cur = self.round(cur, forced2)
        cur, E_star, Td = self.source(cur)
        cur = self.round(cur, forced)
        E_new = self.energy_density(cur)
        self.T = self.T + (E_star - E_new) / self.cv
        self.cores = cur
        self.last_T_dagger = Td
        return self.cores

    def full(self):
        return tt.full(self.cores).reshape(self.n + (self.cores[1].shape[1], self.cores[2].shape[1]))

    def total_energy(self):
        dV = float(np.prod(self.dx))
        return float(np.sum(self.energy_density() + self.cv * self.T) * dV)
