"""Split-space layout of the TT-S_N step (oracle; test infrastructure).

The intensity is a TT with one core per spatial axis followed by the two
angular cores (the alternative to grouping all spatial axes in one core that
Sec. 4.1 and Sec. 7 discuss):

    I[i_1, .., i_ndim, l, p] = G_1[i_1] ... G_ndim[i_ndim] Theta[l] Phi[p],

d = ndim + 2 cores, core k of shape (r_{k-1}, n_k, r_k).  One time step, in
the same order as the grouped stepper of ``ttstep``:

1. transport (Sec. 4.3): the TT sum I - sum_a nu_a [D^-_a I (.) n_a^+ +
   D^+_a I (.) n_a^-] of Sec. 4.1's addition.  Term (a, +/-) is the TT whose
   core for axis a is D^-/+ applied along that core's mode (ghost slices of
   Sec. 4.5: zero for vacuum, wrapped for periodic), scaled by -nu_a; the
   other spatial cores are unchanged and the angular cores carry the masked
   direction cosines (rank one, as in the grouped layout);
2. source (Sec. 3.2, 4.4): E* by TT integration (contract the angular cores
   with the quadrature weights, then the spatial cores), T-dagger from the
   quartic, I^{m+1} = s (.) I* + e (x) 1 (x) 1.  The spatial fields s and e
   enter as spatial TTs from a TT-SVD of the field (``field_tt``): the
   Hadamard product with s multiplies the spatial ranks (Sec. 4.1,
   Multiplication; rank one when sigma_a and sigma_s are uniform), e is one
   more TT term;
3. rounding (App. A) of the whole d-core TT to eps, once per step or after
   transport and again after the source;
4. temperature: C_v (T^{m+1} - T^m) = E* - E^{m+1}, E^{m+1} integrated from the
   rounded TT (energy conserved through the source and the rounding).
"""
import numpy as np

from . import angles, tt
from .quartic import t_dagger
from .rounding import round_gram, round_ttsvd

PERIODIC = 0
VACUUM = 1
OUTFLOW = 2


def field_tt(F, rel_tol=1e-15):
    """TT of a spatial field F (shape n) by TT-SVD (Oseledets 2011): sequential
    reshapes and SVDs, keeping singular values above rel_tol times the largest
    of each unfolding (exact to rounding for rel_tol near eps_mach)."""
    F = np.asarray(F, float)
    n = F.shape
    cores = []
    rest = F.reshape(1, -1)
    r = 1
    for k in range(len(n) - 1):
        M = rest.reshape(r * n[k], -1)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        keep = max(1, int(np.sum(S > rel_tol * (S[0] if S.size and S[0] > 0 else 1.0))))
        cores.append(U[:, :keep].reshape(r, n[k], keep))
        rest = S[:keep, None] * Vt[:keep]
        r = keep
    cores.append(rest.reshape(r, n[-1], 1))
    return cores


def spatial_full(spatial_cores, right):
    """Contract spatial cores (r_{k-1}, n_k, r_k) with a right vector of the
    last spatial bond: the field sum_a G_1 ... G_ndim[:, :, a] right[a]."""
    out = np.ones((1, 1))
    for G in spatial_cores:
        out = np.tensordot(out, G, axes=([out.ndim - 1], [0]))
    out = np.tensordot(out, right, axes=([out.ndim - 1], [0]))
    return out.reshape(out.shape[1:])


class SplitTTSN:
    def __init__(self, n, L, n_theta, n_phi, c, a_r, dt, bc, sigma_a, cv, T0,
                 cores, sigma_s=None, eps=0.0, max_rank=None, rounds_per_step=1,
                 rounding="gram"):
        self.ndim = len(n)
        self.n = tuple(n)
        self.dx = [L[a] / n[a] for a in range(self.ndim)]
        self.c, self.a_r, self.dt = float(c), float(a_r), float(dt)
        self.bc = list(bc)
        self.g = angles.grid(n_theta, n_phi)
        self.sigma_a = np.broadcast_to(np.asarray(sigma_a, float), self.n).copy()
        self.sigma_s = (np.zeros(self.n) if sigma_s is None
                        else np.broadcast_to(np.asarray(sigma_s, float), self.n).copy())
        self.cv = np.broadcast_to(np.asarray(cv, float), self.n).copy()
        self.T = np.array(T0, float).reshape(self.n).copy()
        self.cores = [np.array(G, float) for G in cores]
        assert len(self.cores) == self.ndim + 2
        self.eps, self.max_rank = eps, max_rank
        self.rounds_per_step = rounds_per_step
        self.rounding = rounding
        self.last_ranks = []
        self.last_sigmas = []

    @staticmethod
    def isotropic_cores(I_field, n_theta, n_phi, rel_tol=1e-15):
        """Split TT of an isotropic intensity field I(x) (shape n)."""
        return field_tt(I_field, rel_tol) + [np.ones((1, n_theta, 1)), np.ones((1, n_phi, 1))]

    # -- D^-/+ along the mode of one spatial core (Sec. 4.3, ghosts of Sec. 4.5)
    def _shift(self, G, axis, offset):
        """Slice i of the result is slice i + offset of G's mode (periodic wrap,
        a zero ghost slice, or the edge slice for outflow)."""
        if self.bc[axis] == PERIODIC:
            return np.roll(G, -offset, axis=1)
        if self.bc[axis] == OUTFLOW:
            idx = np.clip(np.arange(G.shape[1]) + offset, 0, G.shape[1] - 1)
            return G[:, idx]
        Z = np.zeros_like(G)
        N = G.shape[1]
        if offset > 0:
            Z[:, : N - offset] = G[:, offset:]
        else:
            Z[:, -offset:] = G[:, : N + offset]
        return Z

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

    def transport(self, cores):
        nd = self.ndim
        terms = [cores]
        for a in range(nd):
            nu = self.c * self.dt / self.dx[a]
            Ga = cores[a]
            Dm = Ga - self._shift(Ga, a, -1)
            Dp = self._shift(Ga, a, +1) - Ga
            (tp, pp), (tm, pm) = self._masks(a)
            for D, tmask, pmask in ((Dm, tp, pp), (Dp, tm, pm)):
                term = [G.copy() for G in cores]
                term[a] = -nu * D
                term[nd] = cores[nd] * tmask[None, :, None]
                term[nd + 1] = cores[nd + 1] * pmask[None, :, None]
                terms.append(term)
        return tt.add_many(terms)

    def energy_density(self, cores=None):
        """E = (1/c) sum_lp I w_l v_p (Eq. tt_energy_density), field of shape n."""
        cores = self.cores if cores is None else cores
        nd = self.ndim
        Th, Ph = cores[nd], cores[nd + 1]
        phibar = np.einsum("bp,p->b", Ph[:, :, 0], self.g["v"])
        thbar = np.einsum("alb,l,b->a", Th, self.g["w"], phibar)
        return spatial_full(cores[:nd], thbar) / self.c

    def source(self, cores):
        c, a_r, dt = self.c, self.a_r, self.dt
        k_a = c * dt * self.sigma_a
        k_s = c * dt * self.sigma_s
        E_star = self.energy_density(cores)
        Td = t_dagger(self.T.reshape(-1), E_star.reshape(-1), k_a.reshape(-1),
                      self.cv.reshape(-1), a_r).reshape(self.n)
        B = c * a_r * Td ** 4 / (4.0 * np.pi)
        J_new = (c * E_star / (4.0 * np.pi) + k_a * B) / (1.0 + k_a)
        s = 1.0 / (1.0 + k_a + k_s)
        e = s * (k_s * J_new + k_a * B)
        nt, npf = len(self.g["mu"]), len(self.g["phi"])
        ones = [np.ones((1, nt, 1)), np.ones((1, npf, 1))]
        if np.all(s == s.flat[0]):
            scaled = tt.scale(cores, float(s.flat[0]))
        else:
            scaled = tt.hadamard(cores, field_tt(s) + ones)
        return tt.add(scaled, field_tt(e) + ones), E_star, Td

    def round(self, cores, forced=None):
        if self.rounding is None:
            return cores
        fn = round_gram if self.rounding == "gram" else round_ttsvd
        out, sig = fn(cores, self.eps, self.max_rank, forced)
        self.last_sigmas.append(sig)
        self.last_ranks.append(tt.ranks(out))
        return out

    def step(self, forced=None, forced2=None, with_source=True):
        self.last_ranks = []
        self.last_sigmas = []
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
        return tt.full(self.cores)

    def total_energy(self):
        dV = float(np.prod(self.dx))
        return float(np.sum(self.energy_density() + self.cv * self.T) * dV)
