"""Dense discrete-ordinates stepper (oracle; test infrastructure).

A plain full-tensor implementation of one time step of the paper's scheme,
written directly from its definitions with no tensor train involved:

* transport (Sec. 3.1): explicit RK1 finite-volume update, Eq. lhs, applied
  unsplit over the spatial axes, with the upwind interface flux of Eq. upwind
  (F = c n_a U_L if n_a >= 0 else c n_a U_R, piecewise-constant states);
* boundaries (Sec. 4.5): ghost cells, periodic = copy of the opposite edge,
  vacuum = zero ghost (no inflow) or a given rank-one inflow intensity,
  outflow = copy of the edge cell;
* source (Sec. 3.2): backward-Euler absorption/emission/scattering, Eq.
  couple_a / couple_b, with T-dagger from ``quartic.t_dagger``;
* temperature (Sec. 3.2, energy-conserving update): C_v (T^{m+1} - T^m) equals
  E* - E^{m+1}, where E* is the radiation energy entering the source stage
  (the post-transport moment) and E^{m+1} the energy after it;
* fixed external sources (optional): S = sum_k x_k(cell) theta_k(l) phi_k(p),
  an inhomogeneous term of the transport equation taken explicitly with the
  streaming, so the transport stage gives I* = L I + c dt S;
* interface fluxes (Sec. 3.1): ``upwind`` (Eq. upwind), ``rusanov`` (Eq.
  rusanov_flux_toro with S+ = rusanov_s c) or ``hll`` (Eq. hll with the wave
  speeds S_L, S_R of Sec. 3.1's piecewise definitions and the harmonic-mean
  optical depth of Eq. tauc, constants beta and tau_threshold), or
  ``rusanov_tau``: Eq. rusanov_flux_toro with a speed informed by the face's
  optical depth (Sec. 3.1), S+ = c |n_a| min(1, 1 / tau_c) with tau_c from
  Eq. tauc (constant beta = hll_beta): the thick-limit speed c |n_a| / tau_c
  of the series expansion after Eq. hll where tau_c >= 1, and c |n_a| (the
  flux is then upwinding) where the face is thin.  The ghost cell of a vacuum
  face takes the boundary cell's own opacity for Eq. tauc; a face with
  S_R = S_L (n_a = 0) carries no flux.

The intensity array has shape (N_x[, N_y[, N_z]], N_theta, N_phi); spatial
fields have shape (N_x[, N_y[, N_z]]).
"""
import numpy as np

from . import angles
from .quartic import t_dagger

PERIODIC = 0
VACUUM = 1
OUTFLOW = 2


class DenseSN:
    def __init__(self, n, L, n_theta, n_phi, c, a_r, dt, bc, sigma_a, cv, T0,
                 I0, sigma_s=None, sources=None, flux="upwind", rusanov_s=1.0, hll_beta=1.0,
                 hll_tau_threshold=1.0, inflow=None):
        self.flux = flux
        # inflow[(axis, side)] = (g, theta, phi): on that vacuum face the ghost
        # cells hold the rank-one intensity g(cell) theta(l) phi(p) instead of
        # zero (Sec. 4.5 ghost cells with a Dirichlet value); g is a field of
        # the grid's shape, read on the face's layer of cells
        self.inflow = {k: tuple(np.asarray(v, float) for v in vals) for k, vals in (inflow or {}).items()}
        self.rusanov_s = float(rusanov_s)
        self.hll_beta, self.hll_tau_threshold = float(hll_beta), float(hll_tau_threshold)
        self.ndim = len(n)
        self.n = tuple(n)
        self.dx = [L[a] / n[a] for a in range(self.ndim)]
        self.c, self.a_r, self.dt = float(c), float(a_r), float(dt)
        self.bc = list(bc)  # one entry per axis (same rule on both faces)
        self.g = angles.grid(n_theta, n_phi)
        self.nvec = angles.normals(self.g)
        self.dOmega = angles.solid_angles(self.g)
        self.sigma_a = np.array(sigma_a, float).reshape(self.n)
        self.sigma_s = (np.zeros(self.n) if sigma_s is None
                        else np.array(sigma_s, float).reshape(self.n))
        self.cv = np.array(cv, float).reshape(self.n)
        self.T = np.array(T0, float).reshape(self.n).copy()
        self.I = np.array(I0, float).reshape(self.n + (n_theta, n_phi)).copy()
        # S[i..., l, p] = sum_k x_k[i...] theta_k[l] phi_k[p]
        self.S = np.zeros_like(self.I)
        for x, th, ph in (sources or []):
            self.S += (np.asarray(x, float).reshape(self.n)[..., None, None]
                       * np.outer(np.asarray(th, float), np.asarray(ph, float)))

    # -- Sec. 3 discrete energy density: E_i = (1/c) sum_lp I_ilp dOmega_lp
    def energy_density(self, I=None):
        I = self.I if I is None else I
        return np.einsum("...lp,lp->...", I, self.dOmega) / self.c

    def _ghost_pad(self, I, axis):
        """Add one ghost cell on each side of ``axis`` (Sec. 4.5): zero (vacuum),
        the opposite edge (periodic) or a copy of the edge cell (outflow)."""
        pad = [(0, 0)] * I.ndim
        pad[axis] = (1, 1)
        if self.bc[axis] == OUTFLOW:
            return np.pad(I, pad, mode="edge")
        P = np.pad(I, pad)  # zeros: vacuum ghosts
        for side in (0, 1):
            if (axis, side) in self.inflow and self.bc[axis] == VACUUM:
                g, th, ph = self.inflow[(axis, side)]
                layer = [slice(None)] * (I.ndim - 2)
                layer[axis] = 0 if side == 0 else self.n[axis] - 1
                ghost = [slice(None)] * I.ndim
                ghost[axis] = 0 if side == 0 else -1
                P[tuple(ghost)] = g.reshape(self.n)[tuple(layer)][..., None, None] * np.outer(th, ph)
        if self.bc[axis] == PERIODIC:
            lo = [slice(None)] * I.ndim
            hi = [slice(None)] * I.ndim
            lo[axis] = 0
            hi[axis] = -1
            src_last = [slice(None)] * I.ndim
            src_first = [slice(None)] * I.ndim
            src_last[axis] = -1
            src_first[axis] = 0
            P[tuple(lo)] = I[tuple(src_last)]
            P[tuple(hi)] = I[tuple(src_first)]
        return P

    def _face_tau(self, a):
        """Eq. tauc at the N+1 faces of axis a: 2 beta dx / (1/sigma_L + 1/sigma_R),
        sigma = sigma_a + sigma_s, with the ghost cells' opacity (periodic: the
        wrapped cell, vacuum: the boundary cell itself); 0 if either is 0."""
        sig = self.sigma_a + self.sigma_s
        pad = [(0, 0)] * sig.ndim
        pad[a] = (1, 1)
        P = np.pad(sig, pad, mode="wrap" if self.bc[a] == PERIODIC else "edge")
        N = self.n[a]
        sl_L = [slice(None)] * sig.ndim
        sl_R = [slice(None)] * sig.ndim
        sl_L[a] = slice(0, N + 1)
        sl_R[a] = slice(1, N + 2)
        sL, sR = P[tuple(sl_L)], P[tuple(sl_R)]
        tau = np.zeros_like(sL)
        ok = (sL > 0.0) & (sR > 0.0)
        tau[ok] = 2.0 * self.hll_beta * self.dx[a] / (1.0 / sL[ok] + 1.0 / sR[ok])
        return tau

    def _hll_speeds(self, na, tau):
        """S_R, S_L of Sec. 3.1 (after Eq. hll) for normal component na (angles)
        and face optical depth tau (cells), broadcast to cells x angles."""
        c, thr = self.c, self.hll_tau_threshold
        t = tau[..., None, None]
        n = np.broadcast_to(na, t.shape[:-2] + na.shape)
        big = t >= thr
        with np.errstate(divide="ignore", invalid="ignore"):
            g2 = np.where(big, np.sqrt((1.0 - np.exp(-t ** 2)) / np.where(t > 0, t ** 2, 1.0)), 0.0)
            g4 = np.where(big, np.sqrt((1.0 - np.exp(-t ** 4)) / np.where(t > 0, t ** 2, 1.0)), 0.0)
        small_R = np.sqrt(np.maximum(1.0 - t ** 2 / 2.0, 0.0))
        pos = n >= 0.0
        S_R = np.where(pos, np.where(big, c * n * g2, c * n * small_R),
                       np.where(big, -c * n * g4, -c * n * t))
        S_L = np.where(pos, np.where(big, -c * n * g4, -c * n * t),
                       np.where(big, c * n * g2, c * n * small_R))
        return S_R, S_L

    def transport(self, I):
        """One explicit step of Eq. lhs with the chosen interface flux, summed
        over the spatial axes."""
        out = I.copy()
        for a in range(self.ndim):
            na = self.nvec[a]  # (N_theta, N_phi)
            P = self._ghost_pad(I, a)
            N = self.n[a]
            # face k (k = 0..N) sits between padded cells k and k+1, i.e. at i-1/2
            # for interior cell i = k; U_L = padded[k], U_R = padded[k+1].
            sl_L = [slice(None)] * I.ndim
            sl_R = [slice(None)] * I.ndim
            sl_L[a] = slice(0, N + 1)
            sl_R[a] = slice(1, N + 2)
            UL = P[tuple(sl_L)]
            UR = P[tuple(sl_R)]
            FL, FR = self.c * na * UL, self.c * na * UR
            if self.flux == "upwind":
                F = np.where(na >= 0.0, FL, FR)
            elif self.flux == "rusanov":
                F = 0.5 * (FL + FR) - 0.5 * self.rusanov_s * self.c * (UR - UL)
            elif self.flux == "rusanov_tau":
                tau = self._face_tau(a)[..., None, None]
                w = np.where(tau > 1.0, 1.0 / np.where(tau > 1.0, tau, 1.0), 1.0)
                F = 0.5 * (FL + FR) - 0.5 * self.c * np.abs(na) * w * (UR - UL)
            elif self.flux == "hll":
                S_R, S_L = self._hll_speeds(na, self._face_tau(a))
                den = S_R - S_L
                with np.errstate(divide="ignore", invalid="ignore"):
                    F = np.where(den != 0.0,
                                 (S_R * FL - S_L * FR + S_L * S_R * (UR - UL)) / np.where(den != 0.0, den, 1.0),
                                 0.0)
            else:
                raise ValueError(self.flux)
            hi = [slice(None)] * I.ndim
            lo = [slice(None)] * I.ndim
            hi[a] = slice(1, N + 1)   # F_{i+1/2}
            lo[a] = slice(0, N)       # F_{i-1/2}
            out -= (self.dt / self.dx[a]) * (F[tuple(hi)] - F[tuple(lo)])
        return out + self.c * self.dt * self.S

    def source(self, Istar):
        """Backward-Euler source stage (Eq. couple_a / couple_b); returns
        (I^{m+1}, T^{m+1}, T_dagger, E_star)."""
        c, a_r, dt = self.c, self.a_r, self.dt
        k_a = c * dt * self.sigma_a
        k_s = c * dt * self.sigma_s
        E_star = self.energy_density(Istar)
        J_star = c * E_star / (4.0 * np.pi)
        Td = t_dagger(self.T, E_star, k_a, self.cv, a_r)
        B = c * a_r * Td ** 4 / (4.0 * np.pi)
        J_new = (J_star + k_a * B) / (1.0 + k_a)
        num = Istar + (k_s * J_new + k_a * B)[..., None, None]
        I_new = num / (1.0 + k_a + k_s)[..., None, None]
        E_new = self.energy_density(I_new)
        T_new = self.T + (E_star - E_new) / self.cv
        return I_new, T_new, Td, E_star

    def step(self, with_source=True):
        Istar = self.transport(self.I)
        if with_source:
            self.I, self.T, _, _ = self.source(Istar)
        else:
            self.I = Istar
        return self.I

    def total_energy(self):
        """sum_i (E_i + C_v,i T_i) dV."""
        dV = float(np.prod(self.dx))
        return float(np.sum(self.energy_density() + self.cv * self.T) * dV)
