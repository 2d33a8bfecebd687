"""Seeded synthetic inputs for the TT-S_N step (shared by the CUDA path's tests
and bench and by the oracle's tests).

This module only *generates inputs*: grids, material fields, initial
temperatures, random tensor-train cores.  It contains none of the method's
arithmetic (no transport, quadrature, source or rounding).  The initial
radiation field is described by a radiation temperature ``Tr0``; each side
builds its own initial intensity from it.

Workloads (unit box [0,1]^ndim, cell-centred, c = a_r = 1, C_v = 1):

* ``small_2d``    2D 32x32 cells, 8x16 ordinates, sigma_a = 1, Gaussian T pulse
                  (peak 1, width 0.1, background 0.01), periodic, CFL 0.5,
                  10 steps, eps = 1e-8.
* ``blob_3d``     3D 128^3 cells, 32x64 ordinates, sigma_a = 1e2 inside a union
                  of 16 random spheres (seed 0, centres U[0,1]^3, radii
                  U[0.05, 0.15]) and 1e-2 elsewhere, T = 1 in a sphere of radius
                  0.1 at the centre and 1e-3 outside, vacuum, CFL 0.5,
                  100 steps, eps = 1e-6, rank cap 128.
* ``scaled``      any of the above with other cell / ordinate counts (for tests).
* ``gaussian_diffusion``  the 2D Gaussian-diffusion setup of Sec. 5 (domain
                  5 x 5, 128^2 cells, pure isotropic scattering rho kappa_s = 1e3,
                  no absorption, radiation initialised to a Gaussian E of
                  amplitude A = 1 at t0 = 200 with D = c / (3 rho kappa_s));
                  vacuum faces stand in for outflow.
* ``hohlraum``    the 2D hohlraum of Sec. 5.1: [0, 2]^2, vacuum faces with
                  isotropic unit inflow on x = 0 and y = 0, no material,
                  empty start, to t = 0.75.
* ``line_source`` the 2D line source of Sec. 5.4: [-1.1, 1.1]^2 (stored as
                  [0, 2.2]^2 about its centre), 500^2 cells, a Gaussian pulse of
                  radiation (width 0.03, total energy 1) in an empty vacuum
                  domain, CFL 0.4, to t = 1.
"""
import numpy as np

PERIODIC = 0
VACUUM = 1


def cell_centres(n, L):
    axes = [(np.arange(n[a]) + 0.5) * (L[a] / n[a]) for a in range(len(n))]
    return np.meshgrid(*axes, indexing="ij")


def gaussian_pulse(n, L, peak=1.0, width=0.1, background=0.01, centre=None):
    X = cell_centres(n, L)
    if centre is None:
        centre = [0.5 * L[a] for a in range(len(n))]
    r2 = sum((X[a] - centre[a]) ** 2 for a in range(len(n)))
    return background + peak * np.exp(-r2 / (2.0 * width * width))


def sphere_mask(n, L, centre, radius):
    X = cell_centres(n, L)
    r2 = sum((X[a] - centre[a]) ** 2 for a in range(len(n)))
    return r2 <= radius * radius


def blob_mask(n, L, seed=0, count=16, rmin=0.05, rmax=0.15):
    rng = np.random.default_rng(seed)
    ndim = len(n)
    mask = np.zeros(tuple(n), bool)
    X = cell_centres(n, L)
    for _ in range(count):
        c = rng.uniform(0.0, 1.0, ndim) * np.asarray(L[:ndim])
        r = rng.uniform(rmin, rmax)
        r2 = sum((X[a] - c[a]) ** 2 for a in range(ndim))
        mask |= r2 <= r * r
    return mask


def problem(name="small_2d", n=None, n_theta=None, n_phi=None, **over):
    """Return a dict describing a problem: grid, ordinates, constants, fields
    (fp64 numpy arrays of shape ``n`` in C order), bc per axis, eps, rank cap,
    step count and dt = CFL * min(dx) / c."""
    if name == "small_2d":
        p = dict(n=(32, 32), n_theta=8, n_phi=16, bc=PERIODIC, eps=1e-8,
                 max_rank=128, steps=10, cfl=0.5)
    elif name == "blob_3d":
        p = dict(n=(128, 128, 128), n_theta=32, n_phi=64, bc=VACUUM, eps=1e-6,
                 max_rank=128, steps=100, cfl=0.5)
    else:
        raise ValueError(name)
    if n is not None:
        p["n"] = tuple(n)
    if n_theta is not None:
        p["n_theta"] = n_theta
    if n_phi is not None:
        p["n_phi"] = n_phi
    nn = p["n"]
    ndim = len(nn)
    L = (1.0,) * ndim
    p.update(L=L, c=1.0, a_r=1.0, name=name)
    if name == "small_2d":
        T0 = gaussian_pulse(nn, L, 1.0, 0.1, 0.01)
        sigma_a = np.ones(nn)
    else:
        centre = [0.5] * ndim
        T0 = np.where(sphere_mask(nn, L, centre, 0.1), 1.0, 1e-3)
        sigma_a = np.where(blob_mask(nn, L, seed=0), 1e2, 1e-2)
    p.update(T0=T0, Tr0=T0.copy(), sigma_a=sigma_a, sigma_s=np.zeros(nn),
             cv=np.ones(nn))
    p.update(over)
    dx = min(p["L"][a] / p["n"][a] for a in range(ndim))
    p["dt"] = p["cfl"] * dx / p["c"]
    if np.isscalar(p["bc"]):
        p["bc"] = [int(p["bc"])] * ndim
    return p


def random_fields(n, seed, sigma_range=(0.1, 10.0), T_range=(0.2, 1.0)):
    """Random positive material fields for parity tests."""
    rng = np.random.default_rng(seed)
    nn = tuple(n)
    return dict(
        sigma_a=np.exp(rng.uniform(np.log(sigma_range[0]), np.log(sigma_range[1]), nn)),
        sigma_s=np.zeros(nn),
        cv=rng.uniform(0.5, 2.0, nn),
        T0=rng.uniform(T_range[0], T_range[1], nn),
    )


def random_tt(n_modes, ranks, seed, scale=1.0):
    """Random TT cores with N(0,1) entries: core k has shape
    (ranks[k-1], n_modes[k], ranks[k]) with ranks[-1] = ranks[d] = 1."""
    rng = np.random.default_rng(seed)
    d = len(n_modes)
    r = [1] + list(ranks) + [1]
    return [scale * rng.standard_normal((r[k], n_modes[k], r[k + 1])) for k in range(d)]


def random_positive_tt(n_modes, ranks, seed):
    """Random TT with positive entries in [0.5, 1.5) (a positive intensity)."""
    rng = np.random.default_rng(seed)
    d = len(n_modes)
    r = [1] + list(ranks) + [1]
    return [rng.uniform(0.5, 1.5, (r[k], n_modes[k], r[k + 1])) / r[k] for k in range(d)]


def batch_problems(count=64, seed=0):
    """Independent 2D problems of uneven sizes: grids from {64^2, 128^2, 256^2},
    ordinates from {16x32, 32x64}, uniform sigma_a log-uniform in [1e-2, 1e2],
    a Gaussian T pulse (centre U[0.3,0.7]^2, width U[0.05,0.15], peak
    U[0.5,1], background 0.01) in equilibrium with the radiation, eps from
    {1e-4, 1e-6}, rank cap U{8..96}, periodic, CFL 0.5."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.choice([64, 128, 256]))
        nt, npf = [(16, 32), (32, 64)][int(rng.integers(0, 2))]
        n = (m, m)
        L = (1.0, 1.0)
        centre = rng.uniform(0.3, 0.7, 2)
        T0 = gaussian_pulse(n, L, rng.uniform(0.5, 1.0), rng.uniform(0.05, 0.15), 0.01, centre)
        sig = 10.0 ** rng.uniform(-2, 2)
        p = dict(n=n, L=L, n_theta=nt, n_phi=npf, bc=[PERIODIC, PERIODIC],
                 eps=float(rng.choice([1e-4, 1e-6])), max_rank=int(rng.integers(8, 97)),
                 steps=10, cfl=0.5, c=1.0, a_r=1.0, name="batch",
                 T0=T0, Tr0=T0.copy(), sigma_a=np.full(n, sig), sigma_s=np.zeros(n), cv=np.ones(n))
        p["dt"] = p["cfl"] * (1.0 / m) / p["c"]
        out.append(p)
    return out


def gaussian_random_field(n, seed=0, corr=0.1, L=None):
    """Smooth random field: white noise (seeded) filtered in Fourier space by a
    Gaussian kernel of correlation length ``corr`` (periodic), normalised to
    mean 0 and standard deviation 1."""
    rng = np.random.default_rng(seed)
    n = tuple(n)
    L = L or (1.0,) * len(n)
    noise = rng.standard_normal(n)
    F = np.fft.fftn(noise)
    k2 = np.zeros(n)
    for a, m in enumerate(n):
        k = 2 * np.pi * np.fft.fftfreq(m, d=L[a] / m)
        shape = [1] * len(n)
        shape[a] = m
        k2 = k2 + (k ** 2).reshape(shape)
    g = np.real(np.fft.ifftn(F * np.exp(-0.5 * k2 * corr * corr)))
    return (g - g.mean()) / g.std()


def grf_problem(n=(128, 128), n_theta=32, n_phi=64, steps=20, eps=1e-6, max_rank=0, seed=0,
                centre=None):
    """Adjoint workload: sigma_a = exp(g) with g a Gaussian random field (corr.
    length 0.1, seed), a Gaussian T pulse (peak 1, width 0.1, background 0.01)
    in equilibrium, vacuum boundaries, CFL 0.5.  The pulse sits at 0.8 of the
    last axis (0.5 of the others) by default, 0.15 + 1.5 widths from that face,
    so part of it reaches the face within the run and the escape energy is not
    only the background's."""
    p = problem("small_2d", n=n, n_theta=n_theta, n_phi=n_phi, eps=eps, bc=VACUUM,
                max_rank=max_rank, steps=steps)
    ndim = len(p["n"])
    if centre is None:
        centre = [0.5] * (ndim - 1) + [0.8]
    centre = [c * p["L"][a] for a, c in enumerate(centre)]
    p["T0"] = gaussian_pulse(p["n"], p["L"], 1.0, 0.1, 0.01, centre)
    p["Tr0"] = p["T0"].copy()
    p["sigma_a"] = np.exp(gaussian_random_field(p["n"], seed=seed, corr=0.1))
    p["name"] = "grf_2d"
    return p


def cone_window(n_theta, n_phi, phi0, half_angle=10.0):
    """Angular window of a collimated source in (theta, phi) index space:
    1 on ordinates with |theta_l - 90 deg| <= half_angle and phi_p within
    half_angle of phi0 (degrees, circular), else 0 -- a (theta) x (phi)
    product, so the source is rank one in angle.  Where no ordinate lies
    inside (coarse grids) the nearest ones (all at the least distance) are
    taken."""
    mu = -1.0 + (np.arange(n_theta) + 0.5) * (2.0 / n_theta)
    theta = np.degrees(np.arccos(mu))
    phi = (np.arange(n_phi) + 0.5) * (360.0 / n_phi)
    dth = np.abs(theta - 90.0)
    dph = np.abs((phi - phi0 + 180.0) % 360.0 - 180.0)

    def window(d):
        lim = max(half_angle, d.min() + 1e-9)
        return (d <= lim).astype(float)

    return window(dth), window(dph)


def crossing_beams(n=(256, 256), n_theta=64, n_phi=128, eps=1e-5, max_rank=96, steps=400,
                   strength=(1.0, 0.5), half_angle=10.0):
    """Precision-form workload: two fixed collimated sources whose beams cross.
    Source 1: a 4x4-cell patch at the centre of the x = 0 edge emitting toward
    +x (phi0 = 0); source 2: a 4x4 patch at the centre of the y = 0 edge toward
    +y (phi0 = 90 deg); each isotropic inside a +-half_angle window in
    (theta, phi) with intensities ``strength`` (per unit length, added as
    c dt S per step).  The unequal strengths break the x <-> y mirror symmetry,
    which would otherwise pair the singular values and make a rank cut inside
    a pair ambiguous.  sigma_a = 1e-3 uniform, T = 1e-3 in equilibrium,
    C_v = 1, vacuum, CFL 0.5, eps 1e-5, ranks <= 96."""
    nx, ny = n
    p = problem("small_2d", n=n, n_theta=n_theta, n_phi=n_phi, eps=eps, bc=VACUUM,
                max_rank=max_rank, steps=steps)
    T0 = np.full(n, 1e-3)
    p.update(T0=T0, Tr0=T0.copy(), sigma_a=np.full(n, 1e-3), name="crossing_beams")
    x1 = np.zeros(n)
    x1[0:4, ny // 2 - 2:ny // 2 + 2] = strength[0]
    x2 = np.zeros(n)
    x2[nx // 2 - 2:nx // 2 + 2, 0:4] = strength[1]
    th1, ph1 = cone_window(n_theta, n_phi, 0.0, half_angle)
    th2, ph2 = cone_window(n_theta, n_phi, 90.0, half_angle)
    p["sources"] = [(x1, th1, ph1), (x2, th2, ph2)]
    return p


def gaussian_diffusion(n=(128, 128), n_theta=8, n_phi=16, sigma_s=1e3, t0=200.0, amp=1.0, L=5.0,
                       eps=1e-6, max_rank=0, cfl=0.5):
    """Scattering-dominated diffusion of a 2D Gaussian pulse: E(0, x, y) =
    A / (4 pi D t0) exp(-r^2 / (4 D t0)) about the domain centre, D = c / (3
    sigma_s), sigma_a = 0 (the material decouples), given through the
    radiation temperature Tr0 = E^(1/4) (a_r = 1).  The paper runs it with the
    Rusanov flux at S+ = 0."""
    p = problem("small_2d", n=n, n_theta=n_theta, n_phi=n_phi, eps=eps, bc=VACUUM,
                max_rank=max_rank, L=(L, L), cfl=cfl)
    D = p["c"] / (3.0 * sigma_s)
    xc = cell_centres(p["n"], p["L"])
    centre = [0.5 * L, 0.5 * L]
    r2 = sum((x - c0) ** 2 for x, c0 in zip(xc, centre))
    E0 = amp / (4.0 * np.pi * D * t0) * np.exp(-r2 / (4.0 * D * t0))
    p.update(sigma_a=np.zeros(p["n"]), sigma_s=np.full(p["n"], float(sigma_s)),
             T0=np.full(p["n"], 1e-3), Tr0=E0 ** 0.25, name="gaussian_diffusion",
             D=D, t0=t0, amp=amp, centre=centre)
    return p


def hohlraum(n=(256, 256), n_theta=32, n_phi=64, eps=1e-4, max_rank=0, t_lim=0.75, cfl=0.5):
    """The 2D hohlraum of Sec. 5.1: domain [0, 2]^2, vacuum faces, isotropic
    unit inflow (I = J = 1) through the x = 0 and y = 0 faces, no material
    (sigma = 0), radiation initially absent, run to t = 0.75.  ``inflow`` maps
    (axis, side) to the rank-one ghost intensity (face field, theta, phi)."""
    p = problem("small_2d", n=n, n_theta=n_theta, n_phi=n_phi, eps=eps, bc=VACUUM,
                max_rank=max_rank, L=(2.0, 2.0), cfl=cfl)
    nn = p["n"]
    p.update(sigma_a=np.zeros(nn), T0=np.full(nn, 1e-3), Tr0=np.zeros(nn), name="hohlraum",
             t_lim=t_lim)
    unit = (np.ones(nn), np.ones(n_theta), np.ones(n_phi))
    p["inflow"] = {(0, 0): unit, (1, 0): unit}
    return p


def line_source(n=(500, 500), n_theta=32, n_phi=64, eps=1e-4, max_rank=0, omega=0.03, U0=1.0,
                half_width=1.1, t_lim=1.0, cfl=0.4):
    """The 2D line source of Sec. 5.4: an isotropic Gaussian pulse of
    radiation, E(0) = U0 / (2 pi omega^2) exp(-r^2 / (2 omega^2)) sampled at
    the cell centres, about the centre of the square [-h, h]^2 (held as
    [0, 2h]^2), no material (sigma = 0, so the source stage leaves I and T
    unchanged), vacuum faces, given through the radiation temperature
    Tr0 = E^(1/4) (a_r = 1).  The front reaches radius c t_lim < h, so no
    radiation leaves by t_lim up to the scheme's numerical spreading."""
    L = 2.0 * half_width
    p = problem("small_2d", n=n, n_theta=n_theta, n_phi=n_phi, eps=eps, bc=VACUUM,
                max_rank=max_rank, L=(L, L), cfl=cfl)
    xc = cell_centres(p["n"], p["L"])
    r = np.sqrt(sum((x - half_width) ** 2 for x in xc))
    E0 = U0 / (2.0 * np.pi * omega ** 2) * np.exp(-r ** 2 / (2.0 * omega ** 2))
    p.update(sigma_a=np.zeros(p["n"]), T0=np.full(p["n"], 1e-3), Tr0=E0 ** 0.25, name="line_source",
             omega=omega, U0=U0, radius=r, t_lim=t_lim)
    return p
