"""Analytic solutions of the paper's validation problems (oracle; test
infrastructure: only the tests, the smoke check and the bench's CPU-baseline
leg use this package).

* ``hohlraum_J``      the mean intensity of the 2D hohlraum (Sec. 5.1):
                      isotropic unit inflow through the x = 0 and y = 0 faces
                      of an empty vacuum domain.
* ``line_source_E``   the radiation energy density of the 2D line source
                      (Sec. 5.4): the vacuum Green's function of a planar
                      delta pulse, E = U0 H(ct - r) / (2 pi ct sqrt((ct)^2 -
                      r^2)), convolved with the Gaussian initial pulse
                      U0 / (2 pi w^2) exp(-r^2 / (2 w^2)).

The convolution is radial.  Writing the Green's function in polar
coordinates about the evaluation point and averaging the Gaussian over the
polar angle gives

    E(t, rho) = int_0^ct  r / (ct sqrt((ct)^2 - r^2))  Gbar(rho, r) dr,
    Gbar(rho, r) = U0 / (2 pi w^2) exp(-(rho^2 + r^2) / (2 w^2)) I_0(rho r / w^2),

with I_0 the modified Bessel function (the angular mean of exp(x cos psi)).
The substitution r = ct sin(a) turns the kernel into sin(a) da on
[0, pi/2] and removes the endpoint singularity; the integral is then taken by
composite Gauss-Legendre quadrature with panels narrower than the pulse
width, and I_0 is evaluated in its exponentially scaled form so that
exp(-(rho - r)^2 / (2 w^2)) i0e(rho r / w^2) stays finite for any radii.
"""
import numpy as np
from scipy.special import i0e


def hohlraum_J(t, x, y, c=1.0):
    """Analytic mean intensity of the hohlraum test (Sec. 5.1, after White
    2023): isotropic I = J = 1 on the x = 0 and y = 0 faces of a vacuum
    domain, the sum of the two faces' single-face solutions."""
    def part(u, v):
        ct = c * t
        with np.errstate(invalid="ignore", divide="ignore"):
            eta = np.arccos(np.minimum(v / np.sqrt(np.maximum(ct ** 2 - u ** 2, 1e-300)), 1.0))
            r = np.sqrt(u ** 2 + v ** 2)
            val = 0.5 - (np.pi - eta) * u / (2 * np.pi * ct) - np.arcsin(u * np.sin(eta) / r) / (2 * np.pi)
        return np.where(u < ct, val, 0.0)
    return part(x, y) + part(y, x)


def _panels(lo, hi, panels, q):
    x, w = np.polynomial.legendre.leggauss(q)
    edges = np.linspace(lo, hi, panels + 1)
    half = 0.5 * (edges[1:] - edges[:-1])
    nodes = (half[:, None] * (x[None] + 1.0) + edges[:-1, None]).ravel()
    weights = (half[:, None] * w[None]).ravel()
    return nodes, weights


def line_source_E(t, rho, omega, U0=1.0, c=1.0, panels=None, q=16):
    """E(t, rho) of the Gaussian line source (Sec. 5.4) at radii ``rho`` (any
    shape) from the pulse centre: the radial form of the convolution above.
    ``panels`` Gauss-Legendre panels of ``q`` points on a in [0, pi/2]; by
    default four panels per pulse width w / (ct)."""
    rho = np.asarray(rho, float)
    ct = c * float(t)
    norm = U0 / (2.0 * np.pi * omega ** 2)
    if ct == 0.0:
        return norm * np.exp(-rho ** 2 / (2.0 * omega ** 2))
    if panels is None:
        panels = int(np.clip(np.ceil(4.0 * ct / omega), 32, 8192))
    a, wa = _panels(0.0, 0.5 * np.pi, panels, q)
    r = ct * np.sin(a)
    kern = np.sin(a) * wa
    flat = rho.reshape(-1)
    out = np.empty(flat.shape)
    step = max(1, (1 << 22) // a.size)
    for s in range(0, flat.size, step):
        R = flat[s:s + step, None]
        g = np.exp(-(R - r) ** 2 / (2.0 * omega ** 2)) * i0e(R * r / omega ** 2)
        out[s:s + step] = norm * (g @ kern)
    return out.reshape(rho.shape)


def line_source_green(t, rho, U0=1.0, c=1.0):
    """The vacuum Green's function of the planar delta pulse (Sec. 5.4):
    U0 H(ct - rho) / (2 pi ct sqrt((ct)^2 - rho^2)), zero outside the front."""
    rho = np.asarray(rho, float)
    ct = c * float(t)
    with np.errstate(invalid="ignore", divide="ignore"):
        v = U0 / (2.0 * np.pi * ct * np.sqrt(ct ** 2 - rho ** 2))
    return np.where(rho < ct, v, 0.0)
