"""Latitude-longitude angular grid of Sec. 3 (oracle; test infrastructure).

The grid samples cos(theta) and phi uniformly and is a tensor product, so the
solid angle of ordinate (l, p) factors as dOmega_lp = w_l * v_p with
w_l = 2/N_theta (width in mu = cos(theta)) and v_p = 2*pi/N_phi; the weights
sum to 4*pi.  Ordinates sit at the cell centres in mu and in phi, and
theta_l = arccos(mu_l).  Unit normals follow Sec. 3:
n = (sin(theta) cos(phi), sin(theta) sin(phi), cos(theta)).
"""
import numpy as np


def grid(n_theta, n_phi):
    """Return dict with mu, sin_theta, phi, w (theta weights), v (phi weights)."""
    dmu = 2.0 / n_theta
    dphi = 2.0 * np.pi / n_phi
    mu = -1.0 + (np.arange(n_theta) + 0.5) * dmu
    phi = (np.arange(n_phi) + 0.5) * dphi
    return {
        "mu": mu,
        "sin_theta": np.sqrt(1.0 - mu * mu),
        "phi": phi,
        "w": np.full(n_theta, dmu),
        "v": np.full(n_phi, dphi),
    }


def normals(g):
    """Direction cosines (n_x, n_y, n_z), each an (N_theta, N_phi) array (Sec. 3)."""
    st = g["sin_theta"][:, None]
    ph = g["phi"][None, :]
    nx = st * np.cos(ph)
    ny = st * np.sin(ph)
    nz = g["mu"][:, None] * np.ones_like(ph)
    return nx, ny, nz


def solid_angles(g):
    """dOmega_lp = w_l v_p, an (N_theta, N_phi) array summing to 4 pi."""
    return np.outer(g["w"], g["v"])
