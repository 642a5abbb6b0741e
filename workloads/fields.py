"""Coefficient fields, initial data, source wavelets and exact solutions.

All functions here are plain functions of element indices, physical
coordinates or time.  Nodal initial data are obtained by the caller, who
evaluates these functions at its own node coordinates.
"""

import numpy as np


def _centroids(verts, tets):
    return verts[tets].mean(axis=1)


def acoustic_coefficients(K, lo=1.0, hi=2.0, seed=0):
    """[K,2] array of (rho, c) per tet, each ~ U[lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(K, 2))


def elastic_two_layer(verts, tets, seed=0):
    """[K,3] (lambda, mu, rho): centroid z < 1/2 -> U[1,2], else U[2,3]."""
    K = tets.shape[0]
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, size=(K, 3))
    upper = _centroids(verts, tets)[:, 2] >= 0.5
    return np.where(upper[:, None], 2.0 + u, 1.0 + u)


def elastic_layered(verts, tets, seed=0, layers=4, perturb=0.3):
    """[K,3] layered (lambda, mu, rho) = (1 + 0.5 l)(2, 1, 1) x (1 + perturb U[-1,1])."""
    K = tets.shape[0]
    rng = np.random.default_rng(seed)
    zc = _centroids(verts, tets)[:, 2]
    layer = np.clip((zc * layers).astype(np.int64), 0, layers - 1)
    base = (1.0 + 0.5 * layer)[:, None] * np.array([2.0, 1.0, 1.0])[None, :]
    return base * (1.0 + perturb * rng.uniform(-1.0, 1.0, size=(K, 3)))


def gaussian_pulse(xyz, width=0.1, centre=(0.5, 0.5, 0.5)):
    """exp(-|x - centre|^2 / width^2) at the points ``xyz[..., 3]``."""
    d = np.asarray(xyz) - np.asarray(centre)
    return np.exp(-np.sum(d * d, axis=-1) / (width * width))


def random_state(K, Nf, Np, seed=0):
    """Seeded random nodal state, layout [K][Nf][Np], float64 in [-1, 1]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(K, Nf, Np))


def ricker(t, f0=4.0, t0=None):
    """Ricker wavelet (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)."""
    if t0 is None:
        t0 = 1.2 / f0
    a = (np.pi * f0 * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def standing_mode_acoustic(xyz, t, rho=1.0, c=1.0):
    """Rigid-wall cube mode of the acoustic system, returns [..., 4] (p, vx, vy, vz).

    p = cos(pi x) cos(pi y) cos(pi z) cos(w t), v_x = pi/(rho w) sin(pi x)
    cos(pi y) cos(pi z) sin(w t) (cyclic), w = c pi sqrt(3).  v.n = 0 on
    every face of the unit cube.
    """
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    w = c * np.pi * np.sqrt(3.0)
    cx, cy, cz = np.cos(np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z)
    sx, sy, sz = np.sin(np.pi * x), np.sin(np.pi * y), np.sin(np.pi * z)
    a = np.pi / (rho * w) * np.sin(w * t)
    return np.stack([cx * cy * cz * np.cos(w * t), a * sx * cy * cz,
                     a * cx * sy * cz, a * cx * cy * sz], axis=-1)


def standing_mode_elastic(xyz, t, mu=1.0, rho=1.0):
    """Traction-free cube mode of the elastic system with lambda = 0.

    Displacement u_i = cos(pi x_i) cos(w t), w = pi sqrt(2 mu / rho).
    Returns [..., 9] = (vx, vy, vz, sxx, syy, szz, sxy, sxz, syz).
    """
    w = np.pi * np.sqrt(2.0 * mu / rho)
    out = np.zeros(xyz.shape[:-1] + (9,))
    for i in range(3):
        out[..., i] = -w * np.cos(np.pi * xyz[..., i]) * np.sin(w * t)
        out[..., 3 + i] = -2.0 * mu * np.pi * np.sin(np.pi * xyz[..., i]) * np.cos(w * t)
    return out
