"""Jittered Kuhn (Freudenthal) cube-tetrahedron meshes of the unit cube.

The unit cube [0,1]^3 is cut into n^3 sub-cubes and each sub-cube into the
six Kuhn tetrahedra that share the sub-cube's (0,0,0)-(1,1,1) diagonal.
Every sub-cube is cut the same way, so the mesh is conforming.  Each vertex
coordinate that does not lie on a boundary plane of the unit cube is moved
by ``jitter * h * U[-1, 1]`` (h = 1/n); coordinates on a boundary plane are
kept, so the outer faces stay planar.  Tetrahedra are returned positively
oriented: det[x2-x1, x3-x1, x4-x1] > 0.

Element order: sub-cubes lexicographically (x fastest), six tets per cube.
"""

import itertools

import numpy as np


def num_nodes_per_element(N):
    """Nodes per tetrahedron for degree N: (N+1)(N+2)(N+3)/6 (Section 2.2)."""
    return (N + 1) * (N + 2) * (N + 3) // 6


def _orient(verts, tets):
    a = verts[tets[:, 1]] - verts[tets[:, 0]]
    b = verts[tets[:, 2]] - verts[tets[:, 0]]
    c = verts[tets[:, 3]] - verts[tets[:, 0]]
    det = np.einsum("ij,ij->i", a, np.cross(b, c))
    neg = det < 0
    t = tets.copy()
    t[neg, 2], t[neg, 3] = tets[neg, 3], tets[neg, 2]
    return t


def kuhn_cube_mesh(n, jitter=0.1, seed=0):
    """Return (verts [nv,3] float64, tets [6 n^3, 4] int64)."""
    n = int(n)
    m = n + 1
    g = np.arange(m, dtype=np.float64) / n
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    if jitter:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-1.0, 1.0, size=verts.shape) * (jitter / n)
        on_bnd = (np.abs(verts) < 1e-14) | (np.abs(verts - 1.0) < 1e-14)
        d[on_bnd] = 0.0
        verts = verts + d

    def vid(i, j, k):
        return i + m * (j + m * k)

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # lexicographic with x fastest
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        off = np.zeros((4, 3), dtype=np.int64)
        for step, axis in enumerate(perm):
            off[step + 1] = off[step]
            off[step + 1, axis] += 1
        tets.append(np.stack([vid(ci + o[0], cj + o[1], ck + o[2]) for o in off], axis=1))
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int64)
    return verts, _orient(verts, tets)


def six_tet_cube(perturb=0.1, seed=0):
    """One unit cube cut into its 6 Kuhn tets with all 8 vertices perturbed.

    Every vertex (corners included) gets ``perturb * U[-1,1]`` per coordinate,
    so the outer boundary is no longer the unit cube, but each boundary face
    is still a planar triangle.
    """
    verts, tets = kuhn_cube_mesh(1, jitter=0.0)
    rng = np.random.default_rng(seed)
    verts = verts + rng.uniform(-1.0, 1.0, size=verts.shape) * perturb
    return verts, _orient(verts, tets)


def n_for_target_nodes(N, target=2_000_000):
    """Sub-cube count per axis whose 6 n^3 Np is closest to ``target``."""
    Np = num_nodes_per_element(N)
    best = None
    for n in range(1, 200):
        err = abs(6 * n ** 3 * Np - target)
        if best is None or err < best[0]:
            best = (err, n)
    return best[1]
