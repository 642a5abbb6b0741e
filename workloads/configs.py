"""Synthetic stand-ins for the five workloads (seed = 1000 + workload index).

1. acoustic, N=2, 4x4x4 cubes x 6 = 384 tets, rho,c ~ U[1,2], Gaussian
   pulse, rigid walls, upwind, 100 AB3 steps (the parity case);
2. acoustic sweep N=1..8, ~2 M nodes per mesh, rho,c ~ U[1,3], 1000 steps;
3. elastic sweep N=1..8, ~2 M nodes, two-layer (lambda, mu, rho), Ricker
   point force;
4. a served stream of 64 acoustic shots, n ~ U{10..32}, N in {3,5,7},
   source position ~ U[0.2,0.8]^3, 500 steps each, Poisson arrivals;
5. large elastic, N=7, n=28 (131 712 tets, 15.8 M nodes), layered medium
   with +-30 % perturbation, 2000 steps.
"""

import numpy as np

from .mesh import kuhn_cube_mesh, n_for_target_nodes
from .fields import acoustic_coefficients, elastic_two_layer, elastic_layered

SWEEP_N = (1, 2, 3, 4, 5, 6, 7, 8)

# A source position inside the cube that avoids mesh vertices, edges and faces
# of the unjittered sub-cube lattice for every n used here.
DEFAULT_SOURCE = (0.5123, 0.4871, 0.5347)


def config1_acoustic_small():
    verts, tets = kuhn_cube_mesh(4, jitter=0.1, seed=1001)
    coeffs = acoustic_coefficients(tets.shape[0], 1.0, 2.0, seed=2001)
    return dict(model="acoustic", N=2, verts=verts, tets=tets, coeffs=coeffs,
                steps=100, flux="upwind", cfl=0.4)


def sweep_mesh(model, N, target_nodes=2_000_000, n=None):
    """Mesh + coefficients of the ~2 M-node sweep at degree N."""
    if n is None:
        n = n_for_target_nodes(N, target_nodes)
    if model == "acoustic":
        verts, tets = kuhn_cube_mesh(n, jitter=0.1, seed=1002)
        coeffs = acoustic_coefficients(tets.shape[0], 1.0, 3.0, seed=2002)
        steps = 1000
    elif model == "elastic":
        verts, tets = kuhn_cube_mesh(n, jitter=0.1, seed=1003)
        coeffs = elastic_two_layer(verts, tets, seed=2003)
        steps = 1000
    else:
        raise ValueError(model)
    return dict(model=model, N=N, n=n, verts=verts, tets=tets, coeffs=coeffs,
                steps=steps, flux="upwind", cfl=0.4, source=DEFAULT_SOURCE)


def config4_requests(count=64, rate=None, seed=1004):
    """Request descriptors of the served stream (meshes built lazily by the caller).

    ``rate`` is the Poisson arrival rate in requests/s (None -> all at t=0).
    """
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for i in range(count):
        n = int(rng.integers(10, 33))
        N = int(rng.choice([3, 5, 7]))
        src = tuple(rng.uniform(0.2, 0.8, size=3))
        if rate:
            t += rng.exponential(1.0 / rate)
        reqs.append(dict(index=i, n=n, N=N, source=src, steps=500, arrival=t,
                         mesh_seed=5000 + i, coeff_seed=6000 + i))
    return reqs


def request_mesh(req):
    verts, tets = kuhn_cube_mesh(req["n"], jitter=0.1, seed=req["mesh_seed"])
    coeffs = acoustic_coefficients(tets.shape[0], 1.0, 3.0, seed=req["coeff_seed"])
    return verts, tets, coeffs


def config5_elastic_large(n=28):
    verts, tets = kuhn_cube_mesh(n, jitter=0.1, seed=1005)
    coeffs = elastic_layered(verts, tets, seed=2005)
    return dict(model="elastic", N=7, n=n, verts=verts, tets=tets, coeffs=coeffs,
                steps=2000, flux="upwind", cfl=0.4, source=DEFAULT_SOURCE)
