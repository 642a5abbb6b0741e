"""FP64 CPU oracle for the nodal DG acoustic/elastic scheme (TEST INFRASTRUCTURE).

This package is a plain, slow, obviously-correct restatement of the method
of Modave, St-Cyr & Warburton, "GPU performance analysis of a nodal
discontinuous Galerkin method for acoustic and elastic models"
(arXiv:1602.07997): the physical models and upwind penalty terms of
Section 2.1, the nodal scheme (local RHS, Eq. dgLocalRhs) and the
third-order Adams-Bashforth update (Eq. updateScheme) of Section 2.2.

It is test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may
import it.  The CUDA library never imports, links or calls it, and it shares
no code with the CUDA library: operators are built here by quadrature from a
Bernstein basis in barycentric coordinates (the library uses an orthonormal-basis route), face
nodes are matched by physical coordinates (the library matches integer
lattice barycentrics), and every step runs in float64 with numpy.

Modules
-------
refelem  reference tetrahedron: warp-and-blend nodes, basis, quadrature,
         mass / differentiation / face-mass / lift matrices.
mesh     per-element geometry (Jacobian, inverse metric, normals, Fscale)
         and face / face-node connectivity.
dg       acoustic and elastic right-hand sides (volume + flux + lift),
         boundary ghosts, AB3 time stepping, discrete energy, sources.

The independent weak-form evaluation by physical-coordinate quadrature that
pins ``dg`` on tiny meshes lives with its test (tests/test_oracle_brute.py).
"""

from . import refelem, mesh, dg  # noqa: F401
