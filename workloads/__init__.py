"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package holds input *generators* only: meshes, per-element coefficient
fields, initial-condition functions of physical coordinates, source wavelets
and random nodal states.  It contains none of the DG method's arithmetic
(no reference element, no operators, no geometry factors, no fluxes), so
that the oracle and the CUDA library can both consume it without sharing
any solver code.

The paper (Section 4) only states that each polynomial degree was run on a
mesh of "approximately 2 million nodes"; no mesh or dataset is named.  The
jittered Kuhn cube meshes below stand in for it.
"""

from .mesh import kuhn_cube_mesh, six_tet_cube, n_for_target_nodes, num_nodes_per_element
from .fields import (acoustic_coefficients, elastic_two_layer, elastic_layered,
                     gaussian_pulse, random_state, ricker, standing_mode_acoustic,
                     standing_mode_elastic)
from .configs import (config1_acoustic_small, sweep_mesh, config4_requests,
                      config5_elastic_large, SWEEP_N)

__all__ = [
    "kuhn_cube_mesh", "six_tet_cube", "n_for_target_nodes", "num_nodes_per_element",
    "acoustic_coefficients", "elastic_two_layer", "elastic_layered", "gaussian_pulse",
    "random_state", "ricker", "standing_mode_acoustic", "standing_mode_elastic",
    "config1_acoustic_small", "sweep_mesh", "config4_requests", "config5_elastic_large",
    "SWEEP_N",
]
