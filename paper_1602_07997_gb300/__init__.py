"""GB300-native nodal discontinuous Galerkin wave solver (acoustic / elastic, AB3).

The compute path is the C-ABI library ``libdg.so`` (hand-written CUDA for
sm_103a, declared in ``include/dg.h``); this package only marshals
arguments to it.  Build it with ``python -m paper_1602_07997_gb300.build``.
"""

from ._lib import (Solver, Server, DGError, suggest_dt, reference_element, fp32_peak, tune_save, tune_load,
                   tune_clear, lib, EXPORTS, ACOUSTIC, ELASTIC)

__all__ = ["Solver", "Server", "DGError", "suggest_dt", "reference_element", "fp32_peak", "tune_save", "tune_load",
           "tune_clear", "lib", "EXPORTS", "ACOUSTIC", "ELASTIC"]
