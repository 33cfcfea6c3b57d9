"""Plain FP64 CPU oracle of the hybrid thermal LB phase-change step (arXiv 1812.10375).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py`` may import it.  It shares
no code with the GPU library and never imports it.
"""
from . import eos, lattice
from .domain import Domain, Params, nucleation_Gw, TOP_WALL, TOP_CONST_RHO, TOP_CONVECTIVE

__all__ = ["eos", "lattice", "Domain", "Params", "nucleation_Gw",
           "TOP_WALL", "TOP_CONST_RHO", "TOP_CONVECTIVE"]
