"""hlb_params for the synthetic workload cases (see workloads.py)."""
from __future__ import annotations

from . import hlb
from .workloads import Case


def params_for(case: Case, storage: int = hlb.HLB_STORE_DEVIATION, rho_l: float | None = None,
               rho_v: float | None = None) -> tuple[hlb.hlb_params, float]:
    """Library parameters of a case and its critical temperature Tc.

    rho_l / rho_v override the library's own coexistence solution (so two
    implementations can be run on identical parameters)."""
    p = hlb.default_params(case.nx, case.ny)
    Tc, rl, rv, _ = hlb.eos_coexistence(p)
    p.wall_rows = case.wall_rows
    p.top_bc = hlb.TOP_KIND[case.top_bc]
    p.eos_T_fixed = 1 if case.eos_T_fixed else 0
    p.storage = storage
    p.g_y = case.g_y
    p.Gw0 = case.Gw0
    p.T_bottom = case.T_bottom(Tc)
    p.T_top = case.T_top(Tc)
    p.rho_l = rl if rho_l is None else rho_l
    p.rho_v = rv if rho_v is None else rho_v
    if case.name == "flat_interface":
        # the Dirichlet walls of the 1D conduction case conduct like the adjacent vapour
        p.lambda_w = p.rho_v * p.cv * p.k
    return p, Tc
