"""Shared test helpers: one workload case built for the oracle and for the library."""
from __future__ import annotations

import numpy as np

from oracle import Domain as ODomain, Params as OParams, eos, nucleation_Gw
from paper_1812_10375_gb300 import workloads as wl


def coexistence():
    pr = eos.PR()
    Ts = 0.86 * pr.Tc
    rl, rv, _ = eos.coexistence(Ts, pr)
    return dict(Tc=pr.Tc, Ts=Ts, rho_l=rl, rho_v=rv)


def oracle_domain(case: wl.Case, coex, rho0=None, T0=None, **extra) -> ODomain:
    """The FP64 reference domain of a case; `extra` overrides Params fields."""
    Tc = coex["Tc"]
    if rho0 is None:
        rho0, T0 = wl.initial_fields(case, coex["rho_l"], coex["rho_v"], Tc)
    Gw = nucleation_Gw(case.nx, case.Gw0, case.sites)
    kw = {}
    if case.name == "flat_interface":
        kw["lambda_w"] = coex["rho_v"] * 6.0 * 0.1
    p = OParams(nx=case.nx, ny=case.ny, wall_rows=case.wall_rows, top_bc=case.top_bc,
                T_bottom=case.T_bottom(Tc), T_top=case.T_top(Tc), eos_T_fixed=case.eos_T_fixed,
                g_y=case.g_y, Gw=Gw, rho_l=coex["rho_l"], rho_v=coex["rho_v"], **{**kw, **extra})
    return ODomain(p, rho0, T0)


def gpu_domain(case: wl.Case, coex, storage=0, rho0=None, T0=None, **extra):
    """The library domain of a case; `extra` overrides hlb_params fields."""
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    p, Tc = params_for(case, storage=storage, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    for k, v in extra.items():
        setattr(p, k, v)
    d = hlb.Domain(p)
    if rho0 is None:
        rho0, T0 = wl.initial_fields(case, coex["rho_l"], coex["rho_v"], Tc)
    d.set_fields(torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                 torch.tensor(T0, dtype=torch.float32, device="cuda"))
    if case.sites:
        d.set_nucleation_sites(case.sites)
    return d


def rel_linf(a, b, mask=None):
    """max|a - b| / max|b| over the mask."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def ragged_case(seed=3) -> wl.Case:
    """A closed box spanning several tiles with a ragged tail in both directions."""
    rng = np.random.default_rng(seed)
    sites = wl.draw_sites(rng, 45, 2)
    return wl.Case("ragged", nx=45, ny=37, wall_rows=6, top_bc="convective", T_bottom_over_Tc=0.86 + 0.12,
                   T_top_over_Tc=None, eos_T_fixed=False, g_y=-3e-5, Gw0=0.3, sites=sites)
