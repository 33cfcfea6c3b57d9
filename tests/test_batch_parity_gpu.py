"""The batched step (the benchmark's path: one launch per kernel for all
domains, descriptor tables, CUDA-graph replay) against the FP64 oracle,
domain by domain, element by element.

Three uneven domains share one batch: a sweep-sized 256 x 256 pool (25-row
heater, four seeded nucleation sites, convective top, gravity; most of its
tiles are interior tiles), a 72 x 60 film under a constant-density top and a
45 x 37 closed box with sites.  The pool is stopped after 200 steps (the
early-stop path), the others run to 1000 steps.  Tolerances as in
tests/test_parity_gpu.py: 1e-5 relative L-infinity on rho and T; on u, 1e-5
of the sound speed and U_FLOOR_FACTOR times the error of the oracle's
FP32-stored twin."""
import dataclasses

import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import U_FLOOR_FACTOR, coexistence, oracle_pair, ragged_case, rel_linf, u_error

pytestmark = pytest.mark.gpu
TOL = 1e-5
CS = 1.0 / np.sqrt(3.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def coex():
    return coexistence()


def _errors(fields, od, twin):
    rho_g, ux_g, uy_g, T_g = [t.cpu().numpy() for t in fields]
    rho_o, ux_o, uy_o, T_o = od.fields()
    fl = od.fluid
    du = u_error(ux_g, uy_g, od)
    du_floor = u_error(twin.ux, twin.uy, od)
    umax = float(np.sqrt(ux_o ** 2 + uy_o ** 2)[fl].max())
    err = dict(rho=rel_linf(rho_g, rho_o, fl), u=float(du / CS), T=rel_linf(T_g, T_o))
    return err, du / umax, du, du_floor


def test_batch_matches_oracle_per_domain(coex):
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    cases = [wl.pool(nx=256, ny=256, n_sites=4, seed=wl.BASE_SEED + 7),
             wl.film(nx=72, ny=60),
             dataclasses.replace(ragged_case(3), name="ragged_wall", top_bc="wall", T_top_over_Tc=0.86)]
    plist = [params_for(c, rho_l=coex["rho_l"], rho_v=coex["rho_v"])[0] for c in cases]
    b = hlb.Batch(plist)
    assert hlb.variant_kinds()[0] == hlb.HLB_KIND_SPLIT  # the benchmark's default path
    for i, c in enumerate(cases):
        rho0, T0 = wl.initial_fields(c, coex["rho_l"], coex["rho_v"], coex["Tc"])
        b.set_fields(i, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                     torch.tensor(T0, dtype=torch.float32, device="cuda"))
        b.set_nucleation_sites(i, c.sites)
    b.step(200)
    b.stop(0)
    b.step(800)
    steps = [200, 1000, 1000]
    for i, c in enumerate(cases):
        od, twin = oracle_pair(c, coex, steps[i])
        err, u_rel, du, du_floor = _errors(b.read(i), od, twin)
        dg, do = b.diag(i), od.diag()
        print(f"{c.name} ({c.nx}x{c.ny}, {steps[i]} steps): {err}, u of max|u| {u_rel:.2e}, "
              f"FP32-stored twin {du_floor:.2e} (ratio {du / du_floor:.2f})")
        assert dg.step == steps[i] and dg.error_flags == 0
        assert max(err.values()) < TOL, (c.name, err)
        assert du <= U_FLOOR_FACTOR * du_floor, (c.name, du, du_floor)
        assert dg.mass == pytest.approx(do["mass"], rel=1e-6)
        assert dg.rho_ave == pytest.approx(do["rho_ave"], rel=1e-6)
        assert len(b.flux_history(i)) == steps[i]


def test_pool_400x400_1000_steps(coex):
    """The 400 x 400 pool (25-row heater at Ts + 0.1 Tc, five sites, convective
    top) to 1000 steps through the single-domain step."""
    from helpers import gpu_domain
    case = wl.pool()
    od, twin = oracle_pair(case, coex, 1000)
    gd = gpu_domain(case, coex)
    gd.step(1000)
    err, u_rel, du, du_floor = _errors(gd.read(), od, twin)
    print(f"pool 400x400, 1000 steps: {err}, u of max|u| {u_rel:.2e}, FP32-stored twin {du_floor:.2e} "
          f"(ratio {du / du_floor:.2f})")
    assert max(err.values()) < TOL, err
    assert du <= U_FLOOR_FACTOR * du_floor, (du, du_floor)
