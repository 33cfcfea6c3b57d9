"""The row-marching step kernel (one CTA per full-width segment of rows) against
the tiled step kernel on the same domains: the two evaluate every cell's update
with the same arithmetic, so their fields agree to FP32 rounding, over segment
heights that split each lattice into several segments with a ragged last one
and over all three top boundaries.  Both kernels are also checked against the
FP64 oracle by the parity tests; both are selectable variants beside the
default split step."""
import dataclasses

import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, gpu_domain, ragged_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def coex():
    return coexistence()


def _variants():
    from paper_1812_10375_gb300 import hlb
    kinds = hlb.variant_kinds()
    # the fused tile kernels evaluate each cell with the row-marching kernel's
    # arithmetic; the split step's coefficient form rounds differently
    tiles = [k for k, kind in enumerate(kinds) if kind == hlb.HLB_KIND_FUSED]
    marches = [k for k, kind in enumerate(kinds) if kind == hlb.HLB_KIND_MARCH]
    return tiles, marches


CASES = {
    "ragged": lambda: ragged_case(3),                      # 45 x 37, convective top, sites, gravity
    "flat": lambda: wl.flat_interface(),                   # 4 x 200, top wall (Dirichlet rows 0 and 199)
    "film": lambda: wl.film(nx=200, ny=100),              # constant-density top, 20-row wall
    "pool": lambda: wl.pool(nx=96, ny=130, n_sites=3, heater_rows=10),
    "wide": lambda: dataclasses.replace(ragged_case(7), name="wide", nx=500, ny=75),
}


@pytest.mark.parametrize("name", list(CASES))
def test_march_matches_tile_kernel(coex, name):
    case = CASES[name]()
    tiles, marches = _variants()
    assert marches, "no row-marching variant compiled"
    ref = gpu_domain(case, coex)
    ref.set_tile_variant(tiles[0])
    ref.step(60)
    r_ref = [t.cpu().numpy() for t in ref.read()]
    d_ref = ref.diag()
    for v in marches:
        d = gpu_domain(case, coex)
        d.set_tile_variant(v)
        d.step(60)
        r = [t.cpu().numpy() for t in d.read()]
        # rho and T to 1e-6 of their maxima; u to 1e-6 in lattice units (2e-6
        # of the sound speed, a fifth of the parity tolerance against the oracle)
        for k, (x, y) in enumerate(zip(r, r_ref)):
            err = np.abs(x.astype(np.float64) - y).max()
            tol = 1e-6 if k in (1, 2) else 1e-6 * max(np.abs(y).max(), 1e-30)
            assert err <= tol, (name, v, "rho ux uy T".split()[k], err)
        dg = d.diag()
        assert dg.step == d_ref.step == 60
        assert dg.error_flags == 0
        for key in ("mass", "energy", "rho_ave"):
            a, b = getattr(dg, key), getattr(d_ref, key)
            assert abs(a - b) <= 1e-7 * abs(b), (name, v, key, a, b)
        for key in ("q_bottom", "q_interface", "u_top"):
            a, b = getattr(dg, key), getattr(d_ref, key)
            assert abs(a - b) <= 1e-5 * max(abs(b), 1e-12), (name, v, key, a, b)


def test_march_batch_groups_by_width(coex):
    """A batch of domains of four row strides runs one launch per stride on
    forked streams; each domain matches its own single-domain run bit for bit."""
    cases = [ragged_case(3), wl.film(nx=40, ny=60), dataclasses.replace(ragged_case(5), name="r70", nx=70, ny=50),
             wl.pool(nx=130, ny=64, n_sites=3, heater_rows=10), wl.pool(nx=200, ny=90, n_sites=2, heater_rows=8)]
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    plist = [params_for(c, rho_l=coex["rho_l"], rho_v=coex["rho_v"])[0] for c in cases]
    b = hlb.Batch(plist)
    for i, c in enumerate(cases):
        rho0, T0 = wl.initial_fields(c, coex["rho_l"], coex["rho_v"], coex["Tc"])
        b.set_fields(i, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                     torch.tensor(T0, dtype=torch.float32, device="cuda"))
        b.set_nucleation_sites(i, c.sites)
    _, marches = _variants()
    for v in marches:
        b.set_tile_variant(v)
        b.step(17)  # one captured 16-step graph + one direct launch
    n = 17 * len(marches)
    for i, c in enumerate(cases):
        d = gpu_domain(c, coex)
        for v in marches:
            d.set_tile_variant(v)
            d.step(17)
        for x, y in zip(b.read(i), d.read()):
            assert (x == y).all(), c.name
        assert b.diag(i).step == n
        assert b.diag(i).q_bottom == d.diag().q_bottom
