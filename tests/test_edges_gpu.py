"""Degenerate and ragged lattices against the FP64 oracle, in every compiled
kernel variant: the smallest lattices the library accepts (4 x 6 and a few
more, narrower than one frame halo so that the periodic x fold wraps more than
once), and a lattice whose last tile is one column wide and whose last tile
row is one row high.  Fields carry seeded noise so that an error in the x fold
or at a tile seam shows up (an x-uniform field would hide both).  Tolerance:
the parity bar of the other parity tests (1e-5 relative L-infinity; u in units
of the lattice sound speed)."""
import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, gpu_domain, oracle_domain, rel_linf

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


def _case(name, nx, ny, wall_rows, top_bc, sites=()):
    return wl.Case(name, nx=nx, ny=ny, wall_rows=wall_rows, top_bc=top_bc, T_bottom_over_Tc=wl.TS_OVER_TC + 0.1,
                   T_top_over_Tc=wl.TS_OVER_TC if top_bc == "wall" else None, eos_T_fixed=False, g_y=-3e-5,
                   Gw0=0.3, sites=list(sites))


def _fields(case, coex, seed):
    """A liquid layer under vapour with 2% density noise, and layered T with noise."""
    rng = np.random.default_rng(seed)
    fluid = case.ny - case.wall_rows - (1 if case.top_bc == "wall" else 0)
    rho = wl.tanh_film(case.ny, case.nx, coex["rho_l"], coex["rho_v"], case.wall_rows + 0.5 * fluid, width=2.0)
    rho = rho * (1.0 + 0.02 * rng.standard_normal(rho.shape))
    Ts = wl.TS_OVER_TC * coex["Tc"]
    T = wl.layered_T(case.ny, case.nx, case.wall_rows, case.T_bottom(coex["Tc"]), Ts)
    T[case.wall_rows:] += 1e-3 * coex["Tc"] * rng.standard_normal((case.ny - case.wall_rows, case.nx))
    return rho, T


def _errors(gd, od):
    rho_o, ux_o, uy_o, T_o = od.fields()
    rho_g, ux_g, uy_g, T_g = [t.cpu().numpy() for t in gd.read()]
    fl = od.fluid
    assert np.isfinite(rho_o).all() and np.isfinite(T_o).all()
    du = max(np.abs(ux_g - ux_o)[fl].max(), np.abs(uy_g - uy_o)[fl].max())
    umax = float(np.sqrt(ux_o ** 2 + uy_o ** 2)[fl].max())
    print(f"  u relative to max|u| {du / umax:.2e} (max|u| {umax:.2e})")
    return dict(rho=rel_linf(rho_g, rho_o, fl), u=float(du / CS), T=rel_linf(T_g, T_o))


def _variants():
    from paper_1812_10375_gb300 import hlb
    return list(range(len(hlb.tile_variants())))


TINY = [
    _case("tiny_4x6_wall", 4, 6, 1, "wall"),
    _case("tiny_5x7_const_rho", 5, 7, 1, "const_rho"),
    _case("tiny_7x9_convective", 7, 9, 2, "convective", sites=[(3.0, 3.0, -0.3)]),
]


@pytest.mark.parametrize("case", TINY, ids=[c.name for c in TINY])
def test_smallest_lattices_in_every_variant(coex, case):
    rho0, T0 = _fields(case, coex, seed=case.nx)
    steps = 200
    od = oracle_domain(case, coex, rho0=rho0, T0=T0).step(steps)
    for v in _variants():
        gd = gpu_domain(case, coex, rho0=rho0, T0=T0)
        gd.set_tile_variant(v)
        gd.step(steps)
        err = _errors(gd, od)
        print(case.name, "variant", v, err)
        assert max(err.values()) < TOL, (v, err)
        dg, do = gd.diag(), od.diag()
        assert dg.step == steps
        assert dg.mass == pytest.approx(do["mass"], rel=TOL)


def test_one_column_and_one_row_tails_in_every_variant(coex):
    """nx = 53: tiles of 52 columns leave a one-column tile; ny = 57 leaves a
    one-row tile row for 28-row tiles (and 9 or 17 rows for the others)."""
    case = _case("tails_53x57", 53, 57, 6, "convective", sites=[(10.0, 6.0, -0.3), (40.0, 6.0, -0.6)])
    rho0, T0 = _fields(case, coex, seed=53)
    steps = 120
    od = oracle_domain(case, coex, rho0=rho0, T0=T0).step(steps)
    for v in _variants():
        gd = gpu_domain(case, coex, rho0=rho0, T0=T0)
        gd.set_tile_variant(v)
        gd.step(steps)
        err = _errors(gd, od)
        print(case.name, "variant", v, err)
        assert max(err.values()) < TOL, (v, err)


def test_all_liquid_and_all_vapour_boxes(coex):
    """No interface at all: the closed box keeps its mass to FP32 summation
    rounding and matches the oracle; the uniform vapour box heated from below
    stays single-phase."""
    for name, rho_fill in (("liquid_box", coex["rho_l"]), ("vapour_box", coex["rho_v"])):
        case = _case(name, 40, 30, 3, "wall")
        rng = np.random.default_rng(7)
        rho0 = np.full((case.ny, case.nx), rho_fill) * (1.0 + 1e-3 * rng.standard_normal((case.ny, case.nx)))
        _, T0 = _fields(case, coex, seed=7)
        od = oracle_domain(case, coex, rho0=rho0, T0=T0).step(150)
        gd = gpu_domain(case, coex, rho0=rho0, T0=T0)
        gd.step(150)
        err = _errors(gd, od)
        print(name, err)
        assert max(err.values()) < TOL, err
        dg = gd.diag()
        fluid = slice(case.wall_rows, case.ny - 1)
        # the library starts from the FP32 rounding of rho0
        assert dg.mass == pytest.approx(rho0[fluid].astype(np.float32).astype(np.float64).sum(), rel=1e-6)
        rho = gd.read()[0].cpu().numpy()[fluid]
        mid = 0.5 * (coex["rho_l"] + coex["rho_v"])
        assert (rho > mid).all() if rho_fill > mid else (rho < mid).all()
