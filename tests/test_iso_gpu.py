"""The isotropic central diffusion scheme of Eqs. (20)-(21) on the GPU (the
scheme the paper compares its finite-volume faces against, Section 3.2):
element-by-element parity with the FP64 oracle's isotropic option, and the
paper's contrast at steady state: across a flat liquid-vapour interface
between two Dirichlet walls the finite-volume scheme's wall heat fluxes agree
while the isotropic scheme's differ by the amount the oracle's exact discrete
steady state gives."""
import dataclasses

import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, gpu_domain, oracle_domain, ragged_case, rel_linf
from test_oracle_physics import _steady_wall_flux_difference

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


@pytest.mark.parametrize("name,steps", [("flat", 1000), ("ragged", 300)])
def test_iso_scheme_matches_oracle(coex, name, steps):
    from paper_1812_10375_gb300 import hlb
    case = wl.flat_interface() if name == "flat" else ragged_case(3)
    od = oracle_domain(case, coex, diffusion="iso")
    gd = gpu_domain(case, coex, diffusion=hlb.HLB_DIFF_ISO)
    od.step(steps)
    gd.step(steps)
    rho_o, ux_o, uy_o, T_o = od.fields()
    rho_g, ux_g, uy_g, T_g = [t.cpu().numpy() for t in gd.read()]
    fl = od.fluid
    e_rho = rel_linf(rho_g, rho_o, fl)
    e_T = rel_linf(T_g, T_o)
    e_u = max(np.abs(ux_g - ux_o)[fl].max(), np.abs(uy_g - uy_o)[fl].max()) / CS
    print(f"iso {name}: rel err rho {e_rho:.2e} u {e_u:.2e} T {e_T:.2e}")
    assert max(e_rho, e_T, e_u) <= TOL


def test_iso_is_rejected_by_batches_and_row_marching(coex):
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    p, _ = params_for(ragged_case(3), rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    p.diffusion = hlb.HLB_DIFF_ISO
    assert hlb.lib().hlb_batch_workspace_bytes(1, hlb.C.byref(p)) == 0
    d = gpu_domain(ragged_case(3), coex, diffusion=hlb.HLB_DIFF_ISO)
    marches = [k for k, (w, h, t) in enumerate(hlb.tile_variants()) if w == 0]
    with pytest.raises(hlb.HlbError):
        d.set_tile_variant(marches[0])


def test_paper_contrast_on_gpu(coex):
    """Section 3.2 on the GPU: 4 x 120, liquid in the lower half and vapour in
    the upper half, walls at T = 1 and T = 0 conducting like the phase next to
    them, EOS at Ts, no gravity, run to steady state (300,000 steps, about 20
    diffusion times).  Relative wall-flux difference 2 |q_h - q_l| / (q_h + q_l):
    isotropic within 10% of the oracle's exact discrete steady state of the same
    scheme on the same density profile (about 0.18, as the paper prints), and
    finite volume below 5% of that."""
    from paper_1812_10375_gb300 import hlb
    ny, nx = 120, 4
    case = dataclasses.replace(wl.flat_interface(), name="contrast", ny=ny)
    rho0 = wl.tanh_film(ny, nx, coex["rho_l"], coex["rho_v"], ny / 2.0)
    T0 = np.full((ny, nx), 0.5)
    lam_l, lam_v = coex["rho_l"] * 6.0 * 0.1, coex["rho_v"] * 6.0 * 0.1
    out = {}
    for scheme in (hlb.HLB_DIFF_FV, hlb.HLB_DIFF_ISO):
        d = gpu_domain(case, coex, rho0=rho0, T0=T0, diffusion=scheme, lambda_w=lam_l, lambda_top=lam_v)
        d.step(300000)
        g = d.diag()
        assert g.error_flags == 0
        out[scheme] = 2.0 * abs(g.q_bottom - g.q_top) / (g.q_bottom + g.q_top)
        rho_end = d.read()[0].cpu().numpy().astype(np.float64)
    # the exact steady state of the oracle's isotropic scheme on the interface
    # profile the GPU run relaxed to (the flow is at rest up to spurious currents)
    rho_end[0], rho_end[-1] = rho_end[1], rho_end[-2]
    exact_iso = _steady_wall_flux_difference(coex, "iso", rho0=rho_end)
    print(f"GPU steady wall-flux difference: FV {out[hlb.HLB_DIFF_FV]:.2e}, isotropic {out[hlb.HLB_DIFF_ISO]:.4f} "
          f"(oracle exact {exact_iso:.4f})")
    # the full model keeps small volumetric terms (pressure work on spurious
    # currents) that the conduction-only solution leaves out, so the FV
    # difference is not zero here, but it is far below the isotropic scheme's
    assert out[hlb.HLB_DIFF_FV] < 0.05 * out[hlb.HLB_DIFF_ISO]
    assert out[hlb.HLB_DIFF_ISO] == pytest.approx(exact_iso, rel=0.1)
