"""Energy sub-steps (Eq. 27, N > 1) on the GPU against the FP64 oracle: the
fused kernel takes the first RK4 sub-step of dt/N, k_energy_substep the other
N - 1 on the step's rho^n and u^n.  Parity on fields and diagnostics for the
convective-top box with sites (N = 2 and 3: the last sub-step lands in either
buffer), a closed box heated by an imposed flux (N = 4), and a heater whose
diffusivity lambda_w / (rho_w c_w) = 0.5 is beyond RK4's bound at N = 1 (0.35
for the five-point operator): N = 1 sets the error word, N = 2 matches the
oracle (the stability use of Eq. 27 in Section 2.2).  Tolerances as in the
other parity tests."""
import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, gpu_domain, oracle_domain, ragged_case, rel_linf

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


def _run(case, coex, steps, rho0=None, T0=None, oracle_kw=None, gpu_kw=None):
    od = oracle_domain(case, coex, rho0=rho0, T0=T0, **(oracle_kw or {})).step(steps)
    gd = gpu_domain(case, coex, rho0=rho0, T0=T0, **(gpu_kw or {}))
    gd.step(steps)
    rho_o, ux_o, uy_o, T_o = od.fields()
    rho_g, ux_g, uy_g, T_g = [t.cpu().numpy() for t in gd.read()]
    fl = od.fluid
    du = max(np.abs(ux_g - ux_o)[fl].max(), np.abs(uy_g - uy_o)[fl].max())
    err = dict(rho=rel_linf(rho_g, rho_o, fl), u=float(du / CS), T=rel_linf(T_g, T_o))
    return err, gd, od


def _flux_tol(lam, T):
    """A face flux differences two FP32 temperatures: |dq| <= 2 lambda 1e-5 max|T|."""
    return 2.0 * lam * TOL * float(np.abs(T).max())


@pytest.mark.parametrize("N", [2, 3])
def test_substeps_match_oracle(coex, N):
    case = ragged_case(3)
    err, gd, od = _run(case, coex, 300, oracle_kw=dict(n_sub=N), gpu_kw=dict(n_sub=N))
    dg, do = gd.diag(), od.diag()
    print(f"N={N}", err, "energy", dg.energy, do["energy"], "q_i", dg.q_interface, do["q_interface"])
    assert max(err.values()) < TOL, err
    assert dg.step == 300 and dg.error_flags == 0
    assert dg.energy == pytest.approx(do["energy"], rel=TOL)
    lam_w = 3.0 * coex["rho_l"] * 6.0 * 0.1
    assert dg.q_interface == pytest.approx(do["q_interface"], abs=_flux_tol(lam_w, od.T))
    assert dg.q_bottom == pytest.approx(do["q_bottom"], abs=_flux_tol(lam_w, od.T))
    assert dg.q_bottom_timeavg == pytest.approx(do["q_bottom_timeavg"], abs=_flux_tol(lam_w, od.T))


def test_substeps_top_wall_and_flux_heater(coex):
    """A closed box (top wall) under an imposed flux: every wall flux and the
    energy sum pass through the sub-step kernels' partials."""
    from paper_1812_10375_gb300 import hlb
    case = wl.Case("closed_flux", nx=40, ny=36, wall_rows=4, top_bc="wall", T_bottom_over_Tc=wl.TS_OVER_TC,
                   T_top_over_Tc=wl.TS_OVER_TC - 0.02, eos_T_fixed=False, g_y=-3e-5, Gw0=0.3,
                   sites=[(20.0, 8.0, -0.3)])
    rng = np.random.default_rng(36)
    rho0 = wl.tanh_film(case.ny, case.nx, coex["rho_l"], coex["rho_v"], 20.0, width=3.0)
    rho0 = rho0 * (1.0 + 0.01 * rng.standard_normal(rho0.shape))
    T0 = np.full((case.ny, case.nx), wl.TS_OVER_TC * coex["Tc"])
    q = 2e-4
    err, gd, od = _run(case, coex, 300, rho0, T0,
                       oracle_kw=dict(n_sub=4, bottom_bc="flux", q_in=q),
                       gpu_kw=dict(n_sub=4, bottom_bc=hlb.HLB_BOTTOM_FLUX, q_in=q))
    dg, do = gd.diag(), od.diag()
    print("closed flux N=4", err, dg.q_top, do["q_top"], dg.q_bottom, do["q_bottom"])
    assert max(err.values()) < TOL, err
    lam_w = 3.0 * coex["rho_l"] * 6.0 * 0.1
    tol = _flux_tol(lam_w, od.T)
    for k in ("q_bottom", "q_top", "q_interface"):
        assert getattr(dg, k) == pytest.approx(do[k], abs=tol), k
    assert dg.energy == pytest.approx(do["energy"], rel=TOL)


def test_conductive_heater_needs_substeps(coex):
    case = ragged_case(3)
    lam_w = 0.5 * 3.0 * coex["rho_l"] * 6.0  # diffusivity 0.5 in the 3 rho_l, c_v heater
    d1 = gpu_domain(case, coex, lambda_w=lam_w, n_sub=1)
    d1.step(60)
    assert d1.diag(check_flags=False).error_flags != 0
    err, gd, od = _run(case, coex, 300, oracle_kw=dict(lambda_w=lam_w, n_sub=2),
                       gpu_kw=dict(lambda_w=lam_w, n_sub=2))
    print("conductive heater N=2", err)
    assert max(err.values()) < TOL, err
    assert gd.diag().error_flags == 0


def test_graph_replay_matches_single_launches_with_substeps(coex):
    case = ragged_case(3)
    a = gpu_domain(case, coex, n_sub=2)
    b = gpu_domain(case, coex, n_sub=2)
    a.step(37)
    for _ in range(37):
        b.step(1)
    for x, y in zip(a.read(), b.read()):
        assert (x == y).all()
    assert a.diag().energy == b.diag().energy


def test_n_sub_zero_picks_a_stable_n(coex):
    """n_sub = 0 takes N from the stability bound: 4 for a heater of
    diffusivity 0.65, and the run matches the oracle at that N."""
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    case = ragged_case(3)
    lam_w = 0.65 * 3.0 * coex["rho_l"] * 6.0
    p, _ = params_for(case, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    p.lambda_w = lam_w
    assert hlb.stable_substeps(p) == 4
    err, gd, od = _run(case, coex, 300, oracle_kw=dict(lambda_w=lam_w, n_sub=4),
                       gpu_kw=dict(lambda_w=lam_w, n_sub=0))
    print("n_sub=0 -> 4", err)
    assert max(err.values()) < TOL, err
    assert gd.diag().error_flags == 0
