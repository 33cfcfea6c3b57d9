"""Pins of the oracle's thermodynamics (Section 3.1, Eqs. 7, 14, 28) against facts
that do not come from the oracle itself: Peng-Robinson's critical point, the
paper's printed coexistence densities and latent heat, the Clausius-Clapeyron
relation and finite differences."""
import numpy as np
import pytest

from oracle import eos


def fd(fun, x, h):
    return (fun(x + h) - fun(x - h)) / (2.0 * h)


def test_critical_point_is_the_inflection_with_pr_compressibility(pr):
    """At T = Tc, dp/drho has a double zero at rho_c and Z_c = p_c/(rho_c R T_c) = 0.3074
    (the textbook Peng-Robinson critical compressibility)."""
    Tc = pr.Tc
    rho = np.linspace(0.5, 5.0, 200001)
    slope = fd(lambda r: eos.pressure(r, Tc, pr), rho, 1e-5)
    i = int(np.argmin(slope))
    rho_c = rho[i]
    # 0.45724 and 0.0778 are rounded constants, so the double zero is approximate
    assert abs(slope[i]) < 1e-3 * pr.R * Tc
    Zc = eos.pressure(rho_c, Tc, pr) / (rho_c * pr.R * Tc)
    assert Zc == pytest.approx(0.30740, abs=2e-4)
    assert eos.pressure(rho_c, Tc, pr) == pytest.approx(pr.pc, rel=2e-4)
    # just above Tc there is no two-phase region; just below there is
    with pytest.raises(ValueError):
        eos.spinodals(1.001 * Tc, pr)
    eos.spinodals(0.999 * Tc, pr)


def test_coexistence_matches_paper_and_equal_area(pr, coex, paper):
    """Section 3.1: rho_l ~ 6.5 and rho_v ~ 0.38 at 0.86 Tc.  Equal pressure, and the
    equal-area rule re-checked with an independent trapezoid quadrature in v."""
    Ts, rl, rv, ps = coex["Ts"], coex["rho_l"], coex["rho_v"], coex["ps"]
    pl, pv_ = paper["rho_l_at_0.86Tc"], paper["rho_v_at_0.86Tc"]
    assert rl == pytest.approx(pl["value"], abs=pl["abs_tol"])
    assert rv == pytest.approx(pv_["value"], abs=pv_["abs_tol"])
    assert eos.pressure(rl, Ts, pr) == pytest.approx(ps, abs=1e-13)
    assert eos.pressure(rv, Ts, pr) == pytest.approx(ps, abs=1e-13)
    v = np.linspace(1.0 / rl, 1.0 / rv, 2_000_001)
    pv = eos.pressure(1.0 / v, Ts, pr)
    area = np.sum(0.5 * (pv[1:] + pv[:-1]) * np.diff(v))
    assert area == pytest.approx(ps * (1.0 / rv - 1.0 / rl), rel=1e-9)


def test_latent_heat_clausius_clapeyron_and_paper(pr, coex, paper):
    """Eq. (14) must equal T (v_v - v_l) dp_s/dT (Clausius-Clapeyron), and the paper
    quotes h_fg ~ 0.58 (Section 3.3)."""
    Ts = coex["Ts"]
    h = eos.latent_heat(Ts, pr, coex["rho_l"], coex["rho_v"])
    dT = 1e-5 * pr.Tc
    p_hi = eos.coexistence(Ts + dT, pr)[2]
    p_lo = eos.coexistence(Ts - dT, pr)[2]
    h_cc = Ts * (1.0 / coex["rho_v"] - 1.0 / coex["rho_l"]) * (p_hi - p_lo) / (2.0 * dT)
    assert h == pytest.approx(h_cc, rel=1e-6)
    g = paper["h_fg_at_0.86Tc"]
    assert h == pytest.approx(g["value"], rel=g["rel_tol"])


@pytest.mark.parametrize("rho,Tr", [(0.38, 0.86), (6.5, 0.86), (3.0, 1.1), (1.0, 0.5), (5.0, 4.0)])
def test_T_dp_dT_matches_finite_difference(pr, rho, Tr):
    T = Tr * pr.Tc
    num = T * fd(lambda t: eos.pressure(rho, t, pr), T, 1e-6 * T)
    assert eos.T_dp_dT(rho, T, pr) == pytest.approx(num, rel=1e-7)


def test_T_dp_dT_finite_at_zero_temperature(pr):
    assert np.isfinite(eos.T_dp_dT(2.0, 0.0, pr))
    assert eos.T_dp_dT(2.0, 0.0, pr) == 0.0


def test_psi_from_eq7(pr, coex):
    """Eq. (7) with c = 1, G = -1: p = rho/3 - psi^2/2 must give back the EOS pressure."""
    Ts = coex["Ts"]
    rho = np.linspace(0.05, 7.5, 50)
    psi = eos.psi(rho, Ts, pr)
    assert np.all(psi > 0)
    np.testing.assert_allclose(rho / 3.0 - 0.5 * psi ** 2, eos.pressure(rho, Ts, pr), rtol=1e-12, atol=1e-14)


def test_psi_real_over_the_sweep_range(pr):
    """psi^2 > 0 for rho in (0, 8] up to 1.16 Tc (the hottest wall of the sweep);
    it turns negative by 1.3 Tc, where the device flags the cell."""
    rho = np.linspace(1e-3, 8.0, 4000)
    for Tr in (0.5, 0.86, 1.0, 1.16):
        assert eos.psi_squared(rho, Tr * pr.Tc, pr).min() > 0
    assert eos.psi_squared(rho, 1.3 * pr.Tc, pr).min() < 0
