"""Pins of three oracle functions that the conservation and steady-state pins
cannot see: the density dependence of the shear viscosity (Eq. 3 with the
kinematic viscosities of Section 3.1), the buoyancy force of Eq. (9) with its
lagged mean density, and the convective outlet of Section 4.2.

Each pin compares the oracle with something other than its own formula: the
viscous decay rate of a shear wave, a linear response recovered from two runs
that differ only in g, and the exact delay of the implicit upwind scheme for a
signal linear in time."""
import copy

import numpy as np
import pytest

from oracle import Domain, Params
from oracle.lattice import M_INV, m_eq


def _shear_wave(coex, rho_value, tau_l=0.8, tau_v=1.0, steps=(50, 550)):
    """Uniform density between two halfway bounce-back walls (rows 0 and ny-1
    solid, x periodic), EOS at Ts, no gravity and no wetting force, started from
    the equilibrium of u_x(y) = U0 sin(pi (y - 1/2) / H): the lowest no-slip
    shear mode.  Returns the kinematic viscosity measured from its decay."""
    nx, ny, W_ = 4, 34, 1
    H = ny - 1 - W_  # fluid rows; the walls sit half a cell outside them
    Ts = coex["Ts"]
    p = Params(nx=nx, ny=ny, wall_rows=W_, top_bc="wall", T_bottom=Ts, T_top=Ts, eos_T_fixed=True, Gw=0.0,
               g_y=0.0, rho_l=coex["rho_l"], rho_v=coex["rho_v"], tau_l=tau_l, tau_v=tau_v)
    rho0 = np.full((ny, nx), rho_value)
    d = Domain(p, rho0, np.full((ny, nx), Ts))
    y = np.arange(ny, dtype=np.float64)
    shape = np.sin(np.pi * (y - (W_ - 0.5)) / H)
    ux0 = 1e-4 * shape[:, None] * np.ones((1, nx))
    feq = np.einsum("ij,jyx->iyx", M_INV, m_eq(rho0, ux0, np.zeros_like(ux0)))
    d.fs = np.where(d.fluid[None], feq, 0.0)
    fl_rows = slice(W_, ny - 1)
    amps = []
    n_done = 0
    for n in steps:
        d.step(n - n_done)
        n_done = n
        u = d.ux[fl_rows, 0]
        s = shape[fl_rows]
        amps.append(float(u @ s / (s @ s)))
        assert np.allclose(d.ux[fl_rows], d.ux[fl_rows, :1])  # stays uniform in x
    k = np.pi / H
    return -np.log(amps[1] / amps[0]) / (k * k * (steps[1] - steps[0]))


@pytest.mark.parametrize("phase", ["liquid", "vapour"])
def test_shear_viscosity_follows_the_density(coex, paper, phase):
    """Section 3.1 gives nu_l = 0.1 and nu_v = 0.5/3; with nu = (tau - 1/2)/3
    (Eq. 3, dt = 1) the shear mode of uniform liquid must decay at nu_l and that
    of uniform vapour at nu_v.  Taking tau_v = tau_l, dropping the density
    dependence, or a wrong nu(tau) relation moves one of them by 40% or more."""
    rho = coex["rho_l"] if phase == "liquid" else coex["rho_v"]
    nu = _shear_wave(coex, rho)
    expect = paper["nu_l"]["value"] if phase == "liquid" else paper["nu_v"]["value"]
    print(f"{phase}: measured nu {nu:.5f}, expected {expect:.5f}")
    assert nu == pytest.approx(expect, rel=0.02)


def _open_film(coex, g_y):
    """A film that reaches the constant-density top, so that mass leaves the
    domain and the mean density changes from step to step."""
    nx, ny, W_ = 8, 16, 2
    Ts = coex["Ts"]
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    x = np.ones((ny, 1)) * np.arange(nx, dtype=np.float64)[None, :]
    rho0 = coex["rho_v"] + (coex["rho_l"] - coex["rho_v"]) * 0.5 * (1.0 - np.tanh((y - 11.0 - np.sin(x)) / 2.0))
    p = Params(nx=nx, ny=ny, wall_rows=W_, top_bc="const_rho", T_bottom=Ts + 0.05 * coex["Tc"], g_y=g_y, Gw=0.3,
               rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    T0 = np.where(y < W_, p.T_bottom, Ts)
    return Domain(p, rho0, T0)


def test_buoyancy_is_linear_in_density_with_the_lagged_mean(coex):
    """Eq. (9): F_b = (rho - rho_ave) g, with rho_ave the fluid mean of the
    previous step.  Two copies of one domain take step 2 with g and with
    g + dg: their pre-collision populations, densities, psi and the other
    forces are identical, and u = (sum e f + F/2) / rho (Eq. 5), so
    2 rho du_y / dg = rho - rho_ave exactly.  Regressed over all fluid cells,
    the slope must be 1 (the sign and size of the force) and the intercept the
    mean density of step 1, not that of step 2 (mass leaves through the open
    top, so the two differ)."""
    g, dg = -3e-5, -1e-4
    base = _open_film(coex, g).step(1)
    rho_ave_1 = base.diag()["rho_ave"]
    a, b = copy.deepcopy(base), copy.deepcopy(base)
    b.p.g_y = g + dg
    a.step(1)
    b.step(1)
    fl = a.fluid
    assert np.array_equal(a.rho, b.rho)
    rho = a.rho[fl]
    lhs = 2.0 * rho * (b.uy[fl] - a.uy[fl]) / dg
    slope, icept = np.polyfit(rho, lhs, 1)
    rho_ave_2 = a.diag()["rho_ave"]
    print(f"slope {slope:.12f}, intercept {-icept:.12f}; rho_ave step 1 {rho_ave_1:.12f}, step 2 {rho_ave_2:.12f}")
    assert abs(rho_ave_2 - rho_ave_1) > 1e-6 * rho_ave_1
    assert slope == pytest.approx(1.0, abs=1e-9)
    assert -icept == pytest.approx(rho_ave_1, abs=1e-9 * rho_ave_1)
    assert np.abs(lhs - (rho - rho_ave_1)).max() < 1e-9 * rho_ave_1
    np.testing.assert_array_equal(b.ux[fl], a.ux[fl])  # gravity acts along y only


def _convective_pool(coex):
    nx, ny, W_ = 12, 24, 3
    Ts, Tc = coex["Ts"], coex["Tc"]
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    x = np.ones((ny, 1)) * np.arange(nx, dtype=np.float64)[None, :]
    # a liquid film with a wavy surface under vapour: the flow near the top is not uniform
    rho0 = coex["rho_v"] + (coex["rho_l"] - coex["rho_v"]) * 0.5 * (1.0 - np.tanh((y - 12.0 - 2.0 * np.sin(2 * np.pi * x / nx)) / 2.0))
    p = Params(nx=nx, ny=ny, wall_rows=W_, top_bc="convective", T_bottom=Ts + 0.12 * Tc, g_y=-3e-4, Gw=0.3,
               rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    return Domain(p, rho0, np.where(y < W_, p.T_bottom, Ts))


def test_convective_outlet_uses_the_lagged_mean_velocity(coex):
    """Section 4.2's outlet, phi_t + U phi_y = 0, as the implicit upwind update
    f_i(top, n) (1 + U) = f_i(top, n-1) + U f_i(top-1, n) of the three populations
    entering the top row.  The U of step n is recovered from every entering
    population of every column, from the stored post-collision populations
    and outlet memory alone; all must give one number, equal to the positive
    part of the mean u_y of row ny - 2 reported by step n - 1 (a rule with U
    and 1 swapped, without the 1 + U, or with the current step's velocity
    gives column-dependent or different values)."""
    d = _convective_pool(coex).step(40)
    checked = 0
    for _ in range(6):
        u_prev = d.diag()["u_top"]
        ny = d.p.ny
        fs = d.fs.copy()
        prev = d.f_top_prev.copy()
        d.step(1)
        top = d.f_top_prev  # the entering populations of the top row at this step
        # pulled values of row ny - 2 at this step: f_i(x, ny - 2) = f*_i(x - e_i, ny - 1)
        below = np.stack([fs[4, ny - 1, :], np.roll(fs[7, ny - 1, :], -1), np.roll(fs[8, ny - 1, :], 1)])
        mask = np.abs(top - below) > 1e-6 * np.abs(below).max()
        U = (prev - top)[mask] / (top - below)[mask]
        expect = max(0.0, u_prev)
        if expect > 0:
            assert U.size > 10
            np.testing.assert_allclose(U, expect, rtol=1e-7, atol=1e-13)
            checked += 1
    assert checked >= 3


def test_implicit_upwind_outlet_delays_a_linear_signal_by_one_over_U(coex):
    """The same outlet on a signal arriving from below that grows linearly in
    time: phi_t + U phi_y = 0 carries it up by one lattice spacing in 1/U
    steps, and its implicit upwind discretisation reproduces that delay
    exactly once the start-up transient (a factor 1/(1 + U) per step) has
    decayed: phi_top^n = phi_below^n - b / U for phi_below^n = a + b n.  The
    oracle's streaming pass is driven with a fixed U and the post-collision
    populations of the top row set to that signal."""
    d = _convective_pool(coex)
    ny = d.p.ny
    U, a, b = 0.25, 0.02, 1e-3
    for n in range(1, 201):
        d.U = U
        d.fs[4, ny - 1, :] = a + b * n  # pulled into row ny - 2 at this step (e_4 = (0, -1))
        f = d._stream()
        below, top = f[4, ny - 2, :], f[4, ny - 1, :]
    np.testing.assert_allclose(below, a + b * 200, rtol=0, atol=1e-15)
    np.testing.assert_allclose(top, below - b / U, rtol=0, atol=1e-12)
