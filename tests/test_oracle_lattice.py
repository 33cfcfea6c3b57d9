"""Pins of the oracle's D2Q9 MRT collision and streaming (Section 2.1, Eqs. 1-5, 8)
against textbook forms that do not appear in the oracle: the second-order D2Q9
equilibrium, Guo's velocity-space forcing, the BGK limit of MRT, and brute-force
moment sums on a 4 x 4 lattice."""
import numpy as np
import pytest

from oracle import Domain, Params
from oracle.lattice import E, EX, EY, M, M_INV, OPP, W, forcing_moments, m_eq

rng = np.random.default_rng(7)


def textbook_feq(rho, ux, uy):
    eu = EX[:, None] * ux[None] + EY[:, None] * uy[None]
    u2 = ux * ux + uy * uy
    return W[:, None] * rho[None] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * u2[None])


def guo_forcing(ux, uy, Fx, Fy):
    eu = EX[:, None] * ux[None] + EY[:, None] * uy[None]
    cx = 3.0 * (EX[:, None] - ux[None]) + 9.0 * eu * EX[:, None]
    cy = 3.0 * (EY[:, None] - uy[None]) + 9.0 * eu * EY[:, None]
    return W[:, None] * (cx * Fx[None] + cy * Fy[None])


def test_moment_matrix_orthogonal_with_integer_norms():
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)), atol=0)
    assert np.array_equal(np.diag(G), [9, 36, 36, 6, 12, 6, 12, 4, 4])
    np.testing.assert_allclose(M_INV @ M, np.eye(9), atol=1e-15)


def test_eq4_is_moments_of_textbook_equilibrium():
    n = 64
    rho = rng.uniform(0.3, 7.0, n)
    ux, uy = rng.uniform(-0.1, 0.1, (2, n))
    np.testing.assert_allclose(M @ textbook_feq(rho, ux, uy), m_eq(rho, ux, uy), rtol=1e-13, atol=1e-14)


def test_eq8_at_sigma_zero_is_moments_of_guo_forcing():
    """With the last row read as ux Fy + uy Fx the printed S equals M F_Guo."""
    n = 64
    ux, uy = rng.uniform(-0.1, 0.1, (2, n))
    Fx, Fy = rng.uniform(-0.01, 0.01, (2, n))
    S = forcing_moments(ux, uy, Fx, Fy, np.zeros(n), 1.25, 1.25, 0.0, 12.0)
    np.testing.assert_allclose(M @ guo_forcing(ux, uy, Fx, Fy), S, rtol=1e-12, atol=1e-16)


def _domain(nx=4, ny=6, **kw):
    p = Params(nx=nx, ny=ny, wall_rows=1, top_bc="wall", T_bottom=0.05, T_top=0.05,
               eos_T_fixed=True, Gw=0.0, rho_l=6.5, rho_v=0.38, **kw)
    return Domain(p, np.full((ny, nx), 1.0), np.full((ny, nx), 0.05))


def _random_state(ny, nx):
    rho = rng.uniform(0.4, 6.5, (ny, nx))
    f = W[:, None, None] * rho[None] * (1.0 + rng.uniform(-0.2, 0.2, (9, ny, nx)))
    Fx, Fy = rng.uniform(-0.02, 0.02, (2, ny, nx))
    rho = f.sum(0)
    ux = (np.tensordot(EX, f, axes=1) + 0.5 * Fx) / rho
    uy = (np.tensordot(EY, f, axes=1) + 0.5 * Fy) / rho
    return f, rho, ux, uy, Fx, Fy


def test_mrt_reduces_to_bgk_with_guo_forcing():
    """All rates 1/tau and sigma = 0: Eq. (2) must equal BGK with Guo's forcing."""
    tau = 0.9
    d = _domain(s_rho=1 / tau, s_e=1 / tau, s_zeta=1 / tau, s_j=1 / tau, s_q=1 / tau,
                tau_l=tau, tau_v=tau, sigma=0.0)
    f, rho, ux, uy, Fx, Fy = _random_state(6, 4)
    psi = np.ones_like(rho)
    fs = d._collide(f, rho, ux, uy, Fx, Fy, Fx, Fy, psi)
    feq = textbook_feq(rho.ravel(), ux.ravel(), uy.ravel()).reshape(9, 6, 4)
    guo = guo_forcing(ux.ravel(), uy.ravel(), Fx.ravel(), Fy.ravel()).reshape(9, 6, 4)
    want = f - (f - feq) / tau + (1.0 - 0.5 / tau) * guo
    fl = d.fluid
    np.testing.assert_allclose(fs[:, fl], want[:, fl], rtol=1e-12, atol=1e-14)


def test_brute_force_moments_4x4():
    """Collision keeps mass and adds exactly F to the momentum (Eqs. 2, 5, 8)."""
    d = _domain()
    f, rho, ux, uy, Fx, Fy = _random_state(6, 4)
    psi = rng.uniform(0.4, 2.0, rho.shape)
    fs = d._collide(f, rho, ux, uy, Fx, Fy, 0.5 * Fx, 0.5 * Fy, psi)
    fl = d.fluid
    assert fl.sum() == 16
    for y in range(6):
        for x in range(4):
            if not fl[y, x]:
                continue
            assert sum(fs[i, y, x] for i in range(9)) == pytest.approx(sum(f[i, y, x] for i in range(9)), rel=1e-14)
            jx0 = sum(E[i, 0] * f[i, y, x] for i in range(9))
            jy0 = sum(E[i, 1] * f[i, y, x] for i in range(9))
            jx1 = sum(E[i, 0] * fs[i, y, x] for i in range(9))
            jy1 = sum(E[i, 1] * fs[i, y, x] for i in range(9))
            assert jx1 - jx0 == pytest.approx(Fx[y, x], abs=1e-14)
            assert jy1 - jy0 == pytest.approx(Fy[y, x], abs=1e-14)


def test_streaming_moves_populations_and_bounces_back():
    d = _domain(nx=5, ny=7)
    for i in range(1, 9):
        d.fs = np.zeros((9, 7, 5))
        d.fs[i, 3, 0] = 1.0
        f = d._stream()
        dest = (3 + E[i, 1], (0 + E[i, 0]) % 5)
        assert f[i][dest] == 1.0 and f.sum() == 1.0
    # a population heading into the bottom wall comes back reversed at the same node
    for i in (4, 7, 8):
        d.fs = np.zeros((9, 7, 5))
        d.fs[i, 1, 2] = 1.0
        f = d._stream()
        assert f[OPP[i], 1, 2] == 1.0 and f.sum() == 1.0
