"""Peng-Robinson thermodynamics for the oracle (plain FP64, test infrastructure).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import anything under ``oracle/``; the GPU library never does.

Everything here follows Section 3.1 of Hu & Liu, "Study of boiling heat
transfer on the wall with an improved hybrid lattice Boltzmann model"
(arXiv 1812.10375):

* Eq. (28): p = rho R T / (1 - b rho) - a phi(T) rho^2 / (1 + 2 b rho - b^2 rho^2)
  with a = 3/49, b = 2/21, R = 1.
* phi(T) = [1 + kappa (1 - sqrt(T/Tc))]^2,
  kappa = 0.37464 + 1.54226 w - 0.26992 w^2.  The square-root factor is printed
  garbled in Section 3.1 as sqrt(1 - T/Tc); that form has no two-phase region at
  0.86 Tc, so the standard Peng-Robinson form is used (it reproduces the printed
  coexistence densities 6.5 / 0.38).  The acentric factor w is not printed;
  w = 0.344 (water) reproduces those densities.
* Tc and pc from a = 0.45724 R^2 Tc^2 / pc and b = 0.0778 R Tc / pc.
* Eq. (7) with c = 1 and G = -1: p = rho/3 + G psi^2 / 2, hence
  psi = sqrt(2 (rho/3 - p)).
* Eq. (14): latent heat h = int_{v_l}^{v_v} T (dp/dT)_v dv.
* Maxwell's equal-area construction gives the coexistence densities
  (Section 3.1 quotes rho_l ~ 6.5 and rho_v ~ 0.38 at 0.86 Tc).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy import integrate, optimize


@dataclass(frozen=True)
class PR:
    """Peng-Robinson parameters (Section 3.1)."""

    a: float = 3.0 / 49.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    omega: float = 0.344

    @property
    def Tc(self) -> float:
        # a/b = (0.45724/0.0778) R Tc
        return (self.a / self.b) * (0.0778 / 0.45724) / self.R

    @property
    def pc(self) -> float:
        return 0.0778 * self.R * self.Tc / self.b

    @property
    def kappa(self) -> float:
        w = self.omega
        return 0.37464 + 1.54226 * w - 0.26992 * w * w


def alpha_factor(T, eos: PR):
    """1 + kappa (1 - sqrt(T/Tc)); phi(T) is its square.  T < 0 is clamped to 0."""
    Tr = np.maximum(np.asarray(T, dtype=np.float64), 0.0) / eos.Tc
    return 1.0 + eos.kappa * (1.0 - np.sqrt(Tr))


def phi(T, eos: PR):
    return alpha_factor(T, eos) ** 2


def pressure(rho, T, eos: PR):
    """Eq. (28)."""
    rho = np.asarray(rho, dtype=np.float64)
    rep = eos.R * T * rho / (1.0 - eos.b * rho)
    att = eos.a * phi(T, eos) * rho * rho / (1.0 + 2.0 * eos.b * rho - eos.b * eos.b * rho * rho)
    return rep - att


def dp_drho(rho, T, eos: PR):
    """(dp/drho)_T of Eq. (28), used only to bracket the spinodals."""
    rho = np.asarray(rho, dtype=np.float64)
    b = eos.b
    den = 1.0 + 2.0 * b * rho - b * b * rho * rho
    dden = 2.0 * b - 2.0 * b * b * rho
    rep = eos.R * T / (1.0 - b * rho) ** 2
    att = eos.a * phi(T, eos) * (2.0 * rho * den - rho * rho * dden) / (den * den)
    return rep - att


def T_dp_dT(rho, T, eos: PR):
    """T (dp/dT)_rho of Eq. (28), the factor of the latent-heat source of Eq. (17).

    d phi/dT = -kappa [1 + kappa (1 - sqrt(T/Tc))] / sqrt(T Tc), so
    T dp/dT = rho R T / (1 - b rho)
              + a rho^2 kappa [1 + kappa (1 - sqrt(Tr))] sqrt(Tr) / (1 + 2 b rho - b^2 rho^2),
    written with sqrt(Tr) so that it stays finite at T = 0.
    """
    rho = np.asarray(rho, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    sTr = np.sqrt(np.maximum(T, 0.0) / eos.Tc)
    rep = eos.R * T * rho / (1.0 - eos.b * rho)
    den = 1.0 + 2.0 * eos.b * rho - eos.b * eos.b * rho * rho
    att = eos.a * rho * rho * eos.kappa * (1.0 + eos.kappa * (1.0 - sTr)) * sTr / den
    return rep + att


def psi_squared(rho, T, eos: PR):
    """psi^2 = 2 (rho/3 - p_EOS): Eq. (7) with c = 1 and G = -1 (Section 3.1)."""
    return 2.0 * (np.asarray(rho, dtype=np.float64) / 3.0 - pressure(rho, T, eos))


def psi(rho, T, eos: PR):
    """Effective mass; a negative psi^2 (outside the EOS' valid range) gives psi = 0."""
    return np.sqrt(np.maximum(psi_squared(rho, T, eos), 0.0))


def spinodals(T, eos: PR):
    """The two densities where (dp/drho)_T = 0 (bracket for the coexistence roots)."""
    grid = np.linspace(1e-6, 0.999 / eos.b, 20001)
    d = dp_drho(grid, T, eos)
    idx = np.nonzero(np.sign(d[:-1]) != np.sign(d[1:]))[0]
    if len(idx) < 2:
        raise ValueError("no two-phase region at this temperature")
    r1 = optimize.brentq(lambda r: dp_drho(r, T, eos), grid[idx[0]], grid[idx[0] + 1], xtol=1e-15)
    r2 = optimize.brentq(lambda r: dp_drho(r, T, eos), grid[idx[1]], grid[idx[1] + 1], xtol=1e-15)
    return r1, r2


def coexistence(T, eos: PR):
    """Maxwell's equal-area construction in the p-v plane at temperature T.

    Finds p_s and rho_v < rho_l with p(rho_v) = p(rho_l) = p_s and
    int_{v_l}^{v_v} p dv = p_s (v_v - v_l), where v = 1/rho, i.e.
    int_{rho_v}^{rho_l} p(rho) / rho^2 drho = p_s (1/rho_v - 1/rho_l).
    Returns (rho_l, rho_v, p_s).
    """
    s1, s2 = spinodals(T, eos)
    p_hi = float(pressure(s1, T, eos))
    p_lo = max(float(pressure(s2, T, eos)), 1e-14)

    def roots(ps):
        # below rho = p_s / (2 R T) the pressure is below p_s (ideal-gas bound)
        r_min = 0.5 * ps / (eos.R * T)
        rv = optimize.brentq(lambda r: pressure(r, T, eos) - ps, r_min, s1, xtol=1e-15, rtol=1e-15)
        rl = optimize.brentq(lambda r: pressure(r, T, eos) - ps, s2, 0.999999 / eos.b, xtol=1e-15, rtol=1e-15)
        return rv, rl

    def area(ps):
        rv, rl = roots(ps)
        val, _ = integrate.quad(lambda r: pressure(r, T, eos) / (r * r), rv, rl,
                                epsabs=1e-14, epsrel=1e-13, limit=200)
        return val - ps * (1.0 / rv - 1.0 / rl)

    eps = 1e-12 * (p_hi - p_lo)
    ps = optimize.brentq(area, p_lo + eps, p_hi - eps, xtol=1e-16, rtol=1e-15)
    rv, rl = roots(ps)
    return rl, rv, ps


def latent_heat(T, eos: PR, rho_l=None, rho_v=None):
    """Eq. (14) per unit mass: int_{rho_v}^{rho_l} T (dp/dT)_rho / rho^2 drho."""
    if rho_l is None or rho_v is None:
        rho_l, rho_v, _ = coexistence(T, eos)
    val, _ = integrate.quad(lambda r: T_dp_dT(r, T, eos) / (r * r), rho_v, rho_l,
                            epsabs=1e-14, epsrel=1e-13, limit=200)
    return val
