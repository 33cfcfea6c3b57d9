"""D2Q9 lattice and MRT moment space for the oracle (plain FP64, test infrastructure).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import anything under ``oracle/``.

Follows Section 2.1 of Hu & Liu (arXiv 1812.10375):

* Eq. (2): f(x + e, t + 1) = M^-1 [ m - Lambda (m - m_eq) + (I - Lambda/2) S ].
* Eq. (3): Lambda = diag(1/tau_rho, 1/tau_e, 1/tau_zeta, 1/tau_j, 1/tau_q,
  1/tau_j, 1/tau_q, 1/tau_nu, 1/tau_nu).
* Eq. (4): m_eq = rho (1, -2 + 3|u|^2, 1 - 3|u|^2, ux, -ux, uy, -uy, ux^2 - uy^2, ux uy).
* Eq. (8): the forcing moments S of Li et al.

M is the orthogonal D2Q9 transformation whose rows (rho, e, zeta, jx, qx, jy,
qy, pxx, pxy) are the polynomials of the velocities that Eq. (4) implies; the
matrix is built here from those polynomials rather than typed in.
"""
from __future__ import annotations

import numpy as np

# velocities e_0..e_8: rest, 4 axis, 4 diagonal
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
              [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
EX = E[:, 0].astype(np.float64)
EY = E[:, 1].astype(np.float64)
# index of -e_i
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6], dtype=np.int64)
# lattice weights w_i (equilibrium at rest: f_i = w_i rho)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
# interaction weights omega(|e|^2) of Eq. (6): omega(1) = 1/3, omega(2) = 1/12
OMEGA = np.array([0.0] + [1 / 3] * 4 + [1 / 12] * 4, dtype=np.float64)


def _moment_matrix() -> np.ndarray:
    e2 = EX * EX + EY * EY
    rows = [
        np.ones(9),                              # rho
        -4.0 + 3.0 * e2,                         # e (energy)
        4.0 - 10.5 * e2 + 4.5 * e2 * e2,         # zeta (energy square)
        EX,                                      # jx
        (-5.0 + 3.0 * e2) * EX,                  # qx
        EY,                                      # jy
        (-5.0 + 3.0 * e2) * EY,                  # qy
        EX * EX - EY * EY,                       # pxx
        EX * EY,                                 # pxy
    ]
    return np.array(rows, dtype=np.float64)


M = _moment_matrix()
# M is orthogonal: M^-1 = M^T diag(1 / |row|^2) with integer row norms
M_INV = M.T / np.sum(M * M, axis=1)[None, :]


def m_eq(rho, ux, uy):
    """Eq. (4); arrays broadcast, result has a leading axis of 9."""
    u2 = ux * ux + uy * uy
    return np.stack([
        rho,
        rho * (-2.0 + 3.0 * u2),
        rho * (1.0 - 3.0 * u2),
        rho * ux,
        -rho * ux,
        rho * uy,
        -rho * uy,
        rho * (ux * ux - uy * uy),
        rho * ux * uy,
    ])


def forcing_moments(ux, uy, Fx, Fy, Fm2_over_psi2, tau_e, tau_zeta, sigma, sigma_coef):
    """Eq. (8), the forcing term S in moment space.

    Section 2.1 prints two typos that are read as follows: |F_m|^2 is
    F_mx^2 + F_my^2 (printed F_mx^2 + F_mx^2), and the last row is
    ux Fy + uy Fx (printed ux Fx + uy Fy); with sigma = 0 this S is then exactly
    M times the velocity-space forcing of Guo et al.  ``sigma_coef`` multiplies the
    sigma terms (the printed form has 1; Li et al.'s original scheme has 12).
    ``Fm2_over_psi2`` is |F_m|^2 / psi^2 (zero where psi = 0).
    """
    uF = ux * Fx + uy * Fy
    extra_e = sigma_coef * sigma * Fm2_over_psi2 / (tau_e - 0.5)
    extra_z = sigma_coef * sigma * Fm2_over_psi2 / (tau_zeta - 0.5)
    return np.stack([
        np.zeros_like(uF),
        6.0 * uF + extra_e,
        -6.0 * uF - extra_z,
        Fx,
        -Fx,
        Fy,
        -Fy,
        2.0 * (ux * Fx - uy * Fy),
        ux * Fy + uy * Fx,
    ])
