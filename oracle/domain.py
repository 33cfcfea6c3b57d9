"""One domain of the hybrid thermal LB phase-change model, stepped in plain FP64.

Test infrastructure: only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import anything under ``oracle/``.  It shares no code with the
GPU library.

The model is Hu & Liu, arXiv 1812.10375, Section 2:

* flow: D2Q9 MRT pseudo-potential LB, Eqs. (1)-(10);
* energy: Eq. (17) advanced by classical RK4 (Eq. 18) with N sub-steps (Eq. 27),
  the isotropic central gradient of Eq. (19) for u.grad T and div u, and the
  finite-volume diffusion term with harmonic face conductivities of
  Eqs. (22)-(26), or, as the paper's comparison scheme, the isotropic central
  form of Eqs. (20)-(21);
* walls: halfway bounce-back, conjugate heater in the energy equation held at
  T_bottom or heated by an imposed flux (Section 3.3), constant density or
  convective open top (Sections 3.3 and 4.2), wettability-based nucleation
  sites (Section 4.2, Fig. 6b).

Every stage works on full-field arrays indexed [y, x]; x is periodic.  One step
n takes the stored post-collision populations f*^{n-1} and T^n to f*^n and
T^{n+1}:

 1. pull-stream f^n(x) = f*^{n-1}(x - e_i); halfway bounce-back where x - e_i is
    solid; open-top rule for the populations that enter the top row;
 2. rho^n = sum_i f_i^n (Eq. 5);
 3. psi^n = psi(rho^n, T_EOS) (Eqs. 7, 28), T_EOS = T^n or Ts (Section 3.2);
 4. F = F_m + F_ads + F_b (Eqs. 6, 9, 10);
 5. u^n = (sum_i e_i f_i^n + F/2) / rho^n (Eq. 5);
 6. T^{n+1} = RK4^N(T^n) with rho^n, u^n held fixed (Eqs. 17-27);
 7. MRT collision with Li's forcing (Eqs. 2-4, 8) gives f*^n;
 8. FP64 diagnostics.

Readings of points the paper leaves open (each is a parameter or a documented
choice; the same list is kept with the design notes):

* Eq. (6) is used as F_m = -G psi(x) sum_i omega_i psi(x + e_i) e_i with G = -1
  (the printed sign is repulsive with Eq. 7).  A solid neighbour enters the sum
  with the fluid node's own psi(x), so that G_w = 0 is a moderately wetting
  wall and Eq. (10) moves the contact angle either way.
* Eq. (10) reads F_ads = G_w(x) psi(x)^2 sum_i (omega_i / 3) s(x + e_i) e_i: the
  printed weights omega_alpha = w_alpha / 3 are taken as one third of the
  Eq. (6) weights, i.e. the D2Q9 lattice weights 1/9 and 1/36.  G_w is taken
  at the fluid node's column.  With these two readings G_w = 0.3 gives a
  contact angle near the 35 degrees quoted in Section 4.2.
* tau_nu(rho) is linear in rho between tau_v (rho_v) and tau_l (rho_l) and clamped
  to that range; tau_l = 0.8 and tau_v = 1.0 follow from nu_l = 0.1 and
  nu_v = 0.5/3 (Section 3.1).  The other rates are not printed:
  s_rho = s_j = 1, s_e = s_zeta = 0.8, s_q = 1.1.
* rho_ave of Eq. (9) is the fluid-node mean of the previous step's density (the
  initial field at step 0).
* Open top, constant density (Section 3.3): the populations entering the top
  row are the rest equilibrium w_i rho_v.  Convective outlet (Section 4.2):
  f_i^n(top) = [f_i^{n-1}(top) + U f_i^n(top - 1)] / (1 + U) for the entering
  populations, U = max(0, mean u_y of the row below the top at step n-1).
  psi, T and u take zero-gradient ghost values above an open top, so the top
  face carries no conductive heat flux.
* Row 0 is a solid row with Dirichlet T; with a top wall, row ny-1 is a solid
  Dirichlet row too.  Solid rows take part in the energy equation with
  rho_w, cv_w and lambda_w (conjugate heater, Sections 3.3, 4.2).
* The latent-heat source uses T (dp/dT)_rho at the local stage temperature.
* The wall heat fluxes are the RK-weighted conductive fluxes through a face over
  one step, i.e. the heat that crossed it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import eos as _eos
from .lattice import E, EX, EY, M, M_INV, OMEGA, OPP, W, forcing_moments, m_eq

TOP_WALL = "wall"
TOP_CONST_RHO = "const_rho"
TOP_CONVECTIVE = "convective"

# error flag bits (same meaning as the library's device error word)
FLAG_NONFINITE = 1
FLAG_PSI_NEG = 2


@dataclass
class Params:
    nx: int
    ny: int
    wall_rows: int = 1              # rows y < wall_rows are solid; row 0 is a Dirichlet row
    top_bc: str = TOP_WALL
    T_bottom: float = 0.0           # Dirichlet T of row 0
    T_top: float = 0.0              # Dirichlet T of row ny-1 (top wall only)
    eos_T_fixed: bool = False       # EOS at Ts everywhere (Section 3.2)
    n_sub: int = 1                  # N of Eq. (27)
    eos: _eos.PR = field(default_factory=_eos.PR)
    Ts_over_Tc: float = 0.86
    G: float = -1.0
    sigma: float = 0.107
    sigma_coef: float = 12.0        # coefficient of the sigma terms of Eq. (8)
    s_rho: float = 1.0
    s_e: float = 0.8
    s_zeta: float = 0.8
    s_j: float = 1.0
    s_q: float = 1.1
    tau_l: float = 0.8
    tau_v: float = 1.0
    cv: float = 6.0
    k: float = 0.1
    rho_w: float | None = None      # default 3 rho_l
    cv_w: float | None = None       # default cv
    lambda_w: float | None = None   # default 3 rho_l cv k
    lambda_top: float | None = None # conductivity of a top wall row (default lambda_w)
    g_y: float = 0.0
    Gw: np.ndarray | float = 0.3    # per-column wetting strength or a constant
    rho_l: float | None = None      # coexistence densities at Ts (Maxwell if None)
    rho_v: float | None = None
    diffusion: str = "fv"          # "fv" (Eqs. 22-26) or "iso" (Eqs. 20-21, the comparison scheme)
    bottom_bc: str = "dirichlet"   # row 0 held at T_bottom, or "flux": heat q_in per unit time and
    q_in: float = 0.0              # unit length enters row 0 through its bottom face (Section 3.3)

    def resolved(self) -> "Params":
        p = Params(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        Ts = p.Ts_over_Tc * p.eos.Tc
        if p.rho_l is None or p.rho_v is None:
            p.rho_l, p.rho_v, _ = _eos.coexistence(Ts, p.eos)
        if p.rho_w is None:
            p.rho_w = 3.0 * p.rho_l
        if p.cv_w is None:
            p.cv_w = p.cv
        if p.lambda_w is None:
            p.lambda_w = 3.0 * p.rho_l * p.cv * p.k
        if p.lambda_top is None:
            p.lambda_top = p.lambda_w
        p.Gw = np.broadcast_to(np.asarray(p.Gw, dtype=np.float64), (p.nx,)).copy()
        return p

    @property
    def Ts(self) -> float:
        return self.Ts_over_Tc * self.eos.Tc


def nucleation_Gw(nx: int, Gw0: float, sites) -> np.ndarray:
    """Per-column wetting strength with nucleation sites (Section 4.2, Fig. 6b).

    Each site (x_c, width, g_min) is a linear drop from Gw0 to g_min at its
    centre over half the width on either side (x periodic); where sites
    overlap the lowest value wins.
    """
    x = np.arange(nx, dtype=np.float64)
    g = np.full(nx, Gw0, dtype=np.float64)
    for xc, width, gmin in sites:
        d = np.abs(x - xc)
        d = np.minimum(d, nx - d)
        half = 0.5 * width
        inside = d <= half
        g = np.where(inside, np.minimum(g, gmin + (Gw0 - gmin) * d / half), g)
    return g


def _pad(a: np.ndarray) -> np.ndarray:
    """One ghost layer around the last two axes: periodic in x, edge-row copy in y."""
    lead = [(0, 0)] * (a.ndim - 2)
    a = np.pad(a, lead + [(1, 1), (0, 0)], mode="edge")
    return np.pad(a, lead + [(0, 0), (1, 1)], mode="wrap")


def _at(P: np.ndarray, dx: int, dy: int) -> np.ndarray:
    """From a padded array P, b[y, x] = a[y + dy, x + dx] for |dx|, |dy| <= 1."""
    ny, nx = P.shape[-2] - 2, P.shape[-1] - 2
    return P[..., 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]


def _nb(a: np.ndarray, dx: int, dy: int) -> np.ndarray:
    """b[y, x] = a[y + dy, x + dx]; x periodic, y beyond the lattice copies the edge row."""
    return _at(_pad(a), dx, dy)


def iso_grad(a: np.ndarray):
    """Isotropic central gradient, Eq. (19)."""
    P = _pad(a)
    gx = ((_at(P, 1, 0) - _at(P, -1, 0)) / 3.0
          + (_at(P, 1, 1) - _at(P, -1, -1)) / 12.0
          + (_at(P, 1, -1) - _at(P, -1, 1)) / 12.0)
    gy = ((_at(P, 0, 1) - _at(P, 0, -1)) / 3.0
          + (_at(P, 1, 1) - _at(P, -1, -1)) / 12.0
          + (_at(P, -1, 1) - _at(P, 1, -1)) / 12.0)
    return gx, gy


def harmonic(la: np.ndarray, lb: np.ndarray) -> np.ndarray:
    """Face conductivity of Eq. (25) with dx = 1: 2 / (1/la + 1/lb)."""
    return 2.0 / (1.0 / la + 1.0 / lb)


class Domain:
    """State (f*^{n-1}, T^n) of one domain plus the lagged global scalars."""

    def __init__(self, params: Params, rho0: np.ndarray, T0: np.ndarray, conduction_only: bool = False):
        p = params.resolved()
        self.p = p
        nx, ny = p.nx, p.ny
        if p.wall_rows < 1:
            raise ValueError("wall_rows must be >= 1 (row 0 is the bottom wall)")
        y = np.arange(ny)[:, None] * np.ones((1, nx), dtype=np.int64)
        solid = y < p.wall_rows
        if p.top_bc == TOP_WALL:
            solid = solid | (y == ny - 1)
        self.solid = solid
        self.fluid = ~solid
        self.n_fluid = int(self.fluid.sum())
        if p.bottom_bc not in ("dirichlet", "flux"):
            raise ValueError("bottom_bc must be 'dirichlet' or 'flux'")
        dirichlet = (y == 0) & (p.bottom_bc == "dirichlet")
        Tfix = np.where(dirichlet, p.T_bottom, 0.0)
        if p.top_bc == TOP_WALL:
            dirichlet = dirichlet | (y == ny - 1)
            Tfix = np.where(y == ny - 1, p.T_top, Tfix)
        self.dirichlet = dirichlet
        self.T_fix = Tfix.astype(np.float64)
        self.conduction_only = conduction_only

        rho0 = np.asarray(rho0, dtype=np.float64)
        self.rho = np.where(self.fluid, rho0, 0.0)
        self.ux = np.zeros((ny, nx))
        self.uy = np.zeros((ny, nx))
        self.T = np.where(dirichlet, self.T_fix, np.asarray(T0, dtype=np.float64))
        # post-collision populations; the initial state is the rest equilibrium
        self.fs = W[:, None, None] * self.rho[None]
        # entering populations of the top row at the previous step (convective outlet)
        self.f_top_prev = self.fs[[4, 7, 8], ny - 1, :].copy()
        self.rho_ave = float(self.rho[self.fluid].mean())
        self.U = 0.0
        self.n = 0
        self.flags = 0
        self.last = {}
        self.q_bottom_sum = 0.0
        self.vcov_sum = 0.0

    # ------------------------------------------------------------------ flow
    def _stream(self) -> np.ndarray:
        p, fs = self.p, self.fs
        ny = p.ny
        f = np.empty_like(fs)
        Pf = _pad(fs)
        Ps = _pad(self.solid)
        for i in range(9):
            ex, ey = int(E[i, 0]), int(E[i, 1])
            pulled = _at(Pf[i], -ex, -ey)
            src_solid = _at(Ps, -ex, -ey)
            f[i] = np.where(src_solid, fs[OPP[i]], pulled)
        if p.top_bc != TOP_WALL:
            # populations entering the top row from above (e_y = -1)
            for j, i in enumerate((4, 7, 8)):
                if p.top_bc == TOP_CONST_RHO:
                    f[i, ny - 1, :] = W[i] * p.rho_v
                else:
                    f[i, ny - 1, :] = (self.f_top_prev[j] + self.U * f[i, ny - 2, :]) / (1.0 + self.U)
                    self.f_top_prev[j] = f[i, ny - 1, :]
        return np.where(self.fluid[None], f, 0.0)

    def _forces(self, rho, psi):
        """F = F_m + F_ads + F_b (Eqs. 6, 9, 10) on fluid nodes."""
        p = self.p
        solid = self.solid.astype(np.float64)
        Fmx = np.zeros_like(rho)
        Fmy = np.zeros_like(rho)
        Sx = np.zeros_like(rho)
        Sy = np.zeros_like(rho)
        Pp = _pad(psi)
        Ps = _pad(solid)
        for i in range(1, 9):
            ex, ey = int(E[i, 0]), int(E[i, 1])
            sn = _at(Ps, ex, ey)
            # Eq. (6) over all neighbours; a solid neighbour carries psi(x)
            pn = np.where(sn > 0.0, psi, _at(Pp, ex, ey))
            Fmx += OMEGA[i] * pn * ex
            Fmy += OMEGA[i] * pn * ey
            # Eq. (10) weights omega_alpha = omega(|e|^2) / 3
            Sx += OMEGA[i] / 3.0 * sn * ex
            Sy += OMEGA[i] / 3.0 * sn * ey
        Fmx *= -p.G * psi
        Fmy *= -p.G * psi
        Gw = p.Gw[None, :]
        Fax = Gw * psi * psi * Sx
        Fay = Gw * psi * psi * Sy
        Fbx = np.zeros_like(rho)
        Fby = (rho - self.rho_ave) * p.g_y
        fl = self.fluid
        Fx = np.where(fl, Fmx + Fax + Fbx, 0.0)
        Fy = np.where(fl, Fmy + Fay + Fby, 0.0)
        return Fx, Fy, np.where(fl, Fmx, 0.0), np.where(fl, Fmy, 0.0)

    def _collide(self, f, rho, ux, uy, Fx, Fy, Fmx, Fmy, psi):
        p = self.p
        m = np.einsum("ij,jyx->iyx", M, f)
        tau_nu = p.tau_v + (rho - p.rho_v) / (p.rho_l - p.rho_v) * (p.tau_l - p.tau_v)
        tau_nu = np.clip(tau_nu, min(p.tau_l, p.tau_v), max(p.tau_l, p.tau_v))
        ones = np.ones_like(rho)
        s = np.stack([p.s_rho * ones, p.s_e * ones, p.s_zeta * ones, p.s_j * ones, p.s_q * ones,
                      p.s_j * ones, p.s_q * ones, 1.0 / tau_nu, 1.0 / tau_nu])
        psi2 = psi * psi
        Fm2_psi2 = np.where(psi2 > 0.0, (Fmx * Fmx + Fmy * Fmy) / np.where(psi2 > 0.0, psi2, 1.0), 0.0)
        S = forcing_moments(ux, uy, Fx, Fy, Fm2_psi2, 1.0 / p.s_e, 1.0 / p.s_zeta, p.sigma, p.sigma_coef)
        meq = m_eq(rho, ux, uy)
        mstar = m - s * (m - meq) + (1.0 - 0.5 * s) * S
        fs = np.einsum("ij,jyx->iyx", M_INV, mstar)
        return np.where(self.fluid[None], fs, 0.0)

    # ---------------------------------------------------------------- energy
    def energy_coefficients(self, rho, ux, uy):
        """Quantities of Eq. (17) that stay fixed over the RK4 stages of one step."""
        p = self.p
        fl = self.fluid
        lam = np.where(fl, rho * p.cv * p.k, p.lambda_w)
        if p.top_bc == TOP_WALL:
            lam[p.ny - 1] = p.lambda_top
        P = _pad(lam)
        dux, _ = iso_grad(ux)
        _, duy = iso_grad(uy)
        glx, gly = iso_grad(lam)
        return dict(
            lam=lam, glx=glx, gly=gly,
            rho=np.where(fl, rho, 1.0), ux=ux, uy=uy, divu=dux + duy,
            rcv=np.where(fl, rho * p.cv, p.rho_w * p.cv_w),
            lam_e=harmonic(lam, _at(P, 1, 0)), lam_w=harmonic(lam, _at(P, -1, 0)),
            lam_n=harmonic(lam, _at(P, 0, 1)), lam_s=harmonic(lam, _at(P, 0, -1)))

    def energy_rhs(self, T, c):
        """K(T), the right-hand side of Eq. (17).

        Diffusion: finite volume with harmonic face conductivities (Eqs. 22-26),
        or, with ``diffusion="iso"``, the isotropic central form of Eqs. (20)-(21)
        that the paper compares against (it is not conservative).
        Advection and div u: isotropic central differences (Eq. 19).  Solid
        nodes carry only diffusion; Dirichlet rows do not change.
        """
        P = _pad(T)
        if self.p.diffusion == "iso":
            # Eq. (21): lambda * laplacian(T) + grad(lambda) . grad(T), with the
            # isotropic Laplacian of Eq. (20) and the gradients of Eq. (19)
            lap = (_at(P, 1, 1) + _at(P, -1, 1) + _at(P, 1, -1) + _at(P, -1, -1)
                   + 4.0 * (_at(P, 1, 0) + _at(P, -1, 0) + _at(P, 0, 1) + _at(P, 0, -1)) - 20.0 * T) / 6.0
            gTx, gTy = iso_grad(T)
            diff = c["lam"] * lap + c["glx"] * gTx + c["gly"] * gTy
        else:
            diff = (c["lam_e"] * (_at(P, 1, 0) - T) + c["lam_w"] * (_at(P, -1, 0) - T)
                    + c["lam_n"] * (_at(P, 0, 1) - T) + c["lam_s"] * (_at(P, 0, -1) - T))
        k = diff / c["rcv"]
        if self.p.bottom_bc == "flux":
            # Section 3.3: the imposed heat flux enters row 0's control volume from
            # below (beyond the lattice T is the edge copy, so no other flux crosses
            # that face)
            k[0] = k[0] + self.p.q_in / c["rcv"][0]
        gx, gy = iso_grad(T)
        adv = c["ux"] * gx + c["uy"] * gy
        src = _eos.T_dp_dT(c["rho"], T, self.p.eos) / c["rcv"] * c["divu"]
        k = np.where(self.fluid, k - adv - src, k)
        return np.where(self.dirichlet, 0.0, k)

    def _energy(self, rho, ux, uy):
        """T^{n+1} from T^n by N RK4 sub-steps (Eqs. 17, 18, 27)."""
        p = self.p
        c = self.energy_coefficients(rho, ux, uy)
        W_ = p.wall_rows
        ny = p.ny

        def face_fluxes(T):
            # heat per unit time through: the bottom Dirichlet face (into row 1),
            # the top Dirichlet face (out of row ny-2), and the solid->fluid face
            qb = np.sum(c["lam_s"][1] * (T[0] - T[1]))
            qt = np.sum(c["lam_n"][ny - 2] * (T[ny - 2] - T[ny - 1])) if p.top_bc == TOP_WALL else 0.0
            qi = np.sum(c["lam_s"][W_] * (T[W_ - 1] - T[W_]))
            return np.array([qb, qt, qi])

        dt = 1.0 / p.n_sub
        T = self.T
        acc = np.zeros(3)
        for _ in range(p.n_sub):
            h1 = self.energy_rhs(T, c)
            T2 = T + 0.5 * dt * h1
            h2 = self.energy_rhs(T2, c)
            T3 = T + 0.5 * dt * h2
            h3 = self.energy_rhs(T3, c)
            T4 = T + dt * h3
            h4 = self.energy_rhs(T4, c)
            acc += dt / 6.0 * (face_fluxes(T) + 2.0 * face_fluxes(T2) + 2.0 * face_fluxes(T3) + face_fluxes(T4))
            T = T + dt / 6.0 * (h1 + 2.0 * h2 + 2.0 * h3 + h4)
        return T, acc / p.nx, c["rcv"]

    # ------------------------------------------------------------------ step
    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            self._step()
        return self

    def _step(self):
        p = self.p
        fl = self.fluid
        if self.conduction_only:
            rho, ux, uy = self.rho, np.zeros_like(self.rho), np.zeros_like(self.rho)
        else:
            f = self._stream()
            rho = np.where(fl, f.sum(axis=0), 0.0)
            T_eos = np.full_like(rho, p.Ts) if p.eos_T_fixed else self.T
            psi2 = np.where(fl, _eos.psi_squared(np.where(fl, rho, 1.0), T_eos, p.eos), 0.0)
            if np.any(psi2 < 0.0):
                self.flags |= FLAG_PSI_NEG
            psi = np.sqrt(np.maximum(psi2, 0.0))
            Fx, Fy, Fmx, Fmy = self._forces(rho, psi)
            rho_safe = np.where(fl, rho, 1.0)
            ux = np.where(fl, (np.tensordot(EX, f, axes=1) + 0.5 * Fx) / rho_safe, 0.0)
            uy = np.where(fl, (np.tensordot(EY, f, axes=1) + 0.5 * Fy) / rho_safe, 0.0)
        T_new, q, rcv = self._energy(rho, ux, uy)
        if not self.conduction_only:
            self.fs = self._collide(f, rho, ux, uy, Fx, Fy, Fmx, Fmy, psi)
        mass = float(rho[fl].sum())
        u_top = float(uy[p.ny - 2].mean())
        # vapour fraction of the first fluid row above the bottom wall
        vcov = float(np.mean(rho[p.wall_rows] < 0.5 * (p.rho_l + p.rho_v)))
        self.rho, self.ux, self.uy, self.T = rho, ux, uy, T_new
        if not (np.all(np.isfinite(T_new)) and np.all(np.isfinite(self.fs))):
            self.flags |= FLAG_NONFINITE
        self.rho_ave = mass / self.n_fluid
        self.U = max(0.0, u_top)
        self.n += 1
        self.q_bottom_sum += float(q[0])
        self.vcov_sum += vcov
        self.last = dict(step=self.n, mass=mass, energy=float(np.sum(rcv * T_new)),
                         q_bottom=float(q[0]), q_top=float(q[1]), q_interface=float(q[2]),
                         rho_ave=self.rho_ave, u_top=u_top,
                         q_bottom_timeavg=self.q_bottom_sum / self.n, error_flags=self.flags,
                         vapour_coverage=vcov, vapour_coverage_timeavg=self.vcov_sum / self.n)

    # --------------------------------------------------------------- outputs
    def fields(self):
        """(rho^n, ux^n, uy^n, T^{n+1}) of the last step (initial fields before any step)."""
        return self.rho.copy(), self.ux.copy(), self.uy.copy(), self.T.copy()

    def diag(self) -> dict:
        return dict(self.last)
