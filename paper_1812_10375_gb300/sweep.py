"""Boiling-curve sweep driver (Section 4.4, Fig. 11): many independent domains
of different sizes and superheats advanced by the batched step, with the
quasi-steady mean wall heat flux of each point taken over the second half of
its run, a plain one-domain-at-a-time comparator, and the surrogate-driven
early-stop policy."""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import hlb, workloads as wl
from .config import params_for
from .surrogate import downsample, regime_of


@dataclass
class PointResult:
    case: wl.Case
    superheat: float        # (T_wall - Ts) / Tc
    n_sites: int
    history: np.ndarray     # q_bottom per step (first `hist_steps` steps)
    q_qs: float             # mean q_bottom over the second half of the run
    coverage: float         # mean wall vapour fraction over the second half
    regime: int


def make_points(n, seed=wl.BASE_SEED, sides=(256, 320, 384, 448, 512), superheat_range=(0.02, 0.30),
                sites_range=(3, 9), heater_rows=25, aspect=1.0):
    """n sweep points as in workloads.sweep, with optional other sizes."""
    rng = np.random.default_rng(seed)
    dts = np.linspace(superheat_range[0], superheat_range[1], n)
    rng.shuffle(dts)
    out = []
    for d in range(n):
        side = int(rng.choice(np.asarray(sides)))
        nsite = int(rng.integers(sites_range[0], sites_range[1] + 1))
        sites = wl.draw_sites(rng, side, nsite)
        out.append(wl.Case(f"pt{d:03d}_{side}", nx=side, ny=int(round(side * aspect)), wall_rows=heater_rows,
                           top_bc="convective", T_bottom_over_Tc=wl.TS_OVER_TC + float(dts[d]), T_top_over_Tc=None,
                           eos_T_fixed=False, g_y=-wl.GRAVITY, Gw0=0.3, sites=sites))
    return out


def _setup(batch, i, case, p, Tc):
    import torch
    rho0, T0 = wl.initial_fields(case, p.rho_l, p.rho_v, Tc)
    batch.set_fields(i, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                     torch.tensor(T0, dtype=torch.float32, device="cuda"))
    batch.set_nucleation_sites(i, case.sites)


def run_batched(cases, steps, hist_steps, stop_after=None):
    """Run every point for `steps` steps in one batch (one launch per step for all).

    stop_after: optional per-point step counts at which a point is stopped
    early (its results are then partial).  Returns (results, seconds)."""
    import torch
    plist, tcs = [], []
    for c in cases:
        p, Tc = params_for(c)
        plist.append(p)
        tcs.append(Tc)
    b = hlb.Batch(plist)
    for i, c in enumerate(cases):
        _setup(b, i, c, plist[i], tcs[i])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    half = steps // 2
    stops = sorted(set(s for s in (stop_after or []) if s < steps))
    done = 0
    cov_half = [0.0] * len(cases)
    marks = sorted(set(stops + [half, steps]))
    for mark in marks:
        if mark > done:
            b.step(mark - done)
            done = mark
        if mark == half:
            for i in range(len(cases)):
                cov_half[i] = b.diag(i, check_flags=False).vapour_coverage_timeavg * half
        if stop_after:
            for i, s in enumerate(stop_after):
                if s == mark and s < steps:
                    b.stop(i)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    res = []
    for i, c in enumerate(cases):
        h = b.flux_history(i)
        dg = b.diag(i, check_flags=False)
        n = len(h)
        q_qs = float(h[n // 2:].mean()) if n >= 2 else float("nan")
        cov = (dg.vapour_coverage_timeavg * n - cov_half[i]) / max(n - half, 1) if n > half else float("nan")
        res.append(PointResult(c, c.T_bottom_over_Tc - wl.TS_OVER_TC, len(c.sites), h[:hist_steps], q_qs, cov,
                               regime_of(cov) if np.isfinite(cov) else -1))
    b.close()
    return res, seconds


def run_plain(cases, steps):
    """The same points one domain at a time (graph-captured single-domain steps)."""
    import torch
    t0 = time.perf_counter()
    for c in cases:
        p, Tc = params_for(c)
        d = hlb.Domain(p)
        rho0, T0 = wl.initial_fields(c, p.rho_l, p.rho_v, Tc)
        d.set_fields(torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                     torch.tensor(T0, dtype=torch.float32, device="cuda"))
        d.set_nucleation_sites(c.sites)
        d.step(steps)
        d.diag(check_flags=False)
        d.close()
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def features(results, L0):
    hist = np.stack([downsample(r.history, L0) for r in results])
    scal = np.array([[r.superheat, r.n_sites / 10.0] for r in results])
    q = np.array([r.q_qs for r in results])
    lab = np.array([max(r.regime, 0) for r in results], dtype=np.int32)
    return hist, scal, q, lab


def acceptance_score(ens, hist, scal):
    """Ensemble-mean probability that a point does not end in film boiling.

    Up to the transition regime the quasi-steady flux follows from the early
    history; the vapour film of the last regime forms late, after the history
    window, so points headed there run in full."""
    qp, spread, prob = ens.predict(hist, scal)
    return qp, 1.0 - prob[:, -1]


def choose_threshold(ens, results, L0, tol=0.03, floor=0.5):
    """Lowest acceptance score, not below `floor` (the ensemble must expect no
    film), at which every calibration point the policy would accept is within
    `tol` relative error of its full run (1.01: accept none)."""
    hist, scal, q, _ = features(results, L0)
    qp, score = acceptance_score(ens, hist, scal)
    err = np.abs(qp - q) / np.maximum(np.abs(q), 1e-12)
    best = 1.01
    for thr in np.sort(score)[::-1]:
        if thr < floor:
            break
        acc = score >= thr
        if err[acc].max() <= tol:
            best = float(thr)
        else:
            break
    return best


def evaluate_policy(ens, results, L0, threshold, hist_steps, full_steps, cells):
    """Stop a point after `hist_steps` when its acceptance score reaches the
    threshold (the ensemble-mean prediction is then the point's result), else
    run it in full.  Returns the accepted mask, the relative errors of the
    accepted points against their full runs, and the cell updates spent
    relative to running every point in full."""
    hist, scal, q, _ = features(results, L0)
    qp, score = acceptance_score(ens, hist, scal)
    acc = score >= threshold
    err = np.abs(qp - q) / np.maximum(np.abs(q), 1e-12)
    cells = np.asarray(cells, dtype=np.float64)
    spent = np.where(acc, hist_steps, full_steps) * cells
    return acc, err[acc], float(spent.sum() / (full_steps * cells.sum()))
