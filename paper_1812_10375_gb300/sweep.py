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
    n_sub: int = 1          # N of Eq. (27) the point ran with


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
    q_half = [0.0] * len(cases)
    marks = sorted(set(stops + [half, steps]))
    for mark in marks:
        if mark > done:
            b.step(mark - done)
            done = mark
        if mark == half:
            for i in range(len(cases)):
                dg = b.diag(i, check_flags=False)
                cov_half[i] = dg.vapour_coverage_timeavg * half
                q_half[i] = dg.q_bottom_timeavg * half
        if stop_after:
            for i, s in enumerate(stop_after):
                if s == mark and s < steps:
                    b.stop(i)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    res = [_point_result(c, b.flux_history(i), b.diag(i, check_flags=False), half, q_half[i], cov_half[i],
                         hist_steps) for i, c in enumerate(cases)]
    b.close()
    return res, seconds


def _point_result(case, h, dg, half, q_half, cov_half, hist_steps, n_sub=1):
    """A point's result from its flux history and diagnostics: means over the
    second half of the run (steps half+1 .. dg.step); q_half and cov_half are
    the running sums of q_bottom and of the wall vapour fraction at step half."""
    n = len(h)
    if n == dg.step:
        q_qs = float(h[n // 2:].mean()) if n >= 2 else float("nan")
    else:  # the stored history is shorter than the run: use the running sums
        n = dg.step
        q_qs = (dg.q_bottom_timeavg * n - q_half) / max(n - half, 1) if n > half else float("nan")
    cov = (dg.vapour_coverage_timeavg * n - cov_half) / max(n - half, 1) if n > half else float("nan")
    return PointResult(case, case.T_bottom_over_Tc - wl.TS_OVER_TC, len(case.sites), h[:hist_steps], q_qs, cov,
                       regime_of(cov) if np.isfinite(cov) else -1, n_sub)


def run_resumable(cases, steps, hist_steps, ckpt_dir, every=2048, retry=True):
    """run_batched with a checkpoint of every point on disk each `every` steps
    (and at the half-way step), so that a sweep cut short resumes per point.

    Per point k, `ckpt_dir` holds pt<k>.ckpt.npz (the library checkpoint of
    its last good step with the half-way running sums and its N of Eq. 27)
    and, once the point is finished, pt<k>.done.npz (its result).  Calling this
    again with the same cases and directory skips finished points and restores
    the others from their checkpoints; points at different steps advance one
    group at a time until they share a step.

    A point whose device error word is set at a checkpoint boundary is stopped.
    With `retry`, it runs once more, alone, from its last good checkpoint (or
    its initial fields) with N of Eq. (27) doubled: the explicit energy update
    is the part of the step whose stability N controls (Section 2.2), and the
    step being deterministic, running it again unchanged would fail the same
    way.  A point that fails again, or any failed point without `retry`, is
    recorded with NaN means, regime -1 and `failed_at` (the step of the
    detection); its last good checkpoint stays on disk.

    Returns (results, failed_at) with failed_at[k] = -1 for points that ran
    to the end; results[k].n_sub is the N the point finished (or failed) with."""
    import os
    every = max(16, (int(every) + 15) // 16 * 16)  # whole graph chunks
    half = steps // 2
    os.makedirs(ckpt_dir, exist_ok=True)
    ck = lambda k: os.path.join(ckpt_dir, f"pt{k:05d}.ckpt.npz")
    dn = lambda k: os.path.join(ckpt_dir, f"pt{k:05d}.done.npz")
    results, failed_at = [None] * len(cases), [-1] * len(cases)
    for k, c in enumerate(cases):
        if os.path.exists(dn(k)):
            results[k], failed_at[k] = _load_done(dn(k), c, steps)
    meta = {}
    for k in range(len(cases)):
        if results[k] is None and os.path.exists(ck(k)):
            blob, m = hlb.read_checkpoint(ck(k))
            if str(m["name"]) != cases[k].name or int(m["steps"]) != steps:
                raise ValueError(f"{ck(k)} belongs to another sweep")
            meta[k] = (blob, m)
    base_n = {k: params_for(cases[k])[0].n_sub for k in range(len(cases)) if results[k] is None}
    # points resumed inside their retry continue alone at their checkpoint's N
    ck_n = {k: int(meta[k][1].get("n_sub", base_n[k])) for k in meta}
    single = {k: n for k, n in ck_n.items() if n > base_n[k]}
    todo = [k for k in range(len(cases)) if results[k] is None and k not in single]
    if todo:
        plist, tcs = zip(*[params_for(cases[k]) for k in todo])
        b = hlb.Batch(list(plist))
        pos, blobs, q_half, cov_half = [], [], [], []
        for j, k in enumerate(todo):
            if k in meta:
                blob, m = meta[k]
                b.restore(j, blob)
                pos.append(int(m["step"]))
                q_half.append(float(m["q_half"]))
                cov_half.append(float(m["cov_half"]))
            else:
                _setup(b, j, cases[k], plist[j], tcs[j])
                blob = None
                pos.append(0)
                q_half.append(0.0)
                cov_half.append(0.0)
            blobs.append(blob)
        active = [True] * len(todo)
        failed = [False] * len(todo)
        while True:
            left = [j for j in range(len(todo)) if pos[j] < steps and not failed[j]]
            if not left:
                break
            m = min(pos[j] for j in left)
            run = {j for j in left if pos[j] == m}
            for j in range(len(todo)):
                if active[j] and j not in run:
                    b.stop(j)
                    active[j] = False
                elif j in run and not active[j]:
                    b.restore(j, blobs[j])  # its own state: picks up where it stopped
                    active[j] = True
            nxt = min((m // every + 1) * every, steps, half if m < half else steps)
            b.step(nxt - m)
            for j in sorted(run):
                k = todo[j]
                pos[j] = nxt
                dg = b.diag(j, check_flags=False)
                if dg.error_flags:
                    failed[j] = True
                    b.stop(j)
                    active[j] = False
                    if retry and 2 * plist[j].n_sub <= MAX_SUB:
                        single[k] = 2 * plist[j].n_sub
                    else:
                        _record_failure(results, failed_at, k, cases[k], steps, nxt, plist[j].n_sub, dn(k))
                    continue
                if nxt == half:
                    q_half[j] = dg.q_bottom_timeavg * half
                    cov_half[j] = dg.vapour_coverage_timeavg * half
                blobs[j] = b.checkpoint(j)
                hlb.write_checkpoint(ck(k), blobs[j], name=cases[k].name, steps=steps, step=nxt,
                                     q_half=q_half[j], cov_half=cov_half[j], n_sub=plist[j].n_sub)
                if nxt == steps:
                    results[k] = _point_result(cases[k], b.flux_history(j), dg, half, q_half[j], cov_half[j],
                                               hist_steps, plist[j].n_sub)
                    _save_done(dn(k), results[k], steps, -1)
        for j, k in enumerate(todo):  # restored at the last step, finished before its result was written
            if results[k] is None and not failed[j]:
                results[k] = _point_result(cases[k], b.flux_history(j), b.diag(j, check_flags=False), half,
                                           q_half[j], cov_half[j], hist_steps, plist[j].n_sub)
                _save_done(dn(k), results[k], steps, -1)
        b.close()
    for k in sorted(single):
        _run_single(results, failed_at, k, cases[k], single[k], steps, hist_steps, every, ck(k), dn(k))
    return results, failed_at


MAX_SUB = 64  # the library's largest N of Eq. (27)


def _setup_domain(d, case, p, Tc):
    import torch
    rho0, T0 = wl.initial_fields(case, p.rho_l, p.rho_v, Tc)
    d.set_fields(torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                 torch.tensor(T0, dtype=torch.float32, device="cuda"))
    d.set_nucleation_sites(case.sites)


def _record_failure(results, failed_at, k, case, steps, at, n_sub, done_path):
    results[k] = PointResult(case, case.T_bottom_over_Tc - wl.TS_OVER_TC, len(case.sites), np.zeros(0),
                             float("nan"), float("nan"), -1, n_sub)
    failed_at[k] = at
    _save_done(done_path, results[k], steps, at)


def _run_single(results, failed_at, k, case, n_sub, steps, hist_steps, every, ck_path, done_path):
    """One sweep point alone in a domain with N = n_sub, from its checkpoint
    (taken at any N: the checkpoint holds state, not the model) or from its
    initial fields, with checkpoints as in the batch; no further retry."""
    import os
    half = steps // 2
    p, Tc = params_for(case)
    p.n_sub = n_sub
    d = hlb.Domain(p)
    if os.path.exists(ck_path):
        blob, m = hlb.read_checkpoint(ck_path)
        d.restore(blob)
        pos, q_half, cov_half = int(m["step"]), float(m["q_half"]), float(m["cov_half"])
    else:
        _setup_domain(d, case, p, Tc)
        pos, q_half, cov_half = 0, 0.0, 0.0
    dg = d.diag(check_flags=False)
    while pos < steps:
        nxt = min((pos // every + 1) * every, steps, half if pos < half else steps)
        d.step(nxt - pos)
        pos = nxt
        dg = d.diag(check_flags=False)
        if dg.error_flags:
            _record_failure(results, failed_at, k, case, steps, nxt, n_sub, done_path)
            d.close()
            return
        if nxt == half:
            q_half = dg.q_bottom_timeavg * half
            cov_half = dg.vapour_coverage_timeavg * half
        hlb.write_checkpoint(ck_path, d.checkpoint(), name=case.name, steps=steps, step=nxt, q_half=q_half,
                             cov_half=cov_half, n_sub=n_sub)
    results[k] = _point_result(case, d.flux_history(), dg, half, q_half, cov_half, hist_steps, n_sub)
    _save_done(done_path, results[k], steps, -1)
    d.close()


def _save_done(path, r, steps, failed_at):
    import os
    tmp = path + ".tmp.npz"
    np.savez(tmp, name=r.case.name, steps=steps, history=r.history, q=r.q_qs, coverage=r.coverage,
             regime=r.regime, failed_at=failed_at, n_sub=r.n_sub)
    os.replace(tmp, path)


def _load_done(path, case, steps):
    with np.load(path) as z:
        if str(z["name"]) != case.name or int(z["steps"]) != steps:
            raise ValueError(f"{path} belongs to another sweep")
        return (PointResult(case, case.T_bottom_over_Tc - wl.TS_OVER_TC, len(case.sites), z["history"].copy(),
                            float(z["q"]), float(z["coverage"]), int(z["regime"]), int(z["n_sub"])),
                int(z["failed_at"]))


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


def policy_score(prob, kind):
    """Acceptance score from the ensemble-mean regime probabilities: 'not_film'
    is the probability that the point does not end in film boiling (the vapour
    film forms late, after the history window); 'no_boiling' and
    'no_boiling_ratio' the probability that it does not boil at all, where the
    quasi-steady flux is a fixed fraction of the early flux (transient
    conduction)."""
    return 1.0 - prob[:, -1] if kind == "not_film" else prob[:, 0]


# The 'no_boiling_ratio' policy takes the network's regime probabilities but
# not its flux: a point that does not boil conducts heat from the heater into
# the liquid, and its quasi-steady wall flux is the mean flux of the last
# RATIO_WIN steps of the history window times a ratio set by the geometry
# (the heater, the materials and the initial fields are the same for every
# sweep point; only the side nx differs), fitted on the training points that
# ended without boiling.
RATIO_WIN = 500


def late_flux(history, hist_steps):
    """Mean wall flux over the last RATIO_WIN steps of the first hist_steps."""
    h = np.asarray(history, dtype=np.float64)[:hist_steps]
    return float(h[-RATIO_WIN:].mean())


def fit_conduction_ratio(results, hist_steps):
    """Least-squares (c0, c1) of q_qs / late_flux = c0 + c1 / nx over the
    results of regime 0 (no boiling); (0, 0) with fewer than two of them."""
    rows = [r for r in results if r.regime == 0]
    if len(rows) < 2:
        return 0.0, 0.0
    A = np.array([[1.0, 1.0 / r.case.nx] for r in rows])
    y = np.array([r.q_qs / late_flux(r.history, hist_steps) for r in rows])
    c0, c1 = np.linalg.lstsq(A, y, rcond=None)[0]
    return float(c0), float(c1)


def conduction_q(ratio, nx, history, hist_steps):
    """The 'no_boiling_ratio' prediction of the quasi-steady flux of a point."""
    return (ratio[0] + ratio[1] / nx) * late_flux(history, hist_steps)


def policy_q(kind, qp, results, ratio, hist_steps):
    """Predicted quasi-steady flux of each result under a policy kind."""
    if kind != "no_boiling_ratio":
        return qp
    return np.array([conduction_q(ratio, r.case.nx, r.history, hist_steps) for r in results])


def choose_policy(ens, results, L0, tol=0.03, floor=0.5, kind="not_film", ratio=(0.0, 0.0), hist_steps=None):
    """Acceptance by score and ensemble agreement: among the pairs (score
    threshold, spread limit) taken from the calibration points, the one that
    accepts the most calibration points while every accepted one stays within
    `tol` of its full run.  Returns (score threshold, spread limit); (1.01, 0)
    accepts nothing.  `ratio` and `hist_steps` serve the 'no_boiling_ratio'
    kind (conduction_q)."""
    hist, scal, q, _ = features(results, L0)
    qp, spread, prob = ens.predict(hist, scal)
    qp = policy_q(kind, qp, results, ratio, hist_steps)
    score = policy_score(prob, kind)
    err = np.abs(qp - q) / np.maximum(np.abs(q), 1e-12)
    best, best_n = (1.01, 0.0), 0
    for thr in np.unique(score[score >= floor]):
        for smax in np.unique(spread):
            acc = (score >= thr) & (spread <= smax)
            n = int(acc.sum())
            if n > best_n and err[acc].max() <= tol:
                best, best_n = (float(thr), float(smax)), n
    return best


def evaluate_policy(ens, results, L0, threshold, hist_steps, full_steps, cells, spread_max=None, kind="not_film",
                    ratio=(0.0, 0.0)):
    """Stop a point after `hist_steps` when its acceptance score reaches the
    threshold (the policy's prediction is then the point's result: the
    ensemble mean, or conduction_q for 'no_boiling_ratio'), else run it in
    full.  Returns the accepted mask, the relative errors of the accepted
    points against their full runs, and the cell updates spent relative to
    running every point in full."""
    hist, scal, q, _ = features(results, L0)
    qp, spread, prob = ens.predict(hist, scal)
    qp = policy_q(kind, qp, results, ratio, hist_steps)
    score = policy_score(prob, kind)
    acc = score >= threshold
    if spread_max is not None:
        acc &= spread <= spread_max
    err = np.abs(qp - q) / np.maximum(np.abs(q), 1e-12)
    cells = np.asarray(cells, dtype=np.float64)
    spent = np.where(acc, hist_steps, full_steps) * cells
    return acc, err[acc], float(spent.sum() / (full_steps * cells.sum()))


# ------------------------------------------------------------------ frozen policy and points/hour
POLICY_FILE = "surrogate_policy.npz"  # in the package directory, written by train_policy
TRAIN_SEED = wl.BASE_SEED          # the training and calibration points
STUDY_SEED = wl.BASE_SEED + 7777    # fresh points for the points/hour measurement


def policy_path() -> str:
    import os
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), POLICY_FILE)


def train_policy(n=256, full=40000, hist_steps=5000, n_fit=160, members=4, epochs=600, tol=0.02, out=None,
                 cache=None):
    """Train the early-stop ensemble and freeze its policy on calibration data.

    n sweep points (seed TRAIN_SEED, sides 256-512) run `full` steps in one
    batch; the ensemble is fitted by the CUDA kernels on the first n_fit; on
    the remaining points (calibration only) the policy kind ('no_boiling',
    'not_film' or 'no_boiling_ratio', whose conduction ratio is fitted on the
    fit points), the score threshold and the ensemble-spread limit are chosen
    that accept the most calibration points with every accepted one within
    `tol` of its full run (below the 3% bar, to leave room for unseen
    points).  Writes the ensemble and the policy to `out` (policy_path())."""
    import os
    from .surrogate import Ensemble
    pts = make_points(n, seed=TRAIN_SEED)
    if cache and os.path.exists(cache):
        res = _load_results(cache, pts)
    else:
        res, _ = run_batched(pts, full, hist_steps)
        if cache:
            _save_results(cache, res)
    fit, cal = res[:n_fit], res[n_fit:]
    ens = Ensemble(members=members, seed=3, max_batch=max(n_fit, 64))
    L0 = ens.members[0].net.cfg.L0
    hist, scal, q, lab = features(fit, L0)
    ens.fit(hist, scal, q, lab, epochs=epochs, batch=64, lr=1e-3)
    ratio = fit_conduction_ratio(fit, hist_steps)
    best = None
    for kind in ("no_boiling", "not_film", "no_boiling_ratio"):
        thr, smax = choose_policy(ens, cal, L0, tol=tol, kind=kind, ratio=ratio, hist_steps=hist_steps)
        acc, err, _ = evaluate_policy(ens, cal, L0, thr, hist_steps, full, [r.case.nx * r.case.ny for r in cal],
                                      spread_max=smax, kind=kind, ratio=ratio)
        if best is None or int(acc.sum()) > best[3]:
            best = (kind, thr, smax, int(acc.sum()), float(err.max()) if len(err) else 0.0)
    kind, thr, smax, n_acc, e_max = best
    meta = dict(kind=kind, threshold=thr, spread_max=smax, hist_steps=hist_steps, full_steps=full, tol=tol,
                calibration_points=len(cal), calibration_accepted=n_acc, calibration_max_error=e_max,
                train_seed=TRAIN_SEED, fit_points=n_fit, cond_c0=ratio[0], cond_c1=ratio[1])
    ens.save(out or policy_path(), **meta)
    return meta


def _q_second_half(h):
    n = len(h)
    return float(np.mean(h[n // 2:])) if n >= 2 else float("nan")


def pph_study(n=32, full=40000, slots_per_size=None, seed=STUDY_SEED, policy=None):
    """Boiling-curve points per hour, measured in three arms on n fresh points
    (seed STUDY_SEED, C4-shaped: square sides 256-512, 3-9 sites, superheats
    0.02-0.30 Tc), each point `full` steps unless stopped early:

    plain      one domain at a time (graph-captured single-domain steps);
    batched    a batch whose slots hold half of each size's points; a slot is
               refilled with the next point of its size when its point ends
               at `full` steps;
    surrogate  the same slots; after `hist_steps` steps the frozen policy
               (train_policy) either accepts a point, whose prediction is
               then its result and whose slot is refilled at once, or lets
               it run to `full`.

    Every arm counts, per point, its initial fields (set_wall, set_fields,
    the nucleation sites), its steps, the reads of its history and, in the
    surrogate arm, the policy's call; allocating the domains (one per size)
    or the batch is set-up, timed separately and excluded from all three.
    The batched arm gives the full-run wall flux of every point, against
    which the surrogate arm's accepted points are checked."""
    import torch
    from .surrogate import Ensemble
    ens, meta = Ensemble.load(policy or policy_path())
    kind, thr = str(meta["kind"]), float(meta["threshold"])
    smax, hs = float(meta["spread_max"]), int(meta["hist_steps"])
    ratio = (float(meta.get("cond_c0", 0.0)), float(meta.get("cond_c1", 0.0)))
    L0 = ens.members[0].net.cfg.L0
    pts = make_points(n, seed=seed)
    sizes = sorted(set(c.nx for c in pts))
    by_size = {s: [k for k, c in enumerate(pts) if c.nx == s] for s in sizes}
    nslot = {s: max(1, (len(v) + 1) // 2) if slots_per_size is None else min(slots_per_size, len(v))
             for s, v in by_size.items()}
    params = [params_for(c) for c in pts]

    # ---- plain: one domain at a time (one domain per size, allocated up front)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    doms = {}
    for s in sizes:
        k0 = by_size[s][0]
        doms[s] = hlb.Domain(params[k0][0])
    torch.cuda.synchronize()
    setup_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    for k, c in enumerate(pts):
        p, Tc = params[k]
        d = doms[c.nx]
        d.set_wall(p.T_bottom)
        _setup_domain(d, c, p, Tc)
        d.step(full)
        d.diag(check_flags=False)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    for d in doms.values():
        d.close()

    def slot_arm(use_policy):
        """Run all points through the slots; returns (seconds, set-up seconds, per-point record)."""
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        slot_pts = []  # point of each slot
        for s in sizes:
            slot_pts += by_size[s][:nslot[s]]
        queue = {s: list(by_size[s][nslot[s]:]) for s in sizes}
        b = hlb.Batch([params[k][0] for k in slot_pts])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for i, k in enumerate(slot_pts):
            _setup(b, i, pts[k], params[k][0], params[k][1])
        age = [0] * len(slot_pts)
        rec = {}
        live = set(range(len(slot_pts)))
        # the next event of a slot: the policy's look at hist_steps, the end at full
        nxt = lambda i: (hs if use_policy and age[i] < hs else full) - age[i]
        while live:
            step = min(nxt(i) for i in live)
            b.step(step)
            for i in list(live):
                age[i] += step
                k = slot_pts[i]
                done = None
                if age[i] >= full:
                    h = b.flux_history(i)
                    done = dict(q=_q_second_half(h[:full]), steps=full, accepted=False)
                elif use_policy and age[i] == hs:
                    h = b.flux_history(i)[:hs]
                    c = pts[k]
                    hist = downsample(h, L0)[None]
                    scal = np.array([[c.T_bottom_over_Tc - wl.TS_OVER_TC, len(c.sites) / 10.0]])
                    qp, spread, prob = ens.predict(hist, scal)
                    if policy_score(prob, kind)[0] >= thr and spread[0] <= smax:
                        qk = conduction_q(ratio, c.nx, h, hs) if kind == "no_boiling_ratio" else float(qp[0])
                        done = dict(q=qk, steps=hs, accepted=True)
                if done is None:
                    continue
                rec[k] = done
                s = pts[k].nx
                if queue[s]:
                    nk = queue[s].pop(0)
                    slot_pts[i] = nk
                    p, Tc = params[nk]
                    b.set_wall(i, p.T_bottom)
                    _setup(b, i, pts[nk], p, Tc)
                    age[i] = 0
                else:
                    b.stop(i)
                    live.discard(i)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        b.close()
        return t2 - t1, t1 - t0, rec

    t_batch, setup_batch, full_rec = slot_arm(False)
    t_sur, setup_sur, sur_rec = slot_arm(True)
    acc = [k for k, r in sur_rec.items() if r["accepted"]]
    err = [abs(sur_rec[k]["q"] - full_rec[k]["q"]) / max(abs(full_rec[k]["q"]), 1e-12) for k in acc]
    cells = np.array([c.nx * c.ny for c in pts], dtype=np.float64)
    spent = sum(cells[k] * sur_rec[k]["steps"] for k in sur_rec) / (cells.sum() * full)
    ph = lambda secs: n * 3600.0 / secs
    return {"unit": f"boiling-curve points/hour at {full} steps per point (measured, no extrapolation)",
            "points": n, "plain": ph(t_plain), "batched": ph(t_batch), "batched_with_surrogate": ph(t_sur),
            "seconds": {"plain": t_plain, "batched": t_batch, "batched_with_surrogate": t_sur},
            "setup_seconds_excluded": {"plain": setup_plain, "batched": setup_batch,
                                       "batched_with_surrogate": setup_sur},
            "slots": int(sum(nslot.values())), "accepted": len(acc),
            "accepted_max_error": max(err) if err else 0.0,
            "accepted_errors": sorted(round(float(e), 5) for e in err), "work_fraction": float(spent),
            "policy": {"kind": kind, "threshold": thr, "spread_max": smax, "hist_steps": hs,
                       "conduction_ratio": list(ratio) if kind == "no_boiling_ratio" else None,
                       "calibration_max_error": float(meta["calibration_max_error"]),
                       "calibration_accepted": int(meta["calibration_accepted"]),
                       "calibration_points": int(meta["calibration_points"])},
            "seed": seed}


# ------------------------------------------------------------------ Fig. 11 at the paper's scale
PAPER_SITE_MINIMA = (0.0, -0.3, -0.6)


def liquid_cp(p: hlb.hlb_params) -> float:
    """Isobaric specific heat of the saturated liquid at Ts for the
    Peng-Robinson fluid of Eq. (28) with constant c_v:
    c_p = c_v + T (dp/dT)_rho^2 / (rho^2 (dp/drho)_T)."""
    Tc, rho, _, _ = hlb.eos_coexistence(p)
    T = p.Ts_over_Tc * Tc
    kappa = 0.37464 + 1.54226 * p.omega - 0.26992 * p.omega ** 2
    a, b, R = p.a, p.b, p.R
    al = 1.0 + kappa * (1.0 - np.sqrt(T / Tc))
    den = 1.0 + 2.0 * b * rho - (b * rho) ** 2
    dphi_dT = -kappa * al / np.sqrt(T * Tc)
    dp_dT = rho * R / (1.0 - b * rho) - a * dphi_dT * rho ** 2 / den
    dp_drho = (R * T / (1.0 - b * rho) ** 2
               - a * al ** 2 * (2.0 * rho * den - rho ** 2 * (2.0 * b - 2.0 * b * b * rho)) / den ** 2)
    return float(p.cv + T * dp_dT ** 2 / (rho ** 2 * dp_drho))


def paper_cases(ja_values, nx=400, ny=600, heater_rows=25, seed=wl.BASE_SEED, cp=None):
    """Section 4.4's geometry: a 400 x 600 pool on a 25-row heater with three
    nucleation sites of minima 0, -0.3 and -0.6 at seeded columns, one case per
    Jakob number Ja = c_p (T_w - Ts) / h_fg, the wall superheat following from
    Ja with the model's own h_fg.  The paper does not give c_p; the default
    takes c_v (the model's constant specific heat), with which the onset and
    the maximum of the boiling curve fall where the paper puts them; the
    saturated liquid's isobaric c_p of the equation of state (liquid_cp, about
    2.5 c_v) can be passed instead."""
    p0 = hlb.default_params(nx, ny)
    Tc, _, _, h_fg = hlb.eos_coexistence(p0)
    cp = p0.cv if cp is None else cp
    rng = np.random.default_rng(seed)
    sites = wl.draw_sites(rng, nx, 3, minima=PAPER_SITE_MINIMA)
    out = []
    for k, ja in enumerate(ja_values):
        dT = ja * h_fg / cp
        out.append(wl.Case(f"paper_ja{ja:.3f}", nx=nx, ny=ny, wall_rows=heater_rows, top_bc="convective",
                           T_bottom_over_Tc=wl.TS_OVER_TC + dT / Tc, T_top_over_Tc=None, eos_T_fixed=False,
                           g_y=-wl.GRAVITY, Gw0=0.3, sites=sites))
    return out, h_fg, Tc


def paper_curve(ja_values, steps, cp=None, ckpt_dir=None, every=4096):
    """Run the Fig. 11 cases together (one batched launch per step) and return,
    per Jakob number, the quasi-steady wall heat flux (mean over the second
    half of the run), the heat transfer coefficient q / (T_w - Ts), the wall
    vapour coverage and its regime label.  With `ckpt_dir` the run goes
    through run_resumable: checkpoints every `every` steps, resumable per
    point, an unstable point retried once with N of Eq. (27) doubled."""
    cases, h_fg, Tc = paper_cases(ja_values, cp=cp)
    failed = [-1] * len(cases)
    if ckpt_dir is None:
        res, seconds = run_batched(cases, steps, hist_steps=0)
    else:
        t0 = time.perf_counter()
        res, failed = run_resumable(cases, steps, 0, ckpt_dir, every=every)
        seconds = time.perf_counter() - t0
    rows = []
    for ja, r, fa in zip(ja_values, res, failed):
        dT = r.superheat * Tc
        rows.append(dict(Ja=float(ja), superheat_over_Tc=r.superheat, q=r.q_qs, h=r.q_qs / dT,
                         coverage=r.coverage, regime=r.regime, n_sub=r.n_sub, failed_at=fa))
    return rows, seconds


# ------------------------------------------------------------------ surrogate at the sweep's scale
def _save_results(path, res):
    np.savez_compressed(path, history=np.stack([r.history for r in res]), q=[r.q_qs for r in res],
                        coverage=[r.coverage for r in res], regime=[r.regime for r in res])


def _load_results(path, pts):
    z = np.load(path)
    return [PointResult(c, c.T_bottom_over_Tc - wl.TS_OVER_TC, len(c.sites), z["history"][i], float(z["q"][i]),
                        float(z["coverage"][i]), int(z["regime"][i])) for i, c in enumerate(pts)]


def surrogate_study(n=256, full=40000, hist_steps=5000, seed=wl.BASE_SEED, n_fit=160, n_cal=48, members=4,
                    epochs=600, cache=None):
    """The learned early-stop policy on sweep points of the spec's scale: n
    square domains of sides 256-512 (3-9 sites, 25-row heater, superheats
    0.02-0.30 Tc), each run `full` steps in one batch, the first `hist_steps`
    steps of their wall-flux histories as the network input.  An ensemble is
    trained by the CUDA kernels on n_fit points, the acceptance threshold is
    calibrated on the next n_cal, and the policy is evaluated on the rest
    against their full runs.  Returns the numbers of the study (errors,
    accepted points, work fraction, batched seconds)."""
    import os
    from .surrogate import Ensemble
    pts = make_points(n, seed=seed)
    if cache and os.path.exists(cache):
        res, secs = _load_results(cache, pts), float("nan")
    else:
        res, secs = run_batched(pts, full, hist_steps)
        if cache:
            _save_results(cache, res)
    fit, cal, test = res[:n_fit], res[n_fit:n_fit + n_cal], res[n_fit + n_cal:]
    ens = Ensemble(members=members, seed=3, max_batch=max(n_fit, 64))
    L0 = ens.members[0].net.cfg.L0
    hist, scal, q, lab = features(fit, L0)
    losses = ens.fit(hist, scal, q, lab, epochs=epochs, batch=64, lr=1e-3)
    cells = [r.case.nx * r.case.ny for r in test]
    hist_t, scal_t, q_t, _ = features(test, L0)
    qp_t, spread_t, _ = ens.predict(hist_t, scal_t)
    err_all = np.abs(qp_t - q_t) / np.maximum(np.abs(q_t), 1e-12)
    policies = {}
    thr = choose_threshold(ens, cal, L0, tol=0.03)
    acc, err, cost = evaluate_policy(ens, test, L0, thr, hist_steps, full, cells)
    policies["score"] = dict(threshold=thr, accepted=int(acc.sum()), max_error=float(err.max()) if len(err) else 0.0,
                             work_fraction=cost)
    for kind in ("not_film", "no_boiling"):
        for tol in (0.03, 0.02):
            thr2, smax = choose_policy(ens, cal, L0, tol=tol, kind=kind)
            acc, err, cost = evaluate_policy(ens, test, L0, thr2, hist_steps, full, cells, spread_max=smax,
                                             kind=kind)
            policies[f"{kind}_spread_tol{tol}"] = dict(threshold=thr2, spread_max=smax, accepted=int(acc.sum()),
                                                       max_error=float(err.max()) if len(err) else 0.0,
                                                       work_fraction=cost)
    regimes = [r.regime for r in res]
    return dict(points=n, full_steps=full, hist_steps=hist_steps, batched_seconds=secs,
                cell_updates=float(sum(r.case.nx * r.case.ny for r in res)) * full,
                loss_first=[float(l[0].sum()) for l in losses], loss_last=[float(l[-1].sum()) for l in losses],
                held_out=len(test), held_out_median_error=float(np.median(err_all)),
                held_out_error_quartiles=[float(x) for x in np.percentile(err_all, [25, 75, 90])],
                policies=policies, regime_counts=[int(regimes.count(k)) for k in range(5)])


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Fig. 11 boiling curve at the paper's scale (400 x 600, 3 sites)")
    ap.add_argument("--steps", type=int, default=60000)
    ap.add_argument("--ja", type=str, default="0.05,0.07,0.093,0.11,0.13,0.15,0.166,0.176,0.186,0.197,0.21,0.22,0.25,0.3")
    ap.add_argument("--cp-eos", action="store_true", help="c_p of Ja: the saturated liquid's (default c_v)")
    ap.add_argument("--surrogate-study", action="store_true",
                    help="instead: the early-stop policy on 256 sweep points of sides 256-512 (40,000 steps)")
    ap.add_argument("--cache", type=str, default=None, help="npz of the study's runs (written once, then reused)")
    ap.add_argument("--checkpoint-dir", type=str, default=None,
                    help="checkpoint every point there and resume from it (per point) when run again")
    ap.add_argument("--checkpoint-every", type=int, default=4096)
    ap.add_argument("--train-policy", action="store_true",
                    help="instead: train the early-stop ensemble and freeze its policy (writes %s)" % POLICY_FILE)
    ap.add_argument("--pph-study", action="store_true", help="instead: measure points/hour in three arms")
    a = ap.parse_args()
    if a.train_policy:
        print(json.dumps({k: (v.item() if hasattr(v, "item") else v) for k, v in train_policy(cache=a.cache).items()}))
        raise SystemExit(0)
    if a.pph_study:
        print(json.dumps(pph_study()))
        raise SystemExit(0)
    if a.surrogate_study:
        print(json.dumps(surrogate_study(cache=a.cache)))
        raise SystemExit(0)
    cp = liquid_cp(hlb.default_params(8, 8)) if a.cp_eos else None
    rows, sec = paper_curve([float(x) for x in a.ja.split(",")], a.steps, cp=cp, ckpt_dir=a.checkpoint_dir,
                            every=a.checkpoint_every)
    for r in rows:
        print(json.dumps(r))
    print(json.dumps({"points": len(rows), "steps": a.steps, "seconds": sec}))
