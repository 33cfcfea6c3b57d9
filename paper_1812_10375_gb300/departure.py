"""Bubble-departure events from density snapshots of a boiling run.

The paper reads bubble departure and waiting periods off snapshot sequences and
the periodicity of the wall heat flux (Section 4.3, Figs. 7 and 10) without
defining a detector.  This module fixes one, used alike on the GPU fields and on
the FP64 reference fields so the two runs' departure statistics can be
compared:

* vapour is the set of fluid nodes with rho < (rho_l + rho_v) / 2;
* a bubble is a 4-connected vapour component (periodic in x);
* a bubble is attached when it has a node in the first fluid row above the
  heater (y = wall_rows);
* a departure happens between snapshots k - 1 and k when a detached bubble of
  snapshot k covers nodes of a bubble that was attached at k - 1 and none of
  a bubble that was already detached (it left the wall, or pinched off from
  an attached bubble, in that interval; a bubble rising from an earlier
  departure is not counted again).  Each such component counts once, at the
  column of its centroid.  Snapshots must be close enough in time that a
  bubble overlaps its own earlier position.

The departure period is the mean interval between successive events.  This is
analysis of stored snapshots on the host (numpy / scipy), not part of the
time step.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _label_periodic(mask: np.ndarray):
    """4-connected components of a 2-D boolean mask that is periodic in x
    (axis 1).  Returns (labels, n) with labels 1..n, 0 for background."""
    from scipy import ndimage
    lab, n = ndimage.label(mask)
    if n == 0:
        return lab, 0
    # join components that meet across the x boundary
    parent = list(range(n + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    left, right = lab[:, 0], lab[:, -1]
    for a, b in zip(left, right):
        if a and b:
            ra, rb = find(int(a)), find(int(b))
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(k) for k in range(n + 1)])
    uniq = np.unique(roots[1:])
    remap = np.zeros(n + 1, dtype=np.int64)
    remap[uniq] = np.arange(1, len(uniq) + 1)
    return remap[roots][lab], len(uniq)


@dataclass
class Departures:
    """Departure events of a snapshot sequence."""

    times: np.ndarray    # step of the snapshot at which each event was seen
    columns: np.ndarray  # x centroid of the departed bubble (periodic mean)

    @property
    def count(self) -> int:
        return int(len(self.times))

    def period(self) -> float:
        """Mean interval between successive events (nan with fewer than two)."""
        t = np.sort(self.times)
        return float(np.mean(np.diff(t))) if len(t) >= 2 else float("nan")


def _periodic_centroid(xs: np.ndarray, nx: int) -> float:
    ang = 2.0 * np.pi * xs / nx
    a = np.arctan2(np.sin(ang).mean(), np.cos(ang).mean())
    return float((a % (2.0 * np.pi)) * nx / (2.0 * np.pi))


def detect(snapshots, steps, wall_rows: int, rho_l: float, rho_v: float) -> Departures:
    """Departure events of a sequence of density fields (ny x nx arrays, rows
    from the bottom) taken at the given steps."""
    mid = 0.5 * (rho_l + rho_v)
    times, cols = [], []
    prev_lab, prev_att = None, None
    for rho, step in zip(snapshots, steps):
        fluid = np.asarray(rho, dtype=np.float64)[wall_rows:]
        lab, n = _label_periodic(fluid < mid)
        attached = np.zeros(n + 1, dtype=bool)
        attached[np.unique(lab[0][lab[0] > 0])] = True
        if prev_lab is not None:
            for c in range(1, n + 1):
                if attached[c]:
                    continue
                cells = lab == c
                # labels of the previous snapshot under this bubble
                under = np.unique(prev_lab[cells])
                under = under[under > 0]
                if len(under) and prev_att[under].any() and prev_att[under].all():
                    ys, xs = np.nonzero(cells)
                    times.append(step)
                    cols.append(_periodic_centroid(xs, fluid.shape[1]))
        prev_lab, prev_att = lab, attached
    return Departures(np.asarray(times, dtype=np.int64), np.asarray(cols, dtype=np.float64))
