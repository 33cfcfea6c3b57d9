"""Bubble-departure events of a density-snapshot sequence: the oracle's own
statement of the detector (test infrastructure; shares no code with the GPU
library or its host tools).

The paper reads departure and waiting periods off snapshot sequences
(Section 4.3, Figs. 7 and 10) without a formal definition.  The definition
used here:

* vapour: fluid nodes with rho below the mean of the coexistence densities;
* bubble: a 4-connected vapour component, x periodic;
* attached: the bubble has a node in the first fluid row (y = wall_rows);
* departure between snapshots k - 1 and k: a bubble of snapshot k that is not
  attached, lies over at least one node of a bubble that was attached at
  k - 1, and over no node of a bubble that was already detached at k - 1.

Parity unpinned beyond the synthetic sequences of tests/test_departure_cpu.py:
the paper gives no event list to compare with.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage


def periodic_components(mask: np.ndarray):
    """Labels 1..n of the 4-connected components of `mask` (rows y, columns x),
    with components that touch across the x = 0 / x = nx - 1 seam merged."""
    lab, n = ndimage.label(mask)
    if n == 0:
        return lab, 0
    root = np.arange(n + 1)

    def top(a):
        while root[a] != a:
            a = root[a]
        return a

    for a, b in zip(lab[:, 0], lab[:, -1]):
        if a and b:
            ra, rb = top(a), top(b)
            if ra != rb:
                root[max(ra, rb)] = min(ra, rb)
    final = np.array([top(a) for a in range(n + 1)])
    kept = np.unique(final[1:])
    renumber = np.zeros(n + 1, dtype=np.int64)
    renumber[kept] = np.arange(1, kept.size + 1)
    return renumber[final][lab], int(kept.size)


def departure_steps(snapshots, steps, wall_rows: int, rho_l: float, rho_v: float) -> list[int]:
    """Steps at which departures are first seen (one entry per departed bubble)."""
    threshold = 0.5 * (rho_l + rho_v)
    events: list[int] = []
    before = None
    for rho, step in zip(snapshots, steps):
        lab, n = periodic_components(np.asarray(rho, dtype=np.float64)[wall_rows:] < threshold)
        attached = np.zeros(n + 1, dtype=bool)
        attached[lab[0][lab[0] > 0]] = True
        if before is not None:
            lab0, att0 = before
            for c in range(1, n + 1):
                if attached[c]:
                    continue
                under = np.unique(lab0[lab == c])
                under = under[under > 0]
                if under.size and att0[under].all():
                    events.append(int(step))
        before = (lab, attached)
    return events
