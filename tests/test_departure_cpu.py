"""The bubble-departure detector on synthetic snapshot sequences whose events
are known by construction: discs of vapour in liquid that sit on the wall,
rise, leave it and pinch off, including a bubble that straddles the periodic x
boundary and an old bubble rising past a new one."""
import numpy as np

from paper_1812_10375_gb300 import departure

RL, RV = 6.5, 0.38
W = 4  # wall rows below the fluid


def frame(nx, ny, discs):
    """Liquid with vapour discs (xc, yc, r) in lattice coordinates (y includes the wall rows)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    rho = np.full((ny, nx), RL)
    for xc, yc, r in discs:
        dx = np.abs(x - xc)
        dx = np.minimum(dx, nx - dx)  # periodic in x
        rho[(dx ** 2 + (y - yc) ** 2) <= r * r] = RV
    rho[:W] = 0.0  # solid rows carry no density
    return rho


def test_single_bubble_leaves_the_wall_once():
    nx, ny = 40, 60
    # the bubble sits on the wall (touches row W) until step 60, then rises
    centres = [W + 3, W + 3, W + 4, W + 5, W + 9, W + 12, W + 16, W + 20]
    snaps = [frame(nx, ny, [(20, yc, 5)]) for yc in centres]
    steps = [20 * (k + 1) for k in range(len(snaps))]
    dep = departure.detect(snaps, steps, W, RL, RV)
    assert dep.count == 1
    assert dep.times[0] == 100  # first snapshot whose bubble no longer reaches row W (centre W + 9 > r)
    assert abs(dep.columns[0] - 20) < 0.5


def test_bubble_across_the_periodic_boundary_is_one_bubble():
    nx, ny = 40, 60
    centres = [W + 2, W + 3, W + 10, W + 14]
    snaps = [frame(nx, ny, [(0, yc, 6)]) for yc in centres]
    dep = departure.detect(snaps, [1, 2, 3, 4], W, RL, RV)
    assert dep.count == 1 and dep.times[0] == 3
    c = dep.columns[0]
    assert min(c, nx - c) < 0.5  # centroid at x = 0, not at the middle of the two halves


def test_rising_bubble_is_not_counted_again_and_period_is_mean_interval():
    nx, ny = 40, 80
    snaps, steps = [], []
    # bubble A departs between steps 10 and 20, bubble B grows under it and
    # departs between steps 50 and 60 while A is still rising above it
    seq = [
        [(20, W + 3, 5)],
        [(20, W + 9, 5)],
        [(20, W + 12, 5), (20, W + 1, 3)],
        [(20, W + 16, 5), (20, W + 2, 4)],
        [(20, W + 21, 5), (20, W + 3, 5)],
        [(20, W + 26, 5), (20, W + 9, 5)],
        [(20, W + 31, 5), (20, W + 13, 5)],
    ]
    for k, discs in enumerate(seq):
        snaps.append(frame(nx, ny, discs))
        steps.append(10 * k)
    dep = departure.detect(snaps, steps, W, RL, RV)
    assert list(dep.times) == [10, 50]
    assert dep.period() == 40.0


def test_no_vapour_no_events():
    snaps = [frame(32, 40, []) for _ in range(4)]
    dep = departure.detect(snaps, [0, 1, 2, 3], W, RL, RV)
    assert dep.count == 0 and np.isnan(dep.period())
