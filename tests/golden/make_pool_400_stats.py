"""Write tests/golden/pool_400_stats.json (and pool_400_sh012_stats.json):
boiling statistics of the 400 x 400 pool (25-row heater at Ts + 0.1 Tc, or
0.12 Tc, five seeded nucleation sites, convective
top, gravity 3e-5; Section 4.2 geometry at the pool size of the benchmark
configurations) computed by the FP64 oracle alone.

Stored: the wall heat flux q_bottom of every step averaged over blocks of
BLOCK steps, the first-fluid-row vapour coverage over the same blocks, and the
steps at which the oracle's departure detector (oracle/departure.py) sees a
bubble leave the wall, from density snapshots every SNAP steps.  The GPU test
(tests/test_pool_stats_gpu.py) runs the same case and compares time averages
and the departure period with these values (Sections 4.3-4.4).

Runs single-threaded, about 2.5 hours at 0.1 Tc and 80 minutes at 0.12 Tc:
python tests/golden/make_pool_400_stats.py [0.1 | 0.12]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import Domain, Params, eos, nucleation_Gw  # noqa: E402
from oracle.departure import departure_steps  # noqa: E402
from paper_1812_10375_gb300 import workloads as wl  # noqa: E402  (seeded inputs only)

BLOCK = 1000
SNAP = 20
# superheat / Tc -> (output file, steps): the benchmark's pool at 0.1 Tc (its
# bubbles stop departing after three), and the same pool at 0.12 Tc, whose
# first 32,000 steps hold more than four departures
RUNS = {0.1: ("pool_400_stats.json", 60000), 0.12: ("pool_400_sh012_stats.json", 32000)}


def main(superheat: float = 0.1) -> None:
    name, steps = RUNS[superheat]
    out_path = os.path.join(HERE, name)
    pr = eos.PR()
    Ts = wl.TS_OVER_TC * pr.Tc
    rho_l, rho_v, _ = eos.coexistence(Ts, pr)
    case = wl.pool(superheat=superheat)
    rho0, T0 = wl.initial_fields(case, rho_l, rho_v, pr.Tc)
    p = Params(nx=case.nx, ny=case.ny, wall_rows=case.wall_rows, top_bc=case.top_bc,
               T_bottom=case.T_bottom(pr.Tc), T_top=case.T_top(pr.Tc), eos_T_fixed=case.eos_T_fixed,
               g_y=case.g_y, Gw=nucleation_Gw(case.nx, case.Gw0, case.sites), rho_l=rho_l, rho_v=rho_v)
    d = Domain(p, rho0, T0)
    q_blocks, cov_blocks = [], []
    qs, covs = 0.0, 0.0
    snaps, snap_steps, events = [], [], []
    t0 = time.time()
    for n in range(1, steps + 1):
        d.step(1)
        qs += d.last["q_bottom"]
        covs += d.last["vapour_coverage"]
        if n % SNAP == 0:
            snaps.append(d.rho.copy())
            snap_steps.append(n)
            if len(snaps) > 1:
                # the detector compares consecutive snapshots: feed it the last two
                events += departure_steps(snaps[-2:], snap_steps[-2:], case.wall_rows, rho_l, rho_v)
                snaps, snap_steps = snaps[-1:], snap_steps[-1:]
        if n % BLOCK == 0:
            q_blocks.append(qs / BLOCK)
            cov_blocks.append(covs / BLOCK)
            qs = covs = 0.0
            write(out_path, case, superheat, steps, q_blocks, cov_blocks, events, n, time.time() - t0)
            print(f"step {n}: q {q_blocks[-1]:.6e} coverage {cov_blocks[-1]:.4f} departures {events}",
                  flush=True)


def write(out_path, case, superheat, steps, q_blocks, cov_blocks, events, done, seconds) -> None:
    out = {
        "_source": f"tests/golden/make_pool_400_stats.py {superheat} (FP64 oracle only, single thread)",
        "case": {"nx": case.nx, "ny": case.ny, "wall_rows": case.wall_rows, "top_bc": case.top_bc,
                 "superheat_over_Tc": superheat, "sites": case.sites, "seed": wl.BASE_SEED, "g_y": case.g_y},
        "steps_planned": steps, "steps_done": done, "block": BLOCK, "snapshot_every": SNAP,
        "q_bottom_block_means": q_blocks, "vapour_coverage_block_means": cov_blocks,
        "departure_steps": events, "oracle_seconds": round(seconds, 1),
    }
    tmp = out_path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(out, fh, indent=1)
    os.replace(tmp, out_path)


if __name__ == "__main__":
    main(float(sys.argv[1]) if len(sys.argv) > 1 else 0.1)
