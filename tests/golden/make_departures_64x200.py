"""Write tests/golden/departures_64x200.json: the bubble departures of a single
nucleation site (Section 4.3, Fig. 7) computed by the FP64 oracle alone.

The case: a 64 x 200 lattice with a 10-row heater at Ts + 0.11 Tc, one site
(g_min = -0.3) at a seeded x position, a vapour bubble of radius 12 seeded on
it, convective top, gravity 3e-5.  Densities every SNAP steps over STEPS
steps go through the oracle's departure detector (oracle/departure.py); the
four departures it sees (about 10,000 steps apart) and the wall heat flux
averaged over blocks of BLOCK steps are stored.  tests/test_physics_gpu.py
runs the same case on the GPU and compares.

Runs single-threaded for about eight minutes: python tests/golden/make_departures_64x200.py
"""
from __future__ import annotations

import dataclasses
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

STEPS = 45000
SNAP = 20
BLOCK = 1000
OUT = os.path.join(HERE, "departures_64x200.json")


def case_and_fields(rho_l: float, rho_v: float, Tc: float):
    """The seeded case and its initial fields (shared with the GPU test)."""
    case = wl.pool(nx=64, ny=200, n_sites=1, heater_rows=10, superheat=0.11, seed=5)
    case = dataclasses.replace(case, sites=[(case.sites[0][0], 10.0, -0.3)])
    rho0, T0 = wl.initial_fields(case, rho_l, rho_v, Tc)
    rho0 = rho_l + rho_v - wl.droplet(case.ny, case.nx, rho_l, rho_v, case.sites[0][0], case.wall_rows, 12.0)
    return case, rho0, T0


def main() -> None:
    pr = eos.PR()
    Ts = wl.TS_OVER_TC * pr.Tc
    rho_l, rho_v, _ = eos.coexistence(Ts, pr)
    case, rho0, T0 = case_and_fields(rho_l, rho_v, pr.Tc)
    p = Params(nx=case.nx, ny=case.ny, wall_rows=case.wall_rows, top_bc=case.top_bc,
               T_bottom=case.T_bottom(pr.Tc), T_top=case.T_top(pr.Tc), eos_T_fixed=case.eos_T_fixed,
               g_y=case.g_y, Gw=nucleation_Gw(case.nx, case.Gw0, case.sites), rho_l=rho_l, rho_v=rho_v)
    d = Domain(p, rho0, T0)
    prev, events, q_blocks, qs = None, [], [], 0.0
    t0 = time.time()
    for n in range(1, STEPS + 1):
        d.step(1)
        qs += d.last["q_bottom"]
        if n % SNAP == 0:
            if prev is not None:
                events += departure_steps([prev[0], d.rho], [prev[1], n], case.wall_rows, rho_l, rho_v)
            prev = (d.rho.copy(), n)
        if n % BLOCK == 0:
            q_blocks.append(qs / BLOCK)
            qs = 0.0
    out = {"_source": "tests/golden/make_departures_64x200.py (FP64 oracle only, single thread)",
           "case": {"nx": case.nx, "ny": case.ny, "wall_rows": case.wall_rows, "superheat_over_Tc": 0.11,
                    "site": list(case.sites[0]), "bubble_radius": 12.0, "seed": 5, "g_y": case.g_y},
           "steps": STEPS, "snapshot_every": SNAP, "block": BLOCK, "departure_steps": [int(e) for e in events],
           "q_bottom_block_means": q_blocks, "oracle_seconds": round(time.time() - t0, 1)}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: out[k] for k in ("departure_steps", "oracle_seconds")}))


if __name__ == "__main__":
    main()
