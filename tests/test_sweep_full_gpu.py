"""The benchmark's own configuration against the FP64 oracle: the 32-domain
boiling-curve sweep (sides 256-512, 3-9 sites, superheats 0.02-0.30 Tc) in one
batch, with the variant the warm-up autotuner picks and the step replayed from
captured graphs, as bench.py times it.

The oracle cannot run 32 domains of up to 262,144 cells for thousands of steps
in a test, but its step is a function of the state a domain carries, so it can
take one step from the GPU's own state: after 1000 GPU steps (bubbles have
nucleated on the hotter walls) every domain's checkpoint gives the stored
populations, T and the outlet memory, hlb_batch_diag the lagged mean density
and outlet velocity; the oracle steps once from there in FP64 and the GPU's
next step must agree cell by cell, every cell of every domain: rho and T to
1e-5 of their maxima, u to 1e-5 of the sound speed (one step of FP32 rounding
against FP64 from the same FP32 state)."""
import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, oracle_domain

pytestmark = pytest.mark.gpu
TOL = 1e-5
CS = 1.0 / np.sqrt(3.0)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
HEADER = 512  # checkpoint header bytes (include/hlb.h)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build
    build.build()


def _state(blob, nx, ny, rho_ref):
    """Populations (plain form), T^{n+1} and the outlet memory from a checkpoint."""
    n = nx * ny
    a = np.frombuffer(blob, dtype=np.float32, offset=HEADER)
    fs = a[:9 * n].astype(np.float64).reshape(9, ny, nx) + W9[:, None, None] * rho_ref
    T = a[9 * n:10 * n].astype(np.float64).reshape(ny, nx)
    ftop = a[11 * n:11 * n + 3 * nx].astype(np.float64).reshape(3, nx) + W9[[4, 7, 8], None] * rho_ref
    return fs, T, ftop


def test_sweep_step_matches_oracle_from_its_own_state():
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    coex = coexistence()
    cases = wl.sweep()
    plist = [params_for(c, rho_l=coex["rho_l"], rho_v=coex["rho_v"])[0] for c in cases]
    b = hlb.Batch(plist)
    for i, c in enumerate(cases):
        rho0, T0 = wl.initial_fields(c, coex["rho_l"], coex["rho_v"], coex["Tc"])
        b.set_fields(i, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                     torch.tensor(T0, dtype=torch.float32, device="cuda"))
        b.set_nucleation_sites(i, c.sites)
    chosen, _ = b.autotune(steps_per_variant=4)
    b.step(1000 - (b.diag(0).step % 1000))
    states = []
    for i, c in enumerate(cases):
        dg = b.diag(i)
        rho_ref = float(plist[i].rho_v) if plist[i].storage == hlb.HLB_STORE_DEVIATION else 0.0
        states.append((_state(b.checkpoint(i), c.nx, c.ny, rho_ref), dg))
    b.step(1)
    worst = dict(rho=0.0, u=0.0, T=0.0)
    boiling = 0
    for i, c in enumerate(cases):
        (fs, T, ftop), dg = states[i]
        od = oracle_domain(c, coex)
        od.fs = np.where(od.fluid[None], fs, 0.0)
        od.T = T
        od.f_top_prev = ftop
        od.rho_ave = dg.rho_ave
        od.U = max(0.0, dg.u_top)
        od.step(1)
        rho_g, ux_g, uy_g, T_g = [t.cpu().numpy().astype(np.float64) for t in b.read(i)]
        fl = od.fluid
        e_rho = np.abs(rho_g - od.rho)[fl].max() / np.abs(od.rho[fl]).max()
        e_T = np.abs(T_g - od.T).max() / np.abs(od.T).max()
        e_u = max(np.abs(ux_g - od.ux)[fl].max(), np.abs(uy_g - od.uy)[fl].max()) / CS
        worst = {k: max(worst[k], v) for k, v in (("rho", e_rho), ("u", e_u), ("T", e_T))}
        boiling += int((od.rho[c.wall_rows] < 0.5 * (coex["rho_l"] + coex["rho_v"])).any())
        assert max(e_rho, e_T, e_u) < TOL, (c.name, e_rho, e_u, e_T)
        assert b.diag(i).step == dg.step + 1 and b.diag(i).error_flags == 0
    print(f"32-domain sweep, variant {chosen}, step 1001 from the GPU's own state: worst {worst}; "
          f"{boiling} domains with vapour on the wall")
    assert boiling > 0  # the check covers bubbles on the wall, not only conduction
