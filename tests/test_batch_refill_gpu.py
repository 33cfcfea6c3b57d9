"""Slot refill in a batch: a sweep that runs more points than the batch has
slots gives a finished slot the next point of the same size (set_wall,
set_fields, the nucleation sites) while the other slots carry on, at any step
parity.  The refilled slot must then evolve bit for bit as that point does in a
fresh batch, and the slot that carried on as if nothing had happened.

(A batch slot and a single domain agree to FP32 rounding, not bit for bit: the
batched and single-domain kernels are separate instantiations whose last bits
may differ, and a one-ulp difference in T grows to ~1e-5 of max|u| within
fifty steps of a starting flow.  The reference is therefore a batch.)"""
import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build
    build.build()


def _fields(rho0, T0):
    import torch
    return (torch.tensor(rho0, dtype=torch.float32, device="cuda"),
            torch.tensor(T0, dtype=torch.float32, device="cuda"))


def _slot(bt, i):
    return [t.cpu().numpy() for t in bt.read(i)], bt.diag(i), bt.flux_history(i)


def _fresh(cases_params, Tc, steps, slot):
    """Slot `slot` of a fresh batch of the given points after `steps` steps."""
    from paper_1812_10375_gb300 import hlb
    bt = hlb.Batch([p for _, p in cases_params])
    for i, (case, p) in enumerate(cases_params):
        bt.set_fields(i, *_fields(*wl.initial_fields(case, p.rho_l, p.rho_v, Tc)))
        bt.set_nucleation_sites(i, case.sites)
    bt.step(steps)
    out = _slot(bt, slot)
    bt.close()
    return out


def _same(a, b, what):
    (fa, da, ha), (fb, db, hb) = a, b
    for k, (x, y) in enumerate(zip(fa, fb)):
        assert np.array_equal(x, y), (what, "rho ux uy T".split()[k], float(np.abs(x - y).max()))
    assert da.step == db.step and da.error_flags == 0 == db.error_flags, what
    assert (da.mass, da.q_bottom, da.rho_ave) == (db.mass, db.q_bottom, db.rho_ave), what
    assert np.array_equal(ha, hb), what


@pytest.mark.parametrize("first", [37, 48])
def test_refilled_slot_matches_a_fresh_batch(first):
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    coex = coexistence()
    a = wl.pool(nx=96, ny=80, n_sites=2, heater_rows=10, superheat=0.05, seed=wl.BASE_SEED + 1)
    b = wl.pool(nx=96, ny=80, n_sites=3, heater_rows=10, superheat=0.2, seed=wl.BASE_SEED + 2)
    c = wl.pool(nx=96, ny=80, n_sites=1, heater_rows=10, superheat=0.12, seed=wl.BASE_SEED + 3)
    pa, Tc = params_for(a, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    pb, _ = params_for(b, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    pc, _ = params_for(c, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    later = 50
    bt = hlb.Batch([pa, pb])
    for i, (case, p) in enumerate(((a, pa), (b, pb))):
        bt.set_fields(i, *_fields(*wl.initial_fields(case, p.rho_l, p.rho_v, Tc)))
        bt.set_nucleation_sites(i, case.sites)
    bt.step(first)
    # slot 0 finishes point a and takes point c
    bt.set_wall(0, pc.T_bottom)
    bt.set_fields(0, *_fields(*wl.initial_fields(c, pc.rho_l, pc.rho_v, Tc)))
    bt.set_nucleation_sites(0, c.sites)
    bt.step(later)
    got_c, got_b = _slot(bt, 0), _slot(bt, 1)
    bt.close()
    _same(got_c, _fresh([(c, pc), (b, pb)], Tc, later, 0), ("refilled slot", first))
    _same(got_b, _fresh([(a, pa), (b, pb)], Tc, first + later, 1), ("slot that carried on", first))
