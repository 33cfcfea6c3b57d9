"""The step must not read workspace memory that it has not written: a domain
or batch whose workspace starts out as all-ones bytes (a NaN in every float
and double) must give bit for bit the fields and diagnostics of one whose
workspace starts out zeroed.  A caller's memory pool hands out blocks that
held anything before, for instance the NaN state of a sweep point that blew
up, and the library documents no requirement on the workspace's contents.

Every compiled variant (split, fused tile, row-marching) runs each case with
N = 1, 2 and 3 energy sub-steps (Eq. 27)."""
import dataclasses

import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, ragged_case

pytestmark = pytest.mark.gpu
STEPS = 6


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def coex():
    return coexistence()


CASES = {
    "pool": lambda: wl.pool(nx=64, ny=64, n_sites=2, heater_rows=10, seed=wl.BASE_SEED + 9),
    "ragged": lambda: ragged_case(3),
    "film": lambda: wl.film(nx=72, ny=60),
}


def _filled(byte, make):
    """Run make() with every uint8 CUDA tensor torch.empty returns filled with byte."""
    import torch
    real = torch.empty

    def empty(*a, **k):
        t = real(*a, **k)
        if t.dtype == torch.uint8 and t.is_cuda:
            t.fill_(byte)
        return t

    torch.empty = empty
    try:
        return make()
    finally:
        torch.empty = real


def _state(obj, i=None):
    import torch
    fields = obj.read() if i is None else obj.read(i)
    dg = obj.diag(check_flags=False) if i is None else obj.diag(i, check_flags=False)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in fields], dg


def _same(a, b, what):
    (fa, da), (fb, db) = a, b
    assert da.error_flags == 0 and db.error_flags == 0, (what, da.error_flags, db.error_flags)
    for k, (x, y) in enumerate(zip(fa, fb)):
        assert np.array_equal(x, y), (what, "rho ux uy T".split()[k], float(np.nanmax(np.abs(x - y))))
    assert dataclasses.astuple(da) == dataclasses.astuple(db), what


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("N", [1, 2, 3])
def test_domain_ignores_workspace_contents(coex, name, N):
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    case = CASES[name]()
    p, Tc = params_for(case, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    p.n_sub = N
    rho0, T0 = wl.initial_fields(case, coex["rho_l"], coex["rho_v"], Tc)
    rho0 = torch.tensor(rho0, dtype=torch.float32, device="cuda")
    T0 = torch.tensor(T0, dtype=torch.float32, device="cuda")
    kinds = hlb.variant_kinds()
    for v in range(len(kinds)):
        runs = []
        for byte in (0x00, 0xFF):
            d = _filled(byte, lambda: hlb.Domain(p))
            d.set_tile_variant(v)
            d.set_fields(rho0, T0)
            d.set_nucleation_sites(case.sites)
            d.step(STEPS)
            runs.append(_state(d))
            d.close()
        _same(runs[0], runs[1], (name, N, v, kinds[v]))


@pytest.mark.parametrize("N", [1, 2])
def test_batch_ignores_workspace_contents(coex, N):
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    cases = [c() for c in CASES.values()]
    plist = []
    for c in cases:
        p, _ = params_for(c, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
        p.n_sub = N
        plist.append(p)
    runs = []
    for byte in (0x00, 0xFF):
        b = _filled(byte, lambda: hlb.Batch(plist))
        for i, c in enumerate(cases):
            rho0, T0 = wl.initial_fields(c, coex["rho_l"], coex["rho_v"], coex["Tc"])
            b.set_fields(i, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                         torch.tensor(T0, dtype=torch.float32, device="cuda"))
            b.set_nucleation_sites(i, c.sites)
        b.step(STEPS)
        runs.append([_state(b, i) for i in range(len(cases))])
        b.close()
    for i, c in enumerate(cases):
        _same(runs[0][i], runs[1][i], (c.name, N))


def _run_fresh(case, coex, v, N, steps):
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    p, Tc = params_for(case, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    p.n_sub = N
    d = hlb.Domain(p)
    d.set_tile_variant(v)
    rho0, T0 = wl.initial_fields(case, coex["rho_l"], coex["rho_v"], Tc)
    d.set_fields(torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                 torch.tensor(T0, dtype=torch.float32, device="cuda"))
    d.set_nucleation_sites(case.sites)
    d.step(steps)
    out = _state(d)
    d.close()
    return out


def _blow_up(coex, v):
    """Step a 512 x 2048 pool whose heater diffusivity (0.9) is far beyond RK4's
    bound at N = 1 (0.35), from temperatures with a random 1e-3 Tc ripple that
    seeds the unstable checkerboard mode, until it is NaN: its kernels, on every
    SM, leave NaNs in shared memory."""
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    case = wl.pool(nx=512, ny=2048, n_sites=4, heater_rows=10, seed=wl.BASE_SEED + 9)
    p, Tc = params_for(case, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    p.lambda_w = 0.9 * 3.0 * p.rho_l * p.cv
    p.n_sub = 1
    d = hlb.Domain(p)
    d.set_tile_variant(v)
    rho0, T0 = wl.initial_fields(case, coex["rho_l"], coex["rho_v"], Tc)
    T0 = T0 + 1e-3 * Tc * np.random.default_rng(5).standard_normal(T0.shape)
    d.set_fields(torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                 torch.tensor(T0, dtype=torch.float32, device="cuda"))
    d.step(64)
    flags = d.diag(check_flags=False).error_flags
    torch.cuda.synchronize()
    d.close()
    return flags


@pytest.mark.parametrize("N", [1, 2])
def test_step_after_a_run_that_blew_up(coex, N):
    """Shared memory keeps what the last kernel on an SM left there.  A domain
    stepped right after one that went NaN (a sweep point that is retried with
    more sub-steps, say) must match the same domain stepped before it, bit for
    bit, with no error flag: no kernel may read a shared-memory slot it has not
    written, not even to multiply it by zero."""
    from paper_1812_10375_gb300 import hlb
    case = CASES["pool"]()
    for v in range(len(hlb.variant_kinds())):
        ref = _run_fresh(case, coex, v, N, 2)
        assert _blow_up(coex, v) != 0
        _same(ref, _run_fresh(case, coex, v, N, 2), ("after NaN", N, v))
