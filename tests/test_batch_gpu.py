"""Batched sweep (one launch for all domains per step) against single-domain
runs of the same kernel body: results must be bit-identical, including early
stop of one domain and reuse of a stopped slot."""
import dataclasses

import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, gpu_domain, ragged_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def coex():
    return coexistence()


def _cases():
    return [ragged_case(3), wl.film(nx=40, ny=60), dataclasses.replace(ragged_case(5), name="r70", nx=70, ny=50),
            wl.pool(nx=96, ny=64, n_sites=3, heater_rows=10)]


def _batch(cases, coex):
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    plist = [params_for(c, rho_l=coex["rho_l"], rho_v=coex["rho_v"])[0] for c in cases]
    b = hlb.Batch(plist)
    for i, c in enumerate(cases):
        rho0, T0 = wl.initial_fields(c, coex["rho_l"], coex["rho_v"], coex["Tc"])
        b.set_fields(i, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                     torch.tensor(T0, dtype=torch.float32, device="cuda"))
        b.set_nucleation_sites(i, c.sites)
    return b


def test_batch_matches_single_domains(coex):
    """A batch slot against the same domain alone.  The batched and the
    single-domain kernels are separate instantiations of the same device code
    and may round the last bit differently (FMA contraction), so they agree to
    FP32 rounding (_close), not bit for bit; bit-for-bit comparisons are batch
    against batch (tests/test_batch_refill_gpu.py, the two-lane test below)."""
    cases = _cases()
    b = _batch(cases, coex)
    b.step(40)  # two captured 16-step graphs + 8 direct launches
    for i, c in enumerate(cases):
        d = gpu_domain(c, coex)
        d.step(40)
        _close(b.read(i), d.read())
        hist = b.flux_history(i)
        assert len(hist) == 40
        assert hist[-1] == pytest.approx(d.diag().q_bottom, rel=1e-5, abs=1e-12)
        assert b.diag(i).step == 40


def test_stop_and_reuse_slot(coex):
    cases = _cases()
    b = _batch(cases, coex)
    b.step(20)
    b.stop(1)
    b.step(21)
    d = gpu_domain(cases[1], coex)
    d.step(20)
    _close(b.read(1), d.read())
    assert len(b.flux_history(1)) == 20
    assert b.diag(0).step == 41
    # restart slot 1 from fresh fields while the batch is at odd parity
    rho0, T0 = wl.initial_fields(cases[1], coex["rho_l"], coex["rho_v"], coex["Tc"])
    import torch
    b.set_fields(1, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                 torch.tensor(T0, dtype=torch.float32, device="cuda"))
    b.step(7)
    d2 = gpu_domain(cases[1], coex)
    d2.step(7)
    _close(b.read(1), d2.read())
    assert b.diag(1).step == 7


def test_steps_with_every_slot_stopped_change_nothing(coex):
    """The empty case of the early-stop path: with every slot stopped a step
    launches blocks that all return at once.  Fields, checkpoints (state,
    outlet memory and history) and step counters stay as they were, bit for
    bit, no error is raised, and a slot refilled afterwards runs as a fresh
    batch does."""
    import torch
    cases = _cases()
    b = _batch(cases, coex)
    b.step(9)  # odd: the batch stops at buffer parity 1
    for i in range(len(cases)):
        b.stop(i)
    before = [([t.cpu().numpy() for t in b.read(i)], b.checkpoint(i), b.diag(i).step) for i in range(len(cases))]
    b.step(37)  # two captured graphs and five direct launches over stopped slots
    for i in range(len(cases)):
        fields, ck, step = before[i]
        for x, y in zip(fields, b.read(i)):
            assert np.array_equal(x, y.cpu().numpy()), i
        assert b.checkpoint(i) == ck and b.diag(i).step == step == 9
        assert b.diag(i).error_flags == 0
    rho0, T0 = wl.initial_fields(cases[2], coex["rho_l"], coex["rho_v"], coex["Tc"])
    b.set_fields(2, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                 torch.tensor(T0, dtype=torch.float32, device="cuda"))
    b.set_nucleation_sites(2, cases[2].sites)
    b.step(11)
    fresh = _batch(cases, coex)
    fresh.step(11)
    for x, y in zip(b.read(2), fresh.read(2)):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())
    assert b.diag(2).step == 11 and b.diag(0).step == 9


def test_batch_of_one_domain(coex):
    """The smallest batch: one domain (one lane, no lane split) against the
    same domain alone, through graph replay and direct launches."""
    case = _cases()[3]
    b = _batch([case], coex)
    b.step(35)
    d = gpu_domain(case, coex)
    d.step(35)
    _close(b.read(0), d.read())
    assert b.diag(0).step == 35 and len(b.flux_history(0)) == 35


def _close(fields, ref):
    """Two kernel variants evaluate a cell's update with the same arithmetic but
    may round differently (tiled and row-marching kernels) and sum the FP64
    partials in another order: rho and T agree to 1e-6 of their maxima, u to
    1e-6 in lattice units (2e-6 of the sound speed; the parity tolerance
    against the FP64 oracle is 1e-5 of it)."""
    for k, (x, y) in enumerate(zip(fields, ref)):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy()
        tol = 1e-6 if k in (1, 2) else 1e-6 * max(np.abs(y).max(), 1e-30)
        assert np.abs(x - y).max() <= tol, ("rho ux uy T".split()[k], np.abs(x - y).max())


def test_autotune_picks_a_variant_and_keeps_results(coex):
    """The timed autotuning steps are ordinary steps: fields after autotune + k
    steps match an untuned run of the same length to FP32 rounding."""
    from paper_1812_10375_gb300 import hlb
    cases = _cases()
    a = _batch(cases, coex)
    b = _batch(cases, coex)
    nv = len(hlb.tile_variants())
    chosen, ms = a.autotune(steps_per_variant=4)
    assert 0 <= chosen < nv and len(ms) == nv and all(m > 0 for m in ms)
    assert ms[chosen] == min(ms)
    a.step(20)
    b.step(5 * nv + 20)
    for i in range(len(cases)):
        assert a.diag(i).step == b.diag(i).step == 5 * nv + 20
        _close(a.read(i), b.read(i))


def test_set_tile_variant_keeps_fields(coex):
    """Each compiled variant, selected directly, advances the fields like the
    default one, to FP32 rounding."""
    from paper_1812_10375_gb300 import hlb
    cases = _cases()
    ref = _batch(cases, coex)
    ref.step(9)
    nv = len(hlb.tile_variants())
    for v in range(nv):
        b = _batch(cases, coex)
        b.set_tile_variant(v)
        b.step(4)
        b.set_tile_variant((v + 1) % nv)
        b.step(5)
        for i in range(len(cases)):
            assert b.diag(i).step == 9
            _close(b.read(i), ref.read(i))
        with pytest.raises(hlb.HlbError):
            b.set_tile_variant(nv)
        b.close()


def test_nonfinite_input_is_reported_and_blocks_steps(coex):
    """A NaN injected on the host into the initial temperature sets the device
    error word: hlb_diag returns HLB_EUNSTABLE and further steps HLB_ESTATE
    (no GPU fault, the context stays usable)."""
    import torch
    from paper_1812_10375_gb300 import hlb
    from paper_1812_10375_gb300.config import params_for
    case = ragged_case()
    p, Tc = params_for(case, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    d = hlb.Domain(p)
    rho0, T0 = wl.initial_fields(case, coex["rho_l"], coex["rho_v"], Tc)
    T0[20, 10] = np.nan
    d.set_fields(torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                 torch.tensor(T0, dtype=torch.float32, device="cuda"))
    d.step(3)
    with pytest.raises(hlb.HlbError) as e:
        d.diag()
    assert e.value.status == hlb.HLB_EUNSTABLE
    assert d.diag(check_flags=False).error_flags & 1
    with pytest.raises(hlb.HlbError) as e2:
        d.step(1)
    assert e2.value.status == hlb.HLB_ESTATE
    # the context is still usable: a fresh domain steps normally
    ok = gpu_domain(case, coex)
    ok.step(5)
    assert ok.diag().error_flags == 0


def test_two_lanes_match_one_lane_bit_for_bit(coex):
    """The two-lane split step (hlb_batch_set_lanes) only reorders launches of
    independent domains: 37 steps (two captured graphs, direct steps at both
    parities), a slot stopped and refilled half way, give the one-lane fields,
    diagnostics and flux histories bit for bit."""
    import torch
    from paper_1812_10375_gb300 import hlb
    cases = _cases()
    runs = []
    for lanes in (1, 2):
        b = _batch(cases, coex)
        b.set_lanes(lanes)
        b.step(19)
        b.stop(2)
        b.step(3)
        rho0, T0 = wl.initial_fields(cases[2], coex["rho_l"], coex["rho_v"], coex["Tc"])
        b.set_fields(2, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                     torch.tensor(T0, dtype=torch.float32, device="cuda"))
        b.step(15)
        runs.append([([t.cpu().numpy() for t in b.read(i)], b.diag(i), b.flux_history(i)) for i in range(len(cases))])
        b.close()
    for i, ((f1, d1, h1), (f2, d2, h2)) in enumerate(zip(*runs)):
        for x, y in zip(f1, f2):
            assert np.array_equal(x, y), cases[i].name
        assert d1 == d2 and np.array_equal(h1, h2), cases[i].name
    assert runs[0][2][1].step == 15 and runs[0][0][1].step == 37
    with pytest.raises(hlb.HlbError):
        _batch(cases[:1], coex).set_lanes(3)
