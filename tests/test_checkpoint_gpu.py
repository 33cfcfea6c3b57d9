"""Checkpoint / resume through the C ABI: a domain restored from a checkpoint
steps to bit-for-bit the states of the domain it was taken from (single
domains, batch slots at either buffer parity; across the two, the restored
fields read back bit for bit and the two kernels then agree to FP32 rounding), the
restored fields and diagnostics read back unchanged, mismatched or damaged
checkpoints are refused without touching the domain, and the resumable sweep
driver, cut short by a host-side exception, ends with the results of an
uninterrupted sweep."""
import dataclasses

import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, gpu_domain, ragged_case

pytestmark = pytest.mark.gpu

DIAG_FIELDS = ("step", "mass", "energy", "q_bottom", "q_top", "q_interface", "rho_ave", "u_top",
               "q_bottom_timeavg", "error_flags", "vapour_coverage", "vapour_coverage_timeavg")


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def coex():
    return coexistence()


def _same_fields(a, b):
    for k, (x, y) in enumerate(zip(a, b)):
        assert (x == y).all(), "rho ux uy T".split()[k]


def _same_diag(a, b):
    for f in DIAG_FIELDS:
        assert getattr(a, f) == getattr(b, f), f


def _params(case, coex):
    from paper_1812_10375_gb300.config import params_for
    return params_for(case, rho_l=coex["rho_l"], rho_v=coex["rho_v"])[0]


@pytest.mark.parametrize("first", [37, 48])  # odd and even buffer parity at the checkpoint
def test_single_domain_resumes_bit_exact(coex, first):
    from paper_1812_10375_gb300 import hlb
    case = ragged_case(3)
    d = gpu_domain(case, coex)
    d.step(first)
    before = d.read()
    blob = d.checkpoint()
    diag0 = d.diag()
    d.step(45)
    ref, ref_diag = d.read(), d.diag()
    # a fresh handle with the same parameters, never given fields
    e = hlb.Domain(_params(case, coex))
    e.restore(blob)
    _same_fields(e.read(), before)
    _same_diag(e.diag(), diag0)
    e.step(45)
    _same_fields(e.read(), ref)
    _same_diag(e.diag(), ref_diag)
    # the same blob restores the original handle too
    d.restore(blob)
    d.step(45)
    _same_fields(d.read(), ref)
    assert len(blob) <= hlb.checkpoint_bytes(d.params)


def test_wall_change_and_time_averages_survive(coex):
    """A checkpoint taken after a wall change and a time-average reset keeps
    both (T_bottom and the running sums are part of the state)."""
    from paper_1812_10375_gb300 import hlb
    case = wl.pool(nx=96, ny=64, n_sites=3, heater_rows=10)
    d = gpu_domain(case, coex)
    d.step(20)
    d.set_wall(case.T_bottom(coex["Tc"]) + 0.01)
    d.reset_timeavg()
    d.step(13)
    blob = d.checkpoint()
    d.step(40)
    ref, ref_diag = d.read(), d.diag()
    e = gpu_domain(case, coex)  # other wall, other sites' table: both restored
    e.set_nucleation_sites([])
    e.restore(blob)
    e.step(40)
    _same_fields(e.read(), ref)
    _same_diag(e.diag(), ref_diag)


def _batch(cases, coex):
    import torch
    from paper_1812_10375_gb300 import hlb
    b = hlb.Batch([_params(c, coex) for c in cases])
    for i, c in enumerate(cases):
        rho0, T0 = wl.initial_fields(c, coex["rho_l"], coex["rho_v"], coex["Tc"])
        b.set_fields(i, torch.tensor(rho0, dtype=torch.float32, device="cuda"),
                     torch.tensor(T0, dtype=torch.float32, device="cuda"))
        b.set_nucleation_sites(i, c.sites)
    return b


def _cases():
    return [ragged_case(3), dataclasses.replace(ragged_case(5), name="r70", nx=70, ny=50),
            wl.pool(nx=96, ny=64, n_sites=3, heater_rows=10)]


def test_batch_slot_resumes_bit_exact_at_other_parity(coex):
    cases = _cases()
    b = _batch(cases, coex)
    b.step(21)  # odd parity at the checkpoint
    blob = b.checkpoint(1)
    b.step(40)
    ref, ref_diag, ref_hist = b.read(1), b.diag(1), b.flux_history(1)
    # another batch at even parity: slot 1 restored, the others fresh
    c = _batch(cases, coex)
    c.restore(1, blob)
    c.step(40)
    _same_fields(c.read(1), ref)
    _same_diag(c.diag(1), ref_diag)
    np.testing.assert_array_equal(c.flux_history(1), ref_hist)
    assert len(ref_hist) == 61
    # a stopped slot comes back active when restored
    c.stop(1)
    c.step(3)
    c.restore(1, blob)
    c.step(5)
    assert c.diag(1).step == 26


def _close_fields(a, b):
    """Batched and single-domain kernels are separate instantiations of the
    same device code and may round the last bit differently: rho and T to
    1e-6 of their maxima, u to 1e-6 in lattice units."""
    for k, (x, y) in enumerate(zip(a, b)):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        tol = 1e-6 if k in (1, 2) else 1e-6 * max(np.abs(y).max(), 1e-30)
        assert np.abs(x - y).max() <= tol, ("rho ux uy T".split()[k], np.abs(x - y).max())


def test_checkpoint_moves_between_batch_and_single_domain(coex):
    """A batch slot's checkpoint restored into a single domain reads back the
    slot's fields bit for bit; both then step on (different kernel
    instantiations: to FP32 rounding), and the way back likewise."""
    from paper_1812_10375_gb300 import hlb
    cases = _cases()
    b = _batch(cases, coex)
    b.step(19)
    blob = b.checkpoint(2)
    d = hlb.Domain(_params(cases[2], coex))
    d.restore(blob)
    _same_fields(d.read(), b.read(2))
    _same_diag(d.diag(), b.diag(2))
    b.step(30)
    d.step(30)
    _close_fields(d.read(), b.read(2))
    assert d.diag().step == b.diag(2).step == 49
    back = d.checkpoint()
    b.restore(2, back)
    _same_fields(d.read(), b.read(2))
    b.step(16)
    d.step(16)
    _close_fields(d.read(), b.read(2))


def test_mismatched_or_damaged_checkpoints_are_refused(coex):
    from paper_1812_10375_gb300 import hlb
    case = ragged_case(3)
    d = gpu_domain(case, coex)
    d.step(9)
    blob = d.checkpoint()
    other = gpu_domain(dataclasses.replace(case, nx=46), coex)
    other.step(2)
    keep = other.read()
    bad = [blob[:-1],                        # truncated
           b"X" + blob[1:],                  # magic
           blob[:8] + b"\x07" + blob[9:]]    # format version
    for bb in bad:
        with pytest.raises(hlb.HlbError) as ei:
            d.restore(bb)
        assert ei.value.status == hlb.HLB_EINVAL
    with pytest.raises(hlb.HlbError):
        other.restore(blob)  # another lattice size
    _same_fields(other.read(), keep)
    # another storage form (its reference density differs)
    plain = gpu_domain(case, coex, storage=hlb.HLB_STORE_PLAIN)
    with pytest.raises(hlb.HlbError):
        plain.restore(blob)
    # the refused calls left d as it was
    d.step(3)
    e = hlb.Domain(_params(case, coex))
    e.restore(blob)
    e.step(3)
    _same_fields(e.read(), d.read())
    with pytest.raises(hlb.HlbError) as ei:
        hlb.Domain(_params(case, coex)).checkpoint()  # no fields yet
    assert ei.value.status == hlb.HLB_ESTATE


def test_resumable_sweep_after_a_lost_process_matches_uninterrupted(coex, tmp_path, monkeypatch):
    from paper_1812_10375_gb300 import hlb, sweep
    pts = sweep.make_points(3, seed=5, sides=(64, 96), sites_range=(1, 3), heater_rows=10)
    steps = 192
    ref, fa = sweep.run_resumable(pts, steps, 100, str(tmp_path / "ref"), every=64)
    assert fa == [-1, -1, -1]
    plain, _ = sweep.run_batched(pts, steps, 100)
    for r, p in zip(ref, plain):
        np.testing.assert_array_equal(r.history, p.history)
        assert r.q_qs == p.q_qs and r.coverage == p.coverage and r.regime == p.regime

    class Lost(RuntimeError):
        pass

    real_step = hlb.Batch.step
    budget = {"left": 100}

    def step(self, n=1):
        if n > budget["left"]:
            raise Lost("process lost")
        budget["left"] -= n
        real_step(self, n)

    monkeypatch.setattr(hlb.Batch, "step", step)
    with pytest.raises(Lost):
        sweep.run_resumable(pts, steps, 100, str(tmp_path / "cut"), every=64)
    # lost in the chunk after the half-way step 96 (64 + 32 of the 100 steps
    # allowed); the resumed run may take exactly what remains after 96
    budget["left"] = steps - 96
    res, fa2 = sweep.run_resumable(pts, steps, 100, str(tmp_path / "cut"), every=64)
    assert fa2 == fa
    for r, p in zip(res, ref):
        np.testing.assert_array_equal(r.history, p.history)
        assert r.q_qs == p.q_qs and r.coverage == p.coverage and r.regime == p.regime


def test_sweep_retries_an_unstable_point_with_doubled_n(coex, tmp_path, monkeypatch):
    """A heater of diffusivity 0.65 is beyond RK4's bound at N = 1 (the error
    word is set within a dozen steps) and within it at N = 2: the sweep stops
    both points in the batch, runs each again alone with N = 2 from its
    initial fields (no good checkpoint exists yet), and ends with the results
    of a plain N = 2 run."""
    from paper_1812_10375_gb300 import hlb, sweep
    pts = sweep.make_points(2, seed=9, sides=(64,), sites_range=(1, 2), heater_rows=10)
    real = sweep.params_for

    def conductive(c):
        p, Tc = real(c)
        p.lambda_w = 0.65 * 3.0 * p.rho_l * p.cv
        return p, Tc

    monkeypatch.setattr(sweep, "params_for", conductive)
    steps = 128
    res, fa = sweep.run_resumable(pts, steps, 100, str(tmp_path / "s"), every=64)
    assert fa == [-1, -1] and [r.n_sub for r in res] == [2, 2]
    for r, c in zip(res, pts):
        p, Tc = conductive(c)
        p.n_sub = 2
        d = hlb.Domain(p)
        sweep._setup_domain(d, c, p, Tc)
        d.step(steps)
        h = d.flux_history()
        assert len(h) == steps and d.diag().error_flags == 0
        np.testing.assert_array_equal(r.history, h[:100])
        assert r.q_qs == float(h[steps // 2:].mean())
