"""Host logic of the resumable sweep: a process lost mid-sweep resumes each
point from its own checkpoint and ends with the results of an uninterrupted
sweep; an unstable point runs once more alone from its last good checkpoint
with N of Eq. (27) doubled, and is recorded as failed if that fails too.  The
batch and the single domain are host-side fakes with deterministic per-point
dynamics, and the faults are injected on the host (an exception in place of a
lost process, a set error word in place of a non-finite step); no GPU is
used."""
import pickle
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1812_10375_gb300 import hlb, sweep


class Lost(RuntimeError):
    pass


class FakeBatch:
    """Stands in for hlb.Batch: per slot a step counter, running sums and a
    flux history of q(step) = 1 + 0.01 * seed + 0.1 sin(0.37 step + seed)."""
    crash_after = None  # total steps (over all instances) before a Lost is raised
    fail = {}           # seed -> step at which the error word becomes set at N = 1
    fail_always = set()  # seeds whose failure N = 2 does not cure
    steps_run = 0

    def __init__(self, plist, stream=None):
        self.seeds = [p.seed for p in plist]
        self.nsub = [p.n_sub for p in plist]
        self.slot = [None] * len(plist)
        self.active = [True] * len(plist)

    def _fresh(self, j):
        return dict(step=0, qsum=0.0, csum=0.0, hist=[], err=0, seed=self.seeds[j])

    def step(self, n):
        for _ in range(n):
            if FakeBatch.crash_after is not None and FakeBatch.steps_run >= FakeBatch.crash_after:
                raise Lost("process lost")
            FakeBatch.steps_run += 1
            for j, s in enumerate(self.slot):
                if not self.active[j]:
                    continue
                s["step"] += 1
                q = 1.0 + 0.01 * s["seed"] + 0.1 * np.sin(0.37 * s["step"] + s["seed"])
                s["qsum"] += q
                s["csum"] += 0.5 + 0.5 * np.cos(0.11 * s["step"] * (1 + s["seed"]))
                s["hist"].append(q)
                if FakeBatch.fail.get(s["seed"]) == s["step"] and (
                        self.nsub[j] == 1 or s["seed"] in FakeBatch.fail_always):
                    s["err"] = 1

    def diag(self, j, check_flags=True):
        s = self.slot[j]
        n = max(s["step"], 1)
        return SimpleNamespace(step=s["step"], error_flags=s["err"], q_bottom_timeavg=s["qsum"] / n,
                               vapour_coverage_timeavg=s["csum"] / n)

    def checkpoint(self, j):
        return b"FAKE" + pickle.dumps(self.slot[j])

    def restore(self, j, blob):
        assert blob[:4] == b"FAKE"
        self.slot[j] = pickle.loads(blob[4:])
        self.active[j] = True

    def stop(self, j):
        self.active[j] = False

    def flux_history(self, j):
        return np.asarray(self.slot[j]["hist"])

    def close(self):
        pass


class FakeDomain:
    """Stands in for hlb.Domain: one FakeBatch slot."""
    made = []  # N of every domain created

    def __init__(self, p, stream=None):
        self.b = FakeBatch([p])
        FakeDomain.made.append(p.n_sub)

    def step(self, n=1):
        self.b.step(n)

    def diag(self, check_flags=True):
        return self.b.diag(0)

    def checkpoint(self):
        return self.b.checkpoint(0)

    def restore(self, blob):
        self.b.restore(0, blob)

    def flux_history(self):
        return self.b.flux_history(0)

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    FakeBatch.crash_after, FakeBatch.fail, FakeBatch.fail_always, FakeBatch.steps_run = None, {}, set(), 0
    FakeDomain.made = []
    monkeypatch.setattr(hlb, "Batch", FakeBatch)
    monkeypatch.setattr(hlb, "Domain", FakeDomain)
    monkeypatch.setattr(sweep, "params_for", lambda c: (SimpleNamespace(seed=int(c.name[2:5]), n_sub=1), 1.0))
    monkeypatch.setattr(sweep, "_setup", lambda b, j, c, p, Tc: b.slot.__setitem__(j, b._fresh(j)))
    monkeypatch.setattr(sweep, "_setup_domain", lambda d, c, p, Tc: d.b.slot.__setitem__(0, d.b._fresh(0)))
    return FakeBatch


def _cases(n=5):
    return sweep.make_points(n, seed=11, sides=(64,), sites_range=(1, 2), heater_rows=10)


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.case.name == y.case.name
        np.testing.assert_array_equal(x.history, y.history)
        assert (x.q_qs == y.q_qs or (np.isnan(x.q_qs) and np.isnan(y.q_qs)))
        assert (x.coverage == y.coverage or (np.isnan(x.coverage) and np.isnan(y.coverage)))
        assert x.regime == y.regime


def test_lost_process_resumes_each_point_from_its_checkpoint(fake, tmp_path):
    cases, steps = _cases(), 200
    ref, fa_ref = sweep.run_resumable(cases, steps, 50, str(tmp_path / "ref"), every=32)
    assert fa_ref == [-1] * len(cases)
    full = fake.steps_run
    assert full == steps
    # lose the process part-way, twice, then finish
    d = str(tmp_path / "cut")
    for cut in (70, 100):
        fake.steps_run, fake.crash_after = 0, cut
        with pytest.raises(Lost):
            sweep.run_resumable(cases, steps, 50, d, every=32)
    fake.crash_after, fake.steps_run = None, 0
    res, fa = sweep.run_resumable(cases, steps, 50, d, every=32)
    _same(res, ref)
    assert fa == fa_ref
    # the first run was lost after its checkpoint at 64, the second (from 64,
    # through the half-way step 100) after its checkpoint at 160: the last run
    # steps from 160 only
    assert fake.steps_run == steps - 160
    # everything finished: a further call steps nothing
    fake.steps_run = 0
    again, _ = sweep.run_resumable(cases, steps, 50, d, every=32)
    _same(again, ref)
    assert fake.steps_run == 0


def test_points_at_different_steps_realign(fake, tmp_path):
    """A checkpoint directory where points stopped at different steps (the
    process was lost while it wrote one boundary's checkpoints)."""
    cases, steps = _cases(4), 160
    ref, _ = sweep.run_resumable(cases, steps, 40, str(tmp_path / "ref"), every=32)
    d = tmp_path / "mixed"
    fake.crash_after, fake.steps_run = 96, 0
    with pytest.raises(Lost):
        sweep.run_resumable(cases, steps, 40, str(d), every=32)
    # roll point 2 back to a fresh start and point 1 to an older checkpoint
    (d / "pt00002.ckpt.npz").unlink()
    blob, meta = hlb.read_checkpoint(str(d / "pt00001.ckpt.npz"))
    assert int(meta["step"]) == 96
    old_dir = tmp_path / "old"
    fake.crash_after, fake.steps_run = 64, 0
    with pytest.raises(Lost):
        sweep.run_resumable(cases, steps, 40, str(old_dir), every=32)
    (d / "pt00001.ckpt.npz").write_bytes((old_dir / "pt00001.ckpt.npz").read_bytes())
    fake.crash_after, fake.steps_run = None, 0
    res, _ = sweep.run_resumable(cases, steps, 40, str(d), every=32)
    _same(res, ref)
    # point 2 ran from 0 alone to 64, then with point 1 to 96, then with all
    assert fake.steps_run == steps


def test_unstable_point_is_retried_alone_with_doubled_n(fake, tmp_path):
    cases, steps = _cases(), 200
    bad = int(cases[3].name[2:5])
    fake.fail = {bad: 77}  # unstable at N = 1 only
    d = str(tmp_path / "f")
    res, fa = sweep.run_resumable(cases, steps, 50, d, every=32)
    assert fa == [-1] * len(cases)
    assert res[3].n_sub == 2 and all(res[k].n_sub == 1 for k in range(len(cases)) if k != 3)
    assert FakeDomain.made == [2]
    # the batch ran 96 steps with the point (detection at the boundary after 77),
    # then 200 - 96 without it; the retry restarted from the checkpoint at 64
    assert fake.steps_run == steps + (steps - 64)
    # the fake's dynamics do not depend on N: every result equals a sweep
    # without the instability
    fake.fail, fake.steps_run = {}, 0
    ref, _ = sweep.run_resumable(cases, steps, 50, str(tmp_path / "r"), every=32)
    _same(res, ref)
    _, meta = hlb.read_checkpoint(str(tmp_path / "f" / "pt00003.ckpt.npz"))
    assert int(meta["step"]) == steps and int(meta["n_sub"]) == 2


def test_point_failing_at_doubled_n_is_recorded_and_not_rerun(fake, tmp_path):
    cases, steps = _cases(), 200
    bad = int(cases[3].name[2:5])
    fake.fail, fake.fail_always = {bad: 77}, {bad}
    d = str(tmp_path / "f")
    res, fa = sweep.run_resumable(cases, steps, 50, d, every=32)
    assert fa[3] == 96  # the retry from 64 fails again at its first boundary
    assert res[3].regime == -1 and res[3].n_sub == 2 and np.isnan(res[3].q_qs) and np.isnan(res[3].coverage)
    assert all(fa[k] == -1 and res[k].regime >= 0 for k in range(len(cases)) if k != 3)
    # its last good checkpoint stays
    _, meta = hlb.read_checkpoint(str(tmp_path / "f" / "pt00003.ckpt.npz"))
    assert int(meta["step"]) == 64 and int(meta["n_sub"]) == 1
    fake.steps_run = 0
    res2, fa2 = sweep.run_resumable(cases, steps, 50, d, every=32)
    assert fake.steps_run == 0 and fa2 == fa
    # without retries the failure is recorded at N = 1
    fake.steps_run = 0
    res3, fa3 = sweep.run_resumable(cases, steps, 50, str(tmp_path / "nr"), every=32, retry=False)
    assert fa3[3] == 96 and res3[3].n_sub == 1 and FakeDomain.made == [2]
    # the other points match a sweep without the unstable point
    fake.fail = {}
    ref, _ = sweep.run_resumable([c for k, c in enumerate(cases) if k != 3], steps, 50, str(tmp_path / "r"),
                                 every=32)
    _same([r for k, r in enumerate(res) if k != 3], ref)


def test_process_lost_during_a_retry_resumes_the_retry(fake, tmp_path):
    cases, steps = _cases(3), 192
    bad = int(cases[1].name[2:5])
    fake.fail = {bad: 40}
    d = str(tmp_path / "f")
    # the batch finishes (192 steps, detection at 64), then the retry from 32
    # is lost after 100 more steps (its checkpoint at 128 is on disk)
    fake.crash_after = steps + 100
    with pytest.raises(Lost):
        sweep.run_resumable(cases, steps, 40, d, every=32)
    _, meta = hlb.read_checkpoint(str(tmp_path / "f" / "pt00001.ckpt.npz"))
    assert int(meta["step"]) == 128 and int(meta["n_sub"]) == 2
    fake.crash_after, fake.steps_run = None, 0
    res, fa = sweep.run_resumable(cases, steps, 40, d, every=32)
    assert fa == [-1, -1, -1] and res[1].n_sub == 2
    assert fake.steps_run == steps - 128  # only the retry's remainder, alone
    assert FakeDomain.made == [2, 2]
    fake.fail, fake.steps_run = {}, 0
    ref, _ = sweep.run_resumable(cases, steps, 40, str(tmp_path / "r"), every=32)
    _same(res, ref)


def test_checkpoints_of_another_sweep_are_refused(fake, tmp_path):
    cases = _cases(3)
    d = str(tmp_path / "x")
    fake.crash_after = 40
    with pytest.raises(Lost):
        sweep.run_resumable(cases, 100, 20, d, every=32)
    fake.crash_after, fake.steps_run = None, 0
    with pytest.raises(ValueError):
        sweep.run_resumable(cases, 120, 20, d, every=32)  # other length
    with pytest.raises(ValueError):
        sweep.run_resumable(_cases(3)[::-1], 100, 20, d, every=32)  # other points


def test_checkpoint_file_round_trip(tmp_path):
    blob = bytes(range(256)) * 3
    p = str(tmp_path / "c.npz")
    hlb.write_checkpoint(p, blob, step=48, name="pt001_64")
    b2, meta = hlb.read_checkpoint(p)
    assert b2 == blob and int(meta["step"]) == 48 and str(meta["name"]) == "pt001_64"


def test_checkpoint_bytes_covers_header_fields_and_history():
    from paper_1812_10375_gb300 import build
    build.build()
    p = hlb.default_params(64, 96)
    N = 64 * 96
    fields = 4 * (9 * N + 2 * N + 3 * 64 + 64)
    assert hlb.checkpoint_bytes(p) == 512 + (fields + 7) // 8 * 8 + 8 * 65536
    p.ny = 3
    assert hlb.checkpoint_bytes(p) == 0


def test_paper_curve_goes_through_the_resumable_driver(monkeypatch, tmp_path):
    """paper_curve with a checkpoint directory hands the Fig. 11 cases to
    run_resumable and reports each point's N and failure step."""
    from paper_1812_10375_gb300 import build
    build.build()
    seen = {}

    def fake_run(cases, steps, hist_steps, ckpt_dir, every=2048, retry=True):
        seen.update(n=len(cases), steps=steps, dir=ckpt_dir, every=every)
        res = [sweep.PointResult(c, c.T_bottom_over_Tc - 0.86, len(c.sites), np.zeros(0), 1e-3 * (k + 1), 0.1, 1,
                                 1 + k) for k, c in enumerate(cases)]
        return res, [-1, 77][:len(cases)]

    monkeypatch.setattr(sweep, "run_resumable", fake_run)
    rows, secs = sweep.paper_curve([0.1, 0.2], 1000, ckpt_dir=str(tmp_path), every=128)
    assert seen == dict(n=2, steps=1000, dir=str(tmp_path), every=128)
    assert [r["n_sub"] for r in rows] == [1, 2] and [r["failed_at"] for r in rows] == [-1, 77]
    assert rows[1]["h"] == pytest.approx(rows[1]["q"] / (rows[1]["superheat_over_Tc"] * sweep.paper_cases([0.2])[2]))
