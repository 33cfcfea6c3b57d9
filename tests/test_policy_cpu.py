"""Host logic of the surrogate's early-stop policy, with a stand-in ensemble
whose predictions are set by the test: the calibrated threshold and the
(score, spread) pair are the ones a brute-force search over the same
candidates picks, the work fraction is the cell-weighted closed form, and the
features are the block means of the histories.  The regime labels follow the
coverage edges."""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1812_10375_gb300 import sweep
from paper_1812_10375_gb300 import surrogate as sur

L0 = 8


class StandIn:
    """predict() returns fixed (q_pred, spread, regime probabilities)."""

    def __init__(self, qp, spread, prob):
        self.out = (np.asarray(qp, float), np.asarray(spread, float), np.asarray(prob, float))

    def predict(self, hist, scal):
        assert len(hist) == len(self.out[0]) and hist.shape[1] == L0 and scal.shape == (len(hist), 2)
        return self.out


def _results(q, n_hist=40):
    case = SimpleNamespace(nx=10, ny=10, T_bottom_over_Tc=0.96, sites=[(1.0, 2.0, 0.0)])
    return [sweep.PointResult(case, 0.1, 1, np.arange(n_hist, dtype=float) + k, float(qk), 0.1, 1)
            for k, qk in enumerate(q)]


def _prob(p_none, p_film):
    p = np.zeros((len(p_none), 5))
    p[:, 0] = p_none
    p[:, -1] = p_film
    p[:, 1] = 1.0 - p[:, 0] - p[:, -1]
    return p


def test_features_are_block_means():
    res = _results([1.0, 2.0], n_hist=43)
    hist, scal, q, lab = sweep.features(res, L0)
    # 43 // 8 = 5 samples per block, the last 3 dropped
    np.testing.assert_allclose(hist[1], (np.arange(40, dtype=float) + 1).reshape(8, 5).mean(axis=1))
    assert scal.tolist() == [[0.1, 0.1], [0.1, 0.1]] and q.tolist() == [1.0, 2.0] and lab.tolist() == [1, 1]
    with pytest.raises(ValueError):
        sur.downsample(np.zeros(L0 - 1), L0)


def test_threshold_is_the_lowest_safe_score():
    q = np.ones(5)
    qp = q * (1 + np.array([0.01, 0.02, 0.05, 0.01, 0.0]))  # relative errors
    score = np.array([0.9, 0.8, 0.7, 0.6, 0.4])
    ens = StandIn(qp, np.zeros(5), _prob(np.zeros(5), 1.0 - score))
    # accepting down to 0.8 keeps every accepted error within 3%; 0.7 adds a 5% one
    assert sweep.choose_threshold(ens, _results(q), L0, tol=0.03) == pytest.approx(0.8)
    assert sweep.choose_threshold(ens, _results(q), L0, tol=0.06, floor=0.65) == pytest.approx(0.7)
    # an unsafe top score accepts nothing
    ens_bad = StandIn(q * 1.2, np.zeros(5), _prob(np.zeros(5), 1.0 - score))
    assert sweep.choose_threshold(ens_bad, _results(q), L0, tol=0.03) == 1.01


@pytest.mark.parametrize("kind", ["not_film", "no_boiling"])
def test_policy_pair_matches_brute_force(kind):
    rng = np.random.default_rng(3)
    n = 30
    q = 1.0 + rng.random(n)
    err = np.abs(rng.normal(0, 0.03, n))
    qp = q * (1 + err)
    spread = rng.random(n) * 0.1
    p_none, p_film = rng.random(n) * 0.5, rng.random(n) * 0.5
    ens = StandIn(qp, spread, _prob(p_none, p_film))
    thr, smax = sweep.choose_policy(ens, _results(q), L0, tol=0.03, floor=0.3, kind=kind)
    score = 1.0 - p_film if kind == "not_film" else p_none
    best = 0
    for t in np.unique(score[score >= 0.3]):
        for s in np.unique(spread):
            acc = (score >= t) & (spread <= s)
            if acc.any() and err[acc].max() <= 0.03 + 1e-12:
                best = max(best, int(acc.sum()))
    acc = (score >= thr) & (spread <= smax)
    assert int(acc.sum()) == best and best > 0
    assert err[acc].max() <= 0.03 + 1e-12


def test_work_fraction_is_cell_weighted():
    q = np.ones(4)
    score = np.array([0.9, 0.2, 0.95, 0.1])
    ens = StandIn(q * 1.01, np.array([0.0, 0.0, 0.5, 0.0]), _prob(np.zeros(4), 1.0 - score))
    cells = [100, 200, 300, 400]
    acc, err, frac = sweep.evaluate_policy(ens, _results(q), L0, 0.8, hist_steps=10, full_steps=40, cells=cells)
    assert acc.tolist() == [True, False, True, False]
    expect = (10 * 100 + 40 * 200 + 10 * 300 + 40 * 400) / (40 * 1000)
    assert frac == pytest.approx(expect) and np.allclose(err, 0.01)
    # the spread limit removes the third point
    acc, _, frac = sweep.evaluate_policy(ens, _results(q), L0, 0.8, 10, 40, cells, spread_max=0.1)
    assert acc.tolist() == [True, False, False, False]
    assert frac == pytest.approx((10 * 100 + 40 * 900) / (40 * 1000))


def test_regime_labels_follow_the_coverage_edges():
    edges = list(sur.COVERAGE_EDGES)
    assert [sur.regime_of(c) for c in [0.0] + edges + [1.0]] == [0] + list(range(1, len(edges) + 1)) + [len(edges)]
    assert all(sur.regime_of(e - 1e-9) == k for k, e in enumerate(edges))


def _ratio_results(c0, c1, rng, n=12, hs=2000, full_scale=None):
    """Regime-0 results whose quasi-steady flux is exactly (c0 + c1/nx) times
    the mean of the last RATIO_WIN history steps, plus boiling ones (regime 2)
    whose flux is unrelated."""
    out = []
    for k in range(n):
        nx = int(rng.choice([256, 320, 384, 448, 512]))
        case = SimpleNamespace(nx=nx, ny=nx, T_bottom_over_Tc=0.9, sites=[(1.0, 2.0, 0.0)] * 3)
        hist = 1.0 + rng.random(hs)
        late = hist[-sweep.RATIO_WIN:].mean()
        boiling = k % 3 == 2
        q = 5.0 * late if boiling else (c0 + c1 / nx) * late
        out.append(sweep.PointResult(case, 0.05, 3, hist, float(q), 0.0, 2 if boiling else 0))
    return out


def test_conduction_ratio_is_recovered_from_regime_0_points():
    rng = np.random.default_rng(11)
    res = _ratio_results(0.45, -2.0, rng)
    c0, c1 = sweep.fit_conduction_ratio(res, 2000)
    assert c0 == pytest.approx(0.45, rel=1e-9) and c1 == pytest.approx(-2.0, rel=1e-7)
    r = res[0]
    assert sweep.conduction_q((c0, c1), r.case.nx, r.history, 2000) == pytest.approx(r.q_qs, rel=1e-9)
    # the window is the last RATIO_WIN steps of the first hist_steps, whatever follows
    longer = np.concatenate([r.history, np.full(500, 1e6)])
    assert sweep.late_flux(longer, 2000) == pytest.approx(r.history[-sweep.RATIO_WIN:].mean())
    assert sweep.fit_conduction_ratio([res[2]], 2000) == (0.0, 0.0)  # no regime-0 point


def test_ratio_policy_takes_the_ratio_prediction_and_the_no_boiling_score():
    """The 'no_boiling_ratio' kind ignores the ensemble's flux: with exact
    ratios every regime-0 point is within any tolerance, boiling ones are 400%
    off, so the best pair accepts exactly the points whose no-boiling score
    lies above every boiling point's (brute force over the same candidates)."""
    rng = np.random.default_rng(5)
    res = _ratio_results(0.44, -1.5, rng, n=15)
    n = len(res)
    qp = np.full(n, 123.0)  # a useless network flux
    p_none = rng.random(n) * 0.5 + np.array([0.5 if r.regime == 0 else 0.0 for r in res])
    spread = np.zeros(n)
    ens = StandIn(qp, spread, _prob(p_none, np.zeros(n)))
    ratio = sweep.fit_conduction_ratio(res, 2000)
    thr, smax = sweep.choose_policy(ens, res, L0, tol=0.01, floor=0.3, kind="no_boiling_ratio", ratio=ratio,
                                    hist_steps=2000)
    boil = np.array([r.regime != 0 for r in res])
    expect = int(((p_none > p_none[boil].max()) & ~boil).sum())
    acc = (p_none >= thr) & (spread <= smax)
    assert int(acc.sum()) == expect > 0 and not (acc & boil).any()
    acc2, err, frac = sweep.evaluate_policy(ens, res, L0, thr, 2000, 40000, [r.case.nx ** 2 for r in res],
                                            spread_max=smax, kind="no_boiling_ratio", ratio=ratio)
    assert acc2.tolist() == acc.tolist() and err.max() < 1e-9
    # the same points under the network's flux are all rejected
    assert sweep.choose_policy(ens, res, L0, tol=0.01, floor=0.3, kind="no_boiling") == (1.01, 0.0)


def test_frozen_policy_metadata_is_consistent():
    """The committed policy file is one train_policy writes: a known kind, a
    score threshold in range, calibration errors within its tolerance and
    under the 3% bar, and (for the ratio kind) a conduction ratio that keeps
    c0 + c1/nx between 0.4 and 0.5 for the sweep's sides."""
    z = np.load(sweep.policy_path())
    kind = str(z["kind"][()])
    assert kind in ("no_boiling", "not_film", "no_boiling_ratio")
    assert 0.5 <= float(z["threshold"]) <= 1.01
    assert int(z["calibration_accepted"]) <= int(z["calibration_points"])
    assert float(z["calibration_max_error"]) <= float(z["tol"]) < 0.03
    assert int(z["hist_steps"]) < int(z["full_steps"])
    if kind == "no_boiling_ratio":
        c0, c1 = float(z["cond_c0"]), float(z["cond_c1"])
        assert all(0.4 < c0 + c1 / nx < 0.5 for nx in (256, 320, 384, 448, 512))
