"""Surrogate kernels against the FP64 reference (forward, gradients, Adam) and
the sweep policy: a network trained by the project's kernels on runs of the
method itself stops sweep points early, and full runs measure its error."""
import numpy as np
import pytest

from oracle import surrogate as S

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build
    build.build()


def _cfg_pair(tiny):
    from paper_1812_10375_gb300 import surrogate as sur
    if tiny:
        oc = S.Config(L0=23, C1=2, C2=3, C3=3, K=3, S=2, NS=2, H=5, NOUT=6)
    else:
        oc = S.Config()
    gc = sur.hlb_sur_config(oc.L0, oc.C1, oc.C2, oc.C3, oc.K, oc.S, oc.NS, oc.H, oc.NOUT)
    return oc, gc


@pytest.mark.parametrize("tiny", [True, False])
def test_forward_and_gradients_match_fp64_reference(tiny):
    import torch
    from paper_1812_10375_gb300 import surrogate as sur
    oc, gc = _cfg_pair(tiny)
    rng = np.random.default_rng(5)
    B = 8
    theta = S.init_params(oc, rng).astype(np.float32).astype(np.float64)
    theta += 0.05 * rng.normal(size=theta.shape)  # non-zero biases
    theta = theta.astype(np.float32).astype(np.float64)
    hist = rng.normal(size=(B, oc.L0)).astype(np.float32).astype(np.float64)
    scal = rng.normal(size=(B, oc.NS)).astype(np.float32).astype(np.float64)
    target = rng.normal(size=B).astype(np.float32).astype(np.float64)
    label = rng.integers(0, oc.NOUT - 1, size=B)
    net = sur.Net(gc, max_batch=B)
    assert net.n == oc.n_params()
    net.params.copy_(torch.tensor(theta, dtype=torch.float32))
    t = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    y_g = net.forward(t(hist), t(scal)).cpu().numpy().astype(np.float64)
    y_o, _ = S.forward(oc, theta, hist, scal)
    assert np.abs(y_g - y_o).max() / np.abs(y_o).max() < TOL
    loss, grad = net.loss_grad(t(hist), t(scal), t(target), t(label, torch.int32))
    mse, ce, g_o = S.loss_grad(oc, theta, hist, scal, target, label)
    l = loss.cpu().numpy()
    assert l[0] == pytest.approx(mse, rel=TOL) and l[1] == pytest.approx(ce, rel=TOL)
    g_g = grad.cpu().numpy().astype(np.float64)
    o = 0
    for name, shp in oc.shapes():
        n = int(np.prod(shp))
        a, b = g_g[o:o + n], g_o[o:o + n]
        assert np.abs(a - b).max() <= TOL * max(np.abs(b).max(), 1e-8), name
        o += n


def test_adam_matches_reference():
    import torch
    from paper_1812_10375_gb300 import surrogate as sur
    oc, gc = _cfg_pair(True)
    net = sur.Net(gc, max_batch=4)
    rng = np.random.default_rng(9)
    th = net.params.cpu().numpy().astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for t in range(1, 4):
        g = rng.normal(size=th.shape).astype(np.float32)
        net.grad.copy_(torch.tensor(g))
        net.adam(lr=1e-2)
        th, m, v = S.adam(th, g.astype(np.float64), m, v, t, lr=1e-2)
    np.testing.assert_allclose(net.params.cpu().numpy(), th, rtol=1e-5, atol=1e-7)


def test_trained_surrogate_gain_on_sweep():
    """Generate points with the batched step, train an ensemble with the CUDA
    kernels, calibrate the acceptance on separate points, and let it stop
    held-out points early; their full runs measure the error (3% bar)."""
    from paper_1812_10375_gb300 import surrogate as sur, sweep
    pts = sweep.make_points(256, seed=77, sides=(64, 96), sites_range=(1, 4), heater_rows=10, aspect=1.25)
    full, hist_steps = 4000, 1500
    res, secs = sweep.run_batched(pts, full, hist_steps)
    assert all(np.isfinite(r.q_qs) for r in res)
    fit, cal, test = res[:160], res[160:208], res[208:]
    ens = sur.Ensemble(members=4, seed=3, max_batch=160)
    L0 = ens.members[0].net.cfg.L0
    hist, scal, q, lab = sweep.features(fit, L0)
    losses = ens.fit(hist, scal, q, lab, epochs=600, batch=64, lr=1e-3)
    for l in losses:
        assert l[-1].sum() < 0.2 * l[0].sum()
    thr = sweep.choose_threshold(ens, cal, L0, tol=0.03)
    cells = [r.case.nx * r.case.ny for r in test]
    acc, err, cost = sweep.evaluate_policy(ens, test, L0, thr, hist_steps, full, cells)
    print(f"surrogate: score threshold {thr:.4f}, accepted {acc.sum()}/{len(test)} held-out points, "
          f"max error of accepted {err.max() if len(err) else 0:.4f}, work {cost:.3f} of full "
          f"(gain {1 / cost:.2f}x points per unit of work); batched sweep of 256 points {secs:.2f} s")
    assert cost <= 1.0
    assert len(err) == 0 or err.max() <= 0.03
