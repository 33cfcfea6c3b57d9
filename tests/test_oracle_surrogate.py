"""Pins of the FP64 surrogate reference: backpropagation against central finite
differences, the convolution against a brute-force loop, the loss against its
closed form, and Adam's first step (which moves every weight by lr * sign(g))."""
import numpy as np
import pytest

from oracle import surrogate as S

TINY = S.Config(L0=23, C1=2, C2=3, C3=3, K=3, S=2, NS=2, H=5, NOUT=6)


def _batch(cfg, B, seed):
    rng = np.random.default_rng(seed)
    hist = rng.normal(size=(B, cfg.L0))
    scal = rng.normal(size=(B, cfg.NS))
    target = rng.normal(size=B)
    label = rng.integers(0, cfg.NOUT - 1, size=B)
    return hist, scal, target, label


def test_backprop_matches_finite_differences():
    cfg = TINY
    theta = S.init_params(cfg, np.random.default_rng(1))
    hist, scal, target, label = _batch(cfg, 4, 2)
    _, _, g = S.loss_grad(cfg, theta, hist, scal, target, label)
    h = 1e-6
    num = np.empty_like(theta)
    for k in range(theta.size):
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        lp = sum(S.loss_grad(cfg, tp, hist, scal, target, label)[:2])
        lm = sum(S.loss_grad(cfg, tm, hist, scal, target, label)[:2])
        num[k] = (lp - lm) / (2 * h)
    assert cfg.n_params() == theta.size
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)


def test_conv1d_matches_brute_force():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 3, 11))
    W = rng.normal(size=(4, 3, 3))
    b = rng.normal(size=4)
    z = S.conv1d(x, W, b, 2)
    assert z.shape == (2, 4, 5)
    for bb in range(2):
        for o in range(4):
            for t in range(5):
                ref = b[o]
                for c in range(3):
                    for k in range(3):
                        ref += W[o, c, k] * x[bb, c, 2 * t + k]
                assert z[bb, o, t] == pytest.approx(ref, rel=1e-12)


def test_loss_closed_form():
    y = np.array([[0.5, 1.0, 2.0, 0.0, -1.0, 0.5], [1.5, 0.0, 0.0, 0.0, 0.0, 0.0]])
    target = np.array([1.0, 1.0])
    label = np.array([1, 3])
    mse, ce, dy = S.loss_and_dy(y, target, label)
    assert mse == pytest.approx((0.25 + 0.25) / 2)
    lse0 = np.log(np.sum(np.exp(y[0, 1:])))
    lse1 = np.log(5.0)
    assert ce == pytest.approx(((lse0 - y[0, 2]) + (lse1 - 0.0)) / 2)
    np.testing.assert_allclose(dy[1, 1:], (np.full(5, 0.2) - np.eye(5)[3]) / 2)


def test_adam_first_step_is_lr_sign():
    g = np.array([3.0, -0.2, 1e-3])
    th, m, v = S.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-4)


def test_default_sizes():
    cfg = S.Config()
    assert cfg.lengths == (248, 122, 59)
    assert cfg.n_params() == (16 * 5 + 16) + (32 * 16 * 5 + 32) + (32 * 32 * 5 + 32) + \
        (256 * 34 + 256) + (256 * 256 + 256) + (6 * 256 + 6)
