"""FP64 CPU reference of the sweep surrogate network (test infrastructure).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import anything under ``oracle/``.

The paper has no learned component; this network is the project's own
addition to its boiling-curve sweep (Section 4.4, Fig. 11): from the superheat,
the number of nucleation sites and the early wall-heat-flux history q(t) of a
run it predicts the quasi-steady mean wall heat flux and a boiling-regime label.

Architecture (all sizes are parameters of ``Config``):

  history x (B, 1, L0) --conv1d(K, stride S) + ReLU--> (B, C1, L1)
                       --conv1d(K, S) + ReLU--------> (B, C2, L2)
                       --conv1d(K, S) + ReLU--------> (B, C3, L3)
                       --mean over time-------------> (B, C3)
  concat with scalars s (B, NS)                       (B, C3 + NS)
  --linear + ReLU--> (B, H) --linear + ReLU--> (B, H) --linear--> (B, NOUT)

Output 0 is the regression value, outputs 1..NOUT-1 are regime logits.
Loss = mean_b (y0 - t)^2 + mean_b CE(softmax(y[1:]), label).
Convolutions are unpadded: L_out = (L_in - K) // S + 1.

Parameter vector order: W1 (C1, 1, K), b1, W2 (C2, C1, K), b2, W3 (C3, C2, K), b3,
F1 (H, C3 + NS), c1, F2 (H, H), c2, F3 (NOUT, H), c3; each row-major.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Config:
    L0: int = 500
    C1: int = 16
    C2: int = 32
    C3: int = 32
    K: int = 5
    S: int = 2
    NS: int = 2
    H: int = 256
    NOUT: int = 6

    @property
    def lengths(self):
        L1 = (self.L0 - self.K) // self.S + 1
        L2 = (L1 - self.K) // self.S + 1
        L3 = (L2 - self.K) // self.S + 1
        return L1, L2, L3

    def shapes(self):
        return [("W1", (self.C1, 1, self.K)), ("b1", (self.C1,)),
                ("W2", (self.C2, self.C1, self.K)), ("b2", (self.C2,)),
                ("W3", (self.C3, self.C2, self.K)), ("b3", (self.C3,)),
                ("F1", (self.H, self.C3 + self.NS)), ("c1", (self.H,)),
                ("F2", (self.H, self.H)), ("c2", (self.H,)),
                ("F3", (self.NOUT, self.H)), ("c3", (self.NOUT,))]

    def n_params(self) -> int:
        return int(sum(np.prod(s) for _, s in self.shapes()))


def unpack(cfg: Config, theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in cfg.shapes():
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(cfg: Config, parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in cfg.shapes()])


def init_params(cfg: Config, rng: np.random.Generator) -> np.ndarray:
    """He-style uniform initialisation (fan-in), zero biases."""
    parts = {}
    for name, shp in cfg.shapes():
        if len(shp) == 1:
            parts[name] = np.zeros(shp)
        else:
            fan_in = int(np.prod(shp[1:]))
            bound = np.sqrt(6.0 / fan_in)
            parts[name] = rng.uniform(-bound, bound, shp)
    return pack(cfg, parts)


def conv1d(x, W, b, S):
    """z[b, o, t] = b[o] + sum_{c, k} W[o, c, k] x[b, c, S t + k]."""
    B, C, L = x.shape
    O, _, K = W.shape
    Lo = (L - K) // S + 1
    z = np.empty((B, O, Lo))
    for t in range(Lo):
        window = x[:, :, S * t:S * t + K]                  # (B, C, K)
        z[:, :, t] = np.einsum("bck,ock->bo", window, W) + b
    return z


def conv1d_backward(x, W, dz, S):
    B, C, L = x.shape
    O, _, K = W.shape
    Lo = dz.shape[2]
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t in range(Lo):
        window = x[:, :, S * t:S * t + K]
        dW += np.einsum("bo,bck->ock", dz[:, :, t], window)
        dx[:, :, S * t:S * t + K] += np.einsum("bo,ock->bck", dz[:, :, t], W)
    db = dz.sum(axis=(0, 2))
    return dx, dW, db


def forward(cfg: Config, theta, hist, scal):
    """Returns the outputs y (B, NOUT) and the cache for backward."""
    P = unpack(cfg, theta)
    x0 = hist[:, None, :].astype(np.float64)
    z1 = conv1d(x0, P["W1"], P["b1"], cfg.S)
    a1 = np.maximum(z1, 0.0)
    z2 = conv1d(a1, P["W2"], P["b2"], cfg.S)
    a2 = np.maximum(z2, 0.0)
    z3 = conv1d(a2, P["W3"], P["b3"], cfg.S)
    a3 = np.maximum(z3, 0.0)
    pooled = a3.mean(axis=2)
    h0 = np.concatenate([pooled, scal.astype(np.float64)], axis=1)
    z4 = h0 @ P["F1"].T + P["c1"]
    a4 = np.maximum(z4, 0.0)
    z5 = a4 @ P["F2"].T + P["c2"]
    a5 = np.maximum(z5, 0.0)
    y = a5 @ P["F3"].T + P["c3"]
    cache = dict(P=P, x0=x0, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, h0=h0, z4=z4, a4=a4, z5=z5, a5=a5)
    return y, cache


def loss_and_dy(y, target, label):
    """MSE on output 0 plus softmax cross-entropy on the regime logits; dL/dy."""
    B = y.shape[0]
    r = y[:, 0] - target
    mse = float(np.mean(r * r))
    logits = y[:, 1:]
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    prob = e / e.sum(axis=1, keepdims=True)
    ce = float(np.mean(-np.log(prob[np.arange(B), label])))
    dy = np.zeros_like(y)
    dy[:, 0] = 2.0 * r / B
    onehot = np.zeros_like(prob)
    onehot[np.arange(B), label] = 1.0
    dy[:, 1:] = (prob - onehot) / B
    return mse, ce, dy


def backward(cfg: Config, cache, dy) -> np.ndarray:
    P = cache["P"]
    g = {}
    g["F3"] = dy.T @ cache["a5"]
    g["c3"] = dy.sum(axis=0)
    da5 = dy @ P["F3"]
    dz5 = da5 * (cache["z5"] > 0)
    g["F2"] = dz5.T @ cache["a4"]
    g["c2"] = dz5.sum(axis=0)
    da4 = dz5 @ P["F2"]
    dz4 = da4 * (cache["z4"] > 0)
    g["F1"] = dz4.T @ cache["h0"]
    g["c1"] = dz4.sum(axis=0)
    dh0 = dz4 @ P["F1"]
    dpooled = dh0[:, :cfg.C3]
    L3 = cache["a3"].shape[2]
    da3 = np.repeat(dpooled[:, :, None], L3, axis=2) / L3
    dz3 = da3 * (cache["z3"] > 0)
    da2, g["W3"], g["b3"] = conv1d_backward(cache["a2"], P["W3"], dz3, cfg.S)
    dz2 = da2 * (cache["z2"] > 0)
    da1, g["W2"], g["b2"] = conv1d_backward(cache["a1"], P["W2"], dz2, cfg.S)
    dz1 = da1 * (cache["z1"] > 0)
    _, g["W1"], g["b1"] = conv1d_backward(cache["x0"], P["W1"], dz1, cfg.S)
    return pack(cfg, g)


def loss_grad(cfg: Config, theta, hist, scal, target, label):
    y, cache = forward(cfg, theta, hist, scal)
    mse, ce, dy = loss_and_dy(y, target, label)
    return mse, ce, backward(cfg, cache, dy)


def adam(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected; returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
