"""Sweep surrogate: binding of the CUDA training/inference kernels and the
early-stop policy of the boiling-curve sweep.

The network (include/hlb_surrogate.h) reads a run's superheat, site count and
the first steps of its wall-heat-flux history q(t) and predicts the run's
quasi-steady mean wall heat flux and boiling regime.  Every forward, backward
and Adam step runs in libhlb.so; this module only marshals arguments and keeps
the feature scaling.  A plain full run stays the fallback: the policy only
stops a point early when the network is confident, and the full runs measure the
error of the points it stops.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import hlb

REGIMES = ("no boiling", "isolated bubbles", "slugs and columns", "transition", "film")
# thresholds on the time-averaged vapour fraction of the wall row between the
# regimes above (the paper names the regimes visually, Section 4.4)
COVERAGE_EDGES = (0.01, 0.15, 0.35, 0.70)


def regime_of(coverage: float) -> int:
    return int(np.searchsorted(np.asarray(COVERAGE_EDGES), coverage, side="right"))


class hlb_sur_config(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("L0", "C1", "C2", "C3", "K", "S", "NS", "H", "NOUT")]


def _lib():
    L = hlb.lib()
    if not getattr(L, "_sur_ready", False):
        P, vp, st = C.POINTER, C.c_void_p, C.c_int
        sig = {
            "hlb_sur_config_default": (None, [P(hlb_sur_config)]),
            "hlb_sur_param_count": (C.c_size_t, [P(hlb_sur_config)]),
            "hlb_sur_workspace_bytes": (C.c_size_t, [P(hlb_sur_config), C.c_int]),
            "hlb_sur_forward": (st, [P(hlb_sur_config), vp, vp, vp, C.c_int, vp, vp, C.c_size_t, vp]),
            "hlb_sur_loss_grad": (st, [P(hlb_sur_config), vp, vp, vp, vp, vp, C.c_int, vp, vp, vp, C.c_size_t, vp]),
            "hlb_sur_adam": (st, [C.c_longlong, vp, vp, vp, vp, C.c_float, C.c_float, C.c_float, C.c_float,
                                  C.c_int, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        L._sur_ready = True
    return L


def default_config() -> hlb_sur_config:
    c = hlb_sur_config()
    _lib().hlb_sur_config_default(C.byref(c))
    return c


def _p(t):
    return C.c_void_p(t.data_ptr())


class Net:
    """Parameters, Adam state and workspace of one surrogate network on the GPU."""

    def __init__(self, cfg: hlb_sur_config | None = None, seed: int = 0, max_batch: int = 256):
        import torch
        self.cfg = cfg if cfg is not None else default_config()
        L = _lib()
        self.n = int(L.hlb_sur_param_count(C.byref(self.cfg)))
        if self.n == 0:
            raise ValueError("invalid surrogate configuration")
        self.max_batch = max_batch
        self.ws_bytes = int(L.hlb_sur_workspace_bytes(C.byref(self.cfg), max_batch))
        self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device="cuda")
        self.ws = C.c_void_p((self._ws.data_ptr() + 255) & ~255)
        self.params = torch.tensor(self._init(seed), dtype=torch.float32, device="cuda")
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.loss = torch.zeros(2, dtype=torch.float32, device="cuda")
        self.t = 0

    def shapes(self):
        c = self.cfg
        return [(c.C1, 1, c.K), (c.C1,), (c.C2, c.C1, c.K), (c.C2,), (c.C3, c.C2, c.K), (c.C3,),
                (c.H, c.C3 + c.NS), (c.H,), (c.H, c.H), (c.H,), (c.NOUT, c.H), (c.NOUT,)]

    def _init(self, seed: int) -> np.ndarray:
        """Uniform fan-in initialisation, zero biases."""
        rng = np.random.default_rng(seed)
        out = []
        for shp in self.shapes():
            if len(shp) == 1:
                out.append(np.zeros(shp))
            else:
                bound = np.sqrt(6.0 / float(np.prod(shp[1:])))
                out.append(rng.uniform(-bound, bound, shp))
        return np.concatenate([a.ravel() for a in out])

    def _check(self, name, st):
        hlb.check(name, st)

    def forward(self, hist, scal):
        import torch
        B = hist.shape[0]
        out = torch.empty((B, self.cfg.NOUT), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        self._check("hlb_sur_forward", _lib().hlb_sur_forward(
            C.byref(self.cfg), _p(self.params), _p(hist), _p(scal), B, _p(out), self.ws, self.ws_bytes,
            C.c_void_p(stream)))
        return out

    def loss_grad(self, hist, scal, target, label):
        import torch
        B = hist.shape[0]
        stream = torch.cuda.current_stream().cuda_stream
        self._check("hlb_sur_loss_grad", _lib().hlb_sur_loss_grad(
            C.byref(self.cfg), _p(self.params), _p(hist), _p(scal), _p(target), _p(label), B, _p(self.grad),
            _p(self.loss), self.ws, self.ws_bytes, C.c_void_p(stream)))
        return self.loss, self.grad

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        import torch
        self.t += 1
        self._check("hlb_sur_adam", _lib().hlb_sur_adam(
            self.n, _p(self.params), _p(self.grad), _p(self.m), _p(self.v), lr, b1, b2, eps, self.t,
            C.c_void_p(torch.cuda.current_stream().cuda_stream)))


def _level(hist):
    """Final level of each (downsampled) history: the mean of its last 5%."""
    n = max(1, hist.shape[1] // 20)
    return np.maximum(hist[:, -n:].mean(axis=1), 1e-12)


@dataclass
class Scaler:
    """Input and target scaling.  The history enters normalised by its own final
    level, with log(level) as an extra scalar, and the regression target is
    log(q_qs / level): the network learns a correction to persistence of the
    early flux, which for conduction-dominated points is nearly constant."""

    h_mean: float = 0.0
    h_std: float = 1.0
    s_mean: np.ndarray = field(default_factory=lambda: np.zeros(3))
    s_std: np.ndarray = field(default_factory=lambda: np.ones(3))
    t_mean: float = 0.0
    t_std: float = 1.0

    @staticmethod
    def _raw(hist, scal):
        lv = _level(hist)
        return hist / lv[:, None], np.column_stack([scal, np.log(lv)]), lv

    @classmethod
    def fit(cls, hist, scal, q):
        hn, sc, lv = cls._raw(hist, scal)
        t = np.log(np.maximum(q, 1e-12) / lv)
        return cls(float(hn.mean()), float(hn.std() + 1e-12), sc.mean(axis=0), sc.std(axis=0) + 1e-12,
                   float(t.mean()), float(t.std() + 1e-12))

    def x(self, hist, scal):
        hn, sc, _ = self._raw(hist, scal)
        return (hn - self.h_mean) / self.h_std, (sc - self.s_mean) / self.s_std

    def target(self, hist, q):
        return (np.log(np.maximum(q, 1e-12) / _level(hist)) - self.t_mean) / self.t_std

    def q_of(self, hist, y0):
        return _level(hist) * np.exp(y0 * self.t_std + self.t_mean)


def downsample(history: np.ndarray, L0: int) -> np.ndarray:
    """Block-average the first len - len % L0 entries of a flux history to L0 samples."""
    h = np.asarray(history, dtype=np.float64)
    blk = len(h) // L0
    if blk < 1:
        raise ValueError("history shorter than the network input")
    return h[:blk * L0].reshape(L0, blk).mean(axis=1)


class Surrogate:
    """A trained network plus its scaling; predicts (q_qs, regime probabilities)."""

    def __init__(self, cfg=None, seed=0, max_batch=256):
        if cfg is None:
            cfg = default_config()
            cfg.NS = 3  # superheat, site count / 10, log of the history's final level
        self.net = Net(cfg, seed=seed, max_batch=max_batch)
        self.scaler = None

    def fit(self, hist, scal, q, label, epochs=300, batch=64, lr=2e-3, seed=0):
        import torch
        self.scaler = Scaler.fit(hist, scal, q)
        xh, xs = self.scaler.x(hist, scal)
        tq = self.scaler.target(hist, q)
        dev = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
        Xh, Xs, T, Y = dev(xh), dev(xs), dev(tq), dev(label, torch.int32)
        rng = np.random.default_rng(seed)
        n = len(q)
        hist_loss = []
        for ep in range(epochs):
            perm = rng.permutation(n)
            for k in range(0, n, batch):
                idx = torch.tensor(perm[k:k + batch], device="cuda")
                loss, _ = self.net.loss_grad(Xh[idx].contiguous(), Xs[idx].contiguous(), T[idx].contiguous(),
                                             Y[idx].contiguous())
                self.net.adam(lr=lr)
            hist_loss.append(loss.cpu().numpy().copy())
        return np.array(hist_loss)

    def predict(self, hist, scal):
        import torch
        xh, xs = self.scaler.x(hist, scal)
        out = []
        for k in range(0, len(xh), self.net.max_batch):
            y = self.net.forward(torch.tensor(np.ascontiguousarray(xh[k:k + self.net.max_batch]),
                                              dtype=torch.float32, device="cuda"),
                                 torch.tensor(np.ascontiguousarray(xs[k:k + self.net.max_batch]),
                                              dtype=torch.float32, device="cuda"))
            out.append(y.cpu().numpy().astype(np.float64))
        y = np.concatenate(out)
        q = self.scaler.q_of(hist, y[:, 0])
        logits = y[:, 1:]
        p = np.exp(logits - logits.max(axis=1, keepdims=True))
        return q, p / p.sum(axis=1, keepdims=True)


class Ensemble:
    """Several independently initialised networks; their disagreement is the
    uncertainty the early-stop policy uses."""

    def __init__(self, members=4, cfg=None, seed=0, max_batch=256):
        self.members = [Surrogate(cfg, seed=seed + 101 * k, max_batch=max_batch) for k in range(members)]

    def fit(self, hist, scal, q, label, **kw):
        return [m.fit(hist, scal, q, label, seed=kw.pop("seed", 0) + k, **kw) for k, m in enumerate(self.members)]

    def predict(self, hist, scal):
        """Mean predicted q_qs, relative spread (max - min) / |mean|, mean regime probabilities."""
        qs, ps = zip(*[m.predict(hist, scal) for m in self.members])
        qs = np.stack(qs)
        mean = qs.mean(axis=0)
        spread = (qs.max(axis=0) - qs.min(axis=0)) / np.maximum(np.abs(mean), 1e-12)
        return mean, spread, np.mean(np.stack(ps), axis=0)

    _CFG = ("L0", "C1", "C2", "C3", "K", "S", "NS", "H", "NOUT")

    def save(self, path, **meta):
        """Weights, input/target scaling and configuration of every member, plus
        scalar metadata (the frozen early-stop policy), as one .npz file."""
        arrays = {f"m{k}_params": m.net.params.cpu().numpy() for k, m in enumerate(self.members)}
        for k, m in enumerate(self.members):
            sc = m.scaler
            arrays[f"m{k}_scaler"] = np.concatenate([[sc.h_mean, sc.h_std], sc.s_mean, sc.s_std,
                                                     [sc.t_mean, sc.t_std]])
        cfg = self.members[0].net.cfg
        arrays["cfg"] = np.array([getattr(cfg, f) for f in self._CFG], dtype=np.int64)
        np.savez(path, members=len(self.members), **arrays, **{k: np.asarray(v) for k, v in meta.items()})

    @classmethod
    def load(cls, path, max_batch=256):
        """(ensemble, metadata dict) from a file written by save()."""
        import torch
        z = np.load(path)
        cfg = default_config()
        for f, v in zip(cls._CFG, z["cfg"]):
            setattr(cfg, f, int(v))
        n = int(z["members"])
        ens = cls(members=n, cfg=cfg, max_batch=max_batch)
        for k, m in enumerate(ens.members):
            m.net.params.copy_(torch.tensor(z[f"m{k}_params"], dtype=torch.float32, device="cuda"))
            v = z[f"m{k}_scaler"]
            ns = (len(v) - 4) // 2
            m.scaler = Scaler(float(v[0]), float(v[1]), v[2:2 + ns].copy(), v[2 + ns:2 + 2 * ns].copy(),
                              float(v[-2]), float(v[-1]))
        skip = {"members", "cfg"} | {f"m{k}_params" for k in range(n)} | {f"m{k}_scaler" for k in range(n)}
        meta = {k: z[k][()] for k in z.files if k not in skip}
        return ens, meta
