"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/hlb.h declares; its host-only thermodynamics agrees with the oracle.
No kernel is launched here."""
import ctypes
import os
import re

import pytest

from paper_1812_10375_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_1812_10375_gb300 import hlb
    return hlb


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hlb_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    decl = declared_symbols()
    assert len(decl) >= 12
    missing = [n for n in decl if not hasattr(so, n)]
    assert not missing, missing


def test_host_coexistence_matches_oracle(lib):
    from oracle import eos
    p = lib.default_params(8, 8)
    Tc, rl, rv, h = lib.eos_coexistence(p)
    pr = eos.PR()
    orl, orv, _ = eos.coexistence(0.86 * pr.Tc, pr)
    assert Tc == pytest.approx(pr.Tc, rel=1e-14)
    assert rl == pytest.approx(orl, rel=1e-10)
    assert rv == pytest.approx(orv, rel=1e-10)
    assert h == pytest.approx(eos.latent_heat(0.86 * pr.Tc, pr, orl, orv), rel=1e-9)


def test_defaults_are_the_paper_values(lib, paper):
    p = lib.default_params(16, 16)
    assert p.a == pytest.approx(paper["a"]["value"]) and p.b == pytest.approx(paper["b"]["value"])
    assert p.Ts_over_Tc == paper["Ts_over_Tc"]["value"] and p.sigma == paper["sigma"]["value"]
    assert p.cv == paper["cv"]["value"] and p.k == paper["k"]["value"] and p.Gw0 == paper["Gw0"]["value"]
    # tau = 3 nu + 1/2 (Eq. 3 with dt = 1)
    assert p.tau_l == pytest.approx(3 * paper["nu_l"]["value"] + 0.5)
    assert p.tau_v == pytest.approx(3 * paper["nu_v"]["value"] + 0.5)


def test_workspace_size_and_rejections(lib):
    p = lib.default_params(64, 48)
    n = lib.workspace_bytes(p)
    # populations and T double-buffered, plus rho^n, u^n and a T plane of the split step
    assert n >= 2 * 10 * 64 * 48 * 4 + 4 * 64 * 48 * 4
    bad = lib.default_params(2, 48)
    assert lib.workspace_bytes(bad) == 0
    # N of Eq. (27): 1..64, a finite-volume option; N > 1 adds the fused
    # kernels' per-block sub-step partials, and batches take it too
    for bad_n in (-1, 65):  # 0 selects N from the stability bound
        p.n_sub = bad_n
        assert lib.workspace_bytes(p) == 0
    p.n_sub = 2
    extra = 2 * 2 * 4 * 8  # (2 x 2 tiles of 56 x 24) x 4 FP64 partials
    assert lib.workspace_bytes(p) >= n + extra
    assert lib.lib().hlb_batch_workspace_bytes(1, ctypes.byref(p)) > 0
    p.diffusion = lib.HLB_DIFF_ISO
    assert lib.workspace_bytes(p) == 0
    p.diffusion = lib.HLB_DIFF_FV
    w2 = lib.workspace_bytes(p)
    p.n_sub = 64  # the scratch does not grow with N (the sub-steps reuse it)
    assert lib.workspace_bytes(p) == w2
    # nine population planes must stay below 2^31 floats (32-bit offsets in the kernels)
    assert lib.workspace_bytes(lib.default_params(15000, 15000)) > 0
    assert lib.workspace_bytes(lib.default_params(16384, 16384)) == 0


def test_init_rejects_invalid_parameters_without_a_gpu(lib):
    import ctypes as C
    p = lib.default_params(2, 64)  # nx below the minimum
    h = C.c_void_p()
    st = lib.lib().hlb_init(C.byref(h), C.byref(p), C.c_void_p(256), 1 << 20, None)
    assert st == lib.HLB_EINVAL and not h.value
    q = lib.default_params(64, 64)
    q.n_sub = 65
    assert lib.lib().hlb_init(C.byref(h), C.byref(q), C.c_void_p(256), 1 << 30, None) == lib.HLB_EINVAL
    assert lib.lib().hlb_strerror(lib.HLB_EUNSTABLE).decode().startswith("device error word")


def test_tile_variant_entry_points_reject_bad_arguments(lib):
    import ctypes as C
    n = lib.lib().hlb_tile_variants(None, None, None, 0)
    assert n >= 1 and len(lib.tile_variants()) == n
    L = lib.lib()
    assert L.hlb_set_tile_variant(None, 0) == lib.HLB_EINVAL
    assert L.hlb_batch_set_tile_variant(None, 0) == lib.HLB_EINVAL
    assert L.hlb_autotune(None, 4, None, None, 0) == lib.HLB_EINVAL


def test_scheme_and_heater_parameters_are_validated(lib):
    """The diffusion scheme and bottom-boundary selectors take only their
    enumerated values; the isotropic scheme is a single-domain option, so a
    batch workspace of it is refused; an imposed flux must be finite."""
    p = lib.default_params(64, 48)
    assert p.diffusion == lib.HLB_DIFF_FV and p.bottom_bc == lib.HLB_BOTTOM_DIRICHLET
    assert p.lambda_top == 0.0 and p.q_in == 0.0
    p.diffusion = 2
    assert lib.workspace_bytes(p) == 0
    p.diffusion = lib.HLB_DIFF_ISO
    assert lib.workspace_bytes(p) > 0
    assert lib.lib().hlb_batch_workspace_bytes(1, ctypes.byref(p)) == 0
    p.diffusion = lib.HLB_DIFF_FV
    p.bottom_bc = 5
    assert lib.workspace_bytes(p) == 0
    p.bottom_bc = lib.HLB_BOTTOM_FLUX
    p.q_in = float("nan")
    assert lib.workspace_bytes(p) == 0
    p.q_in = 2e-4
    assert lib.workspace_bytes(p) > 0
    assert lib.lib().hlb_batch_workspace_bytes(1, ctypes.byref(p)) > 0


def test_stable_substeps_bound(lib):
    """n_sub = 0 picks N of Eq. (27) from the RK4 stability of the conduction
    operator: N = ceil(16 D_max / 2.785).  The bound is checked here on the
    finite-volume operator assembled from harmonic face conductivities (a
    heater under a liquid-vapour column, periodic x, Dirichlet bottom and top
    rows): its eigenvalues are real, within [-16 D_max, 0], and every RK4
    sub-step amplification |P4(h z)|, h = 1/N, is at most 1 at the chosen N,
    while N = 1 is unstable for the conductive heater."""
    import numpy as np
    p = lib.default_params(64, 48)
    assert lib.stable_substeps(p) == 1
    Tc, rl, rv, _ = lib.eos_coexistence(p)
    q = lib.default_params(64, 48)
    q.n_sub = 0
    assert lib.workspace_bytes(q) == lib.workspace_bytes(p)  # resolves to N = 1
    nx, ny, W = 4, 12, 3
    rho = np.where(np.arange(ny)[:, None] < 7, rl, rv) * np.ones((ny, nx))
    for D_w in (0.1, 0.3, 0.65, 1.3):
        q = lib.default_params(64, 48)
        q.lambda_w = D_w * 3.0 * rl * q.cv
        N = lib.stable_substeps(q)
        assert N == int(np.ceil(16.0 * max(q.k, D_w) / 2.785))
        q.n_sub = 0
        assert lib.workspace_bytes(q) > 0
        q.n_sub = N
        w_n = lib.workspace_bytes(q)
        q.n_sub = 0
        assert lib.workspace_bytes(q) == w_n
        batch_ws = lib.lib().hlb_batch_workspace_bytes
        assert batch_ws(1, ctypes.byref(q)) >= batch_ws(1, ctypes.byref(p))  # batches take any N (split step)
        solid = np.arange(ny)[:, None] < W
        lam = np.where(solid, q.lambda_w, rho * q.cv * q.k)
        rcv = np.where(solid, 3.0 * rl * q.cv, rho * q.cv)
        free = [(y, x) for y in range(1, ny - 1) for x in range(nx)]
        index = {c: k for k, c in enumerate(free)}
        A = np.zeros((len(free), len(free)))
        for (y, x), k in index.items():
            for yy, xx in ((y, (x + 1) % nx), (y, (x - 1) % nx), (y + 1, x), (y - 1, x)):
                lf = 2.0 * lam[y, x] * lam[yy, xx] / (lam[y, x] + lam[yy, xx])
                A[k, k] -= lf / rcv[y, x]
                if (yy, xx) in index:
                    A[k, index[(yy, xx)]] += lf / rcv[y, x]
        z = np.linalg.eigvals(A)
        assert np.abs(z.imag).max() < 1e-9 and z.real.max() < 1e-12
        assert -z.real.min() <= 16.0 * max(q.k, D_w) + 1e-12
        P4 = lambda w: 1 + w + w ** 2 / 2 + w ** 3 / 6 + w ** 4 / 24
        assert np.abs(P4(z.real / N)).max() <= 1.0 + 1e-12
        if D_w >= 0.65:
            assert np.abs(P4(z.real)).max() > 1.0  # N = 1 would diverge
