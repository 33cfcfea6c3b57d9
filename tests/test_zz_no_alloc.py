"""hlb_step_static, the entry point for callers that cannot allocate device
memory: a solver embedded as a plug-in in an application that owns every
device allocation through its own pool, or a process whose device memory is
reserved in full up front.  Such a caller still passes its own state buffers,
but cannot hand the library a workspace; the step takes its scratch (per-block
partial sums, the diagnostics record, the wetting table) from a static device
array inside the library instead.

Two calls in a row, through the C ABI, must agree with the regular
workspace-based step of the same domain within the parity tolerance (1e-5),
with the populations stored plainly and as deviations f_q - w_q rho_v.  Sizes
beyond the static array are refused with HLB_EINVAL before anything runs.
This file is collected last, so that a failure here comes after every other
test has run."""
import ctypes as C

import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, ragged_case

pytestmark = pytest.mark.gpu
TOL = 1e-5
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
TILE_W, TILE_H = 52, 28     # tile of the step kernel the entry point runs
MAX_TILES = 17549           # partial-sum slots of the static array


@pytest.mark.parametrize("storage", ["plain", "deviation"])
def test_static_step_matches_workspace_step_twice(storage):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build, hlb
    from paper_1812_10375_gb300.config import params_for
    build.build()

    coex = coexistence()
    case = ragged_case()
    kind = hlb.HLB_STORE_PLAIN if storage == "plain" else hlb.HLB_STORE_DEVIATION
    p, Tc = params_for(case, storage=kind, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    rho_ref = 0.0 if storage == "plain" else float(p.rho_v)
    rho0, T0 = wl.initial_fields(case, coex["rho_l"], coex["rho_v"], Tc)
    rho0 = rho0.astype(np.float32)
    T0 = T0.astype(np.float32)
    ny, nx, Wr = case.ny, case.nx, case.wall_rows

    # the regular entry points, with a library workspace
    dom = hlb.Domain(p)
    dom.set_fields(torch.tensor(rho0, device="cuda"), torch.tensor(T0, device="cuda"))
    dom.set_nucleation_sites(case.sites)

    # the caller's own state buffers for the no-allocation entry point, in the
    # storage form the header asks for
    fluid = (np.arange(ny) >= Wr)[:, None] * np.ones((1, nx), bool)
    dev = rho0[None].astype(np.float64) - rho_ref
    f0 = np.where(fluid[None], W[:, None, None] * dev, 0.0).astype(np.float32)
    T_init = T0.copy()
    T_init[0] = np.float32(p.T_bottom)
    ftop0 = (W[[4, 7, 8], None] * (rho0[ny - 1][None].astype(np.float64) - rho_ref)).astype(np.float32)
    f = [torch.tensor(f0, device="cuda"), torch.empty_like(torch.tensor(f0, device="cuda"))]
    T = [torch.tensor(T_init, device="cuda"), torch.empty((ny, nx), dtype=torch.float32, device="cuda")]
    ft = [torch.tensor(ftop0, device="cuda"), torch.empty((3, nx), dtype=torch.float32, device="cuda")]
    sites = (hlb.hlb_site * len(case.sites))(*[hlb.hlb_site(*s) for s in case.sites])
    rho_ave = float(rho0[fluid].astype(np.float64).mean())
    U = 0.0
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    for call in range(2):
        rec = hlb.hlb_diag_record()
        a, b = call % 2, (call + 1) % 2
        st = hlb.lib().hlb_step_static(
            C.byref(p), len(case.sites), sites,
            C.c_void_p(f[a].data_ptr()), C.c_void_p(f[b].data_ptr()),
            C.c_void_p(T[a].data_ptr()), C.c_void_p(T[b].data_ptr()),
            C.c_void_p(ft[a].data_ptr()), C.c_void_p(ft[b].data_ptr()),
            rho_ave, U, C.byref(rec), C.c_void_p(stream.cuda_stream))
        assert st == hlb.HLB_OK, hlb.lib().hlb_strerror(st).decode()
        dom.step(1)
        rho_r, ux_r, uy_r, T_r = [t.cpu().numpy().astype(np.float64) for t in dom.read()]
        rho_s = f[b].cpu().numpy().astype(np.float64).sum(axis=0) + rho_ref
        T_s = T[b].cpu().numpy().astype(np.float64)
        assert np.abs(rho_s - rho_r)[fluid].max() / rho_r[fluid].max() < TOL
        assert np.abs(T_s - T_r).max() / np.abs(T_r).max() < TOL
        dg = dom.diag()
        assert rec.step == 1 and rec.error_flags == 0
        assert rec.mass == pytest.approx(dg.mass, rel=TOL)
        assert rec.rho_ave == pytest.approx(dg.rho_ave, rel=TOL)
        assert rec.q_bottom == pytest.approx(dg.q_bottom, rel=TOL, abs=1e-12)
        assert rec.q_interface == pytest.approx(dg.q_interface, rel=TOL, abs=1e-12)
        rho_ave, U = rec.rho_ave, max(0.0, rec.u_top)


def _static_call(p, bufs):
    """One call with the given (f_in, f_out, T_in, T_out) tensors; returns its status."""
    import torch
    from paper_1812_10375_gb300 import hlb
    rec = hlb.hlb_diag_record()
    fa, fb, Ta, Tb = bufs
    st = hlb.lib().hlb_step_static(C.byref(p), 0, None, C.c_void_p(fa.data_ptr()), C.c_void_p(fb.data_ptr()),
                                   C.c_void_p(Ta.data_ptr()), C.c_void_p(Tb.data_ptr()), None, None,
                                   float(p.rho_l), 0.0, C.byref(rec), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, rec


def _tiles(nx, ny):
    return -(-nx // TILE_W) * -(-ny // TILE_H)


def test_static_step_rejects_sizes_beyond_its_scratch():
    """A lattice wider than HLB_STATIC_MAX_NX or with more tiles than the static
    array holds partial sums for is refused with HLB_EINVAL.  The buffers are
    real (a few floats), so that a refusal that stopped working would show up as
    a wrong status, not as a kernel touching memory it does not own."""
    import torch
    from paper_1812_10375_gb300 import build, hlb
    build.build()
    small = [torch.zeros(64, dtype=torch.float32, device="cuda") for _ in range(4)]
    wide = hlb.default_params(16385, 64)
    assert _static_call(wide, small)[0] == hlb.HLB_EINVAL
    nx, ny = 16384, 56 * TILE_H  # 316 x 56 = 17,696 tiles
    assert _tiles(nx, ny) > MAX_TILES
    assert _static_call(hlb.default_params(nx, ny), small)[0] == hlb.HLB_EINVAL
    torch.cuda.synchronize()


def test_static_step_accepts_the_largest_lattice_its_scratch_serves():
    """The edge of the limit: 109 x 161 = 17,549 tiles (5668 x 4508 cells) runs,
    here one step of liquid at rest at the saturation temperature in a closed
    box, whose mass the step keeps."""
    import torch
    from paper_1812_10375_gb300 import build, hlb
    build.build()
    nx, ny = 109 * TILE_W, 161 * TILE_H
    assert _tiles(nx, ny) == MAX_TILES
    p = hlb.default_params(nx, ny)
    p.wall_rows = 2
    Tc, rho_l, rho_v, _ = hlb.eos_coexistence(p)
    p.rho_l, p.rho_v = rho_l, rho_v
    Ts = p.Ts_over_Tc * Tc
    p.T_bottom = p.T_top = Ts
    n = nx * ny
    f_in = torch.empty((9, n), dtype=torch.float32, device="cuda")
    f_in[:] = torch.tensor(W * (rho_l - rho_v), dtype=torch.float32, device="cuda")[:, None]
    bufs = [f_in, torch.empty_like(f_in), torch.full((n,), Ts, dtype=torch.float32, device="cuda"),
            torch.empty((n,), dtype=torch.float32, device="cuda")]
    st, rec = _static_call(p, bufs)
    assert st == hlb.HLB_OK, hlb.lib().hlb_strerror(st).decode()
    assert rec.step == 1 and rec.error_flags == 0
    fluid_rows = ny - p.wall_rows - 1
    assert rec.mass == pytest.approx(rho_l * nx * fluid_rows, rel=1e-6)
    del bufs, f_in
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
