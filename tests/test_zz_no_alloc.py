"""hlb_step_static, the entry point for callers that cannot allocate device
memory (for example a plug-in whose host application owns every allocation, or
a callback running inside someone else's graph capture): it takes its scratch
from a static device array inside the library instead of a workspace.  Two
calls in a row, through the C ABI, must agree with the regular workspace-based
step of the same domain within the parity tolerance (1e-5)."""
import ctypes as C

import numpy as np
import pytest

from paper_1812_10375_gb300 import workloads as wl

from helpers import coexistence, ragged_case

pytestmark = pytest.mark.gpu
TOL = 1e-5
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def test_static_step_matches_workspace_step_twice():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build, hlb
    from paper_1812_10375_gb300.config import params_for
    build.build()

    coex = coexistence()
    case = ragged_case()
    p, Tc = params_for(case, storage=hlb.HLB_STORE_PLAIN, rho_l=coex["rho_l"], rho_v=coex["rho_v"])
    rho0, T0 = wl.initial_fields(case, coex["rho_l"], coex["rho_v"], Tc)
    rho0 = rho0.astype(np.float32)
    T0 = T0.astype(np.float32)
    ny, nx, Wr = case.ny, case.nx, case.wall_rows

    # the regular entry points, with a library workspace
    dom = hlb.Domain(p)
    dom.set_fields(torch.tensor(rho0, device="cuda"), torch.tensor(T0, device="cuda"))
    dom.set_nucleation_sites(case.sites)

    # the caller's own state buffers for the no-allocation entry point
    fluid = (np.arange(ny) >= Wr)[:, None] * np.ones((1, nx), bool)
    f0 = np.where(fluid[None], W[:, None, None] * rho0[None].astype(np.float64), 0.0).astype(np.float32)
    T_init = T0.copy()
    T_init[0] = np.float32(p.T_bottom)
    ftop0 = (W[[4, 7, 8], None] * rho0[ny - 1][None].astype(np.float64)).astype(np.float32)
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
        rho_s = f[b].cpu().numpy().astype(np.float64).sum(axis=0)
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


def test_static_step_rejects_oversized_lattice():
    from paper_1812_10375_gb300 import build, hlb
    build.build()
    p = hlb.default_params(16385, 64)
    rec = hlb.hlb_diag_record()
    st = hlb.lib().hlb_step_static(C.byref(p), 0, None, C.c_void_p(8), C.c_void_p(8), C.c_void_p(8),
                                   C.c_void_p(8), None, None, 1.0, 0.0, C.byref(rec), None)
    assert st == hlb.HLB_EINVAL
