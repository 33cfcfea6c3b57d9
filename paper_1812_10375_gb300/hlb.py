"""Python binding of the C ABI in include/hlb.h (ctypes; argument marshalling only).

Every step of the model runs in the CUDA library ``libhlb.so``; this module only
converts arguments, owns the device workspace (a torch uint8 tensor) and the
stream, and maps status codes to exceptions.  It raises if the library has not
been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("HLB_LIB") or os.path.join(_PKG, "libhlb.so")

HLB_OK, HLB_EINVAL, HLB_ECUDA, HLB_EUNSTABLE, HLB_ETIMEOUT, HLB_ESTATE = 0, -1, -2, -3, -4, -5
HLB_TOP_WALL, HLB_TOP_CONST_RHO, HLB_TOP_CONVECTIVE = 0, 1, 2
HLB_STORE_DEVIATION, HLB_STORE_PLAIN = 0, 1
HLB_DIFF_FV, HLB_DIFF_ISO = 0, 1
HLB_BOTTOM_DIRICHLET, HLB_BOTTOM_FLUX = 0, 1
HLB_KIND_SPLIT, HLB_KIND_FUSED, HLB_KIND_MARCH = 0, 1, 2
TOP_KIND = {"wall": HLB_TOP_WALL, "const_rho": HLB_TOP_CONST_RHO, "convective": HLB_TOP_CONVECTIVE}


class hlb_params(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("nx", "ny", "wall_rows", "top_bc", "eos_T_fixed", "n_sub", "storage")] + [
        (n, C.c_double) for n in (
            "a", "b", "R", "omega", "Ts_over_Tc", "G", "sigma", "sigma_coef",
            "s_rho", "s_e", "s_zeta", "s_j", "s_q", "tau_l", "tau_v", "cv", "k",
            "rho_w", "cv_w", "lambda_w", "g_y", "Gw0", "T_bottom", "T_top", "rho_l", "rho_v")] + [
        ("diffusion", C.c_int), ("lambda_top", C.c_double), ("bottom_bc", C.c_int), ("q_in", C.c_double)]


class hlb_site(C.Structure):
    _fields_ = [("x_center", C.c_double), ("width", C.c_double), ("gw_min", C.c_double)]


class hlb_diag_record(C.Structure):
    _fields_ = [("step", C.c_longlong)] + [(n, C.c_double) for n in (
        "mass", "energy", "q_bottom", "q_top", "q_interface", "rho_ave", "u_top", "q_bottom_timeavg")] + [
        ("error_flags", C.c_int), ("vapour_coverage", C.c_double), ("vapour_coverage_timeavg", C.c_double)]


class HlbError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn}: {msg} (status {status})")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Load libhlb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1812_10375_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, sz, st = C.c_void_p, C.c_size_t, C.c_int
        P = C.POINTER
        sig = {
            "hlb_params_default": (None, [P(hlb_params), C.c_int, C.c_int]),
            "hlb_eos_coexistence": (st, [P(hlb_params), P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double)]),
            "hlb_workspace_bytes": (sz, [P(hlb_params)]),
            "hlb_init": (st, [P(vp), P(hlb_params), vp, sz, vp]),
            "hlb_set_fields": (st, [vp, vp, vp]),
            "hlb_set_wall": (st, [vp, C.c_double]),
            "hlb_set_nucleation_sites": (st, [vp, C.c_int, P(hlb_site)]),
            "hlb_step": (st, [vp, C.c_int]),
            "hlb_read": (st, [vp, vp, vp, vp, vp]),
            "hlb_diag": (st, [vp, P(hlb_diag_record)]),
            "hlb_reset_timeavg": (st, [vp]),
            "hlb_flux_history": (st, [vp, P(C.c_double), C.c_int, P(C.c_int)]),
            "hlb_destroy": (st, [vp]),
            "hlb_strerror": (C.c_char_p, [st]),
            "hlb_batch_workspace_bytes": (sz, [C.c_int, P(hlb_params)]),
            "hlb_batch_init": (st, [P(vp), C.c_int, P(hlb_params), vp, sz, vp]),
            "hlb_batch_set_fields": (st, [vp, C.c_int, vp, vp]),
            "hlb_batch_set_wall": (st, [vp, C.c_int, C.c_double]),
            "hlb_batch_set_nucleation_sites": (st, [vp, C.c_int, C.c_int, P(hlb_site)]),
            "hlb_batch_step": (st, [vp, C.c_int]),
            "hlb_batch_step_profiled": (st, [vp, vp, vp]),
            "hlb_batch_step_phases": (st, [vp, vp, vp, vp]),
            "hlb_batch_set_lanes": (st, [vp, C.c_int]),
            "hlb_batch_read": (st, [vp, C.c_int, vp, vp, vp, vp]),
            "hlb_batch_diag": (st, [vp, C.c_int, P(hlb_diag_record)]),
            "hlb_batch_flux_history": (st, [vp, C.c_int, P(C.c_double), C.c_int, P(C.c_int)]),
            "hlb_batch_stop": (st, [vp, C.c_int]),
            "hlb_batch_destroy": (st, [vp]),
            "hlb_tile_variants": (C.c_int, [P(C.c_int), P(C.c_int), P(C.c_int), C.c_int]),
            "hlb_variant_kind": (C.c_int, [C.c_int]),
            "hlb_variant_energy_rows": (C.c_int, [C.c_int]),
            "hlb_autotune": (st, [vp, C.c_int, P(C.c_int), P(C.c_float), C.c_int]),
            "hlb_batch_autotune": (st, [vp, C.c_int, P(C.c_int), P(C.c_float), C.c_int]),
            "hlb_set_tile_variant": (st, [vp, C.c_int]),
            "hlb_batch_set_tile_variant": (st, [vp, C.c_int]),
            "hlb_checkpoint_bytes": (sz, [P(hlb_params)]),
            "hlb_stable_substeps": (C.c_int, [P(hlb_params)]),
            "hlb_checkpoint_save": (st, [vp, vp, sz, P(sz)]),
            "hlb_checkpoint_load": (st, [vp, vp, sz]),
            "hlb_batch_checkpoint_save": (st, [vp, C.c_int, vp, sz, P(sz)]),
            "hlb_batch_checkpoint_load": (st, [vp, C.c_int, vp, sz]),
            "hlb_step_static": (st, [P(hlb_params), C.c_int, P(hlb_site), vp, vp, vp, vp, vp, vp,
                                     C.c_double, C.c_double, P(hlb_diag_record), vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(fn: str, status: int) -> int:
    if status != HLB_OK:
        raise HlbError(fn, status, lib().hlb_strerror(status).decode())
    return status


def default_params(nx: int, ny: int) -> hlb_params:
    p = hlb_params()
    lib().hlb_params_default(C.byref(p), nx, ny)
    return p


def eos_coexistence(p: hlb_params):
    """(Tc, rho_l, rho_v, h_fg) from the library's host-side Maxwell solver."""
    Tc, rl, rv, h = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    check("hlb_eos_coexistence", lib().hlb_eos_coexistence(C.byref(p), C.byref(Tc), C.byref(rl), C.byref(rv), C.byref(h)))
    return Tc.value, rl.value, rv.value, h.value


def workspace_bytes(p: hlb_params) -> int:
    return int(lib().hlb_workspace_bytes(C.byref(p)))


def stable_substeps(p: hlb_params) -> int:
    """N of Eq. (27) that n_sub = 0 selects (RK4 stability of the conduction operator)."""
    return int(lib().hlb_stable_substeps(C.byref(p)))


def checkpoint_bytes(p: hlb_params) -> int:
    """Largest checkpoint of a domain with parameters p (full flux history)."""
    return int(lib().hlb_checkpoint_bytes(C.byref(p)))


def _save_checkpoint(fn, name, params, *args) -> bytes:
    cap = checkpoint_bytes(params)
    buf = C.create_string_buffer(cap)
    n = C.c_size_t()
    check(name, fn(*args, buf, cap, C.byref(n)))
    return buf.raw[:n.value]


def write_checkpoint(path: str, blob: bytes, **meta):
    """Store a checkpoint (and optional scalar metadata) as an .npz file,
    replacing `path` atomically."""
    import numpy as np
    tmp = path + ".tmp.npz"
    np.savez(tmp, hlb_checkpoint=np.frombuffer(blob, dtype=np.uint8), **meta)
    os.replace(tmp, path)


def read_checkpoint(path: str):
    """(blob, metadata dict) of an .npz written by write_checkpoint."""
    import numpy as np
    with np.load(path) as z:
        meta = {k: z[k][()] for k in z.files if k != "hlb_checkpoint"}
        return z["hlb_checkpoint"].tobytes(), meta


def _ptr(t) -> C.c_void_p:
    if t is None:
        return C.c_void_p(None)
    import torch
    if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.float32):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


@dataclass
class Diag:
    step: int
    mass: float
    energy: float
    q_bottom: float
    q_top: float
    q_interface: float
    rho_ave: float
    u_top: float
    q_bottom_timeavg: float
    error_flags: int
    vapour_coverage: float = 0.0
    vapour_coverage_timeavg: float = 0.0


def tile_variants():
    n = lib().hlb_tile_variants(None, None, None, 0)
    w, h, t = (C.c_int * n)(), (C.c_int * n)(), (C.c_int * n)()
    lib().hlb_tile_variants(w, h, t, n)
    return [(w[k], h[k], t[k]) for k in range(n)]


def variant_kinds():
    """HLB_KIND_* of every compiled variant, in the order of tile_variants()."""
    n = lib().hlb_tile_variants(None, None, None, 0)
    return [int(lib().hlb_variant_kind(k)) for k in range(n)]


def variant_energy_rows():
    """Per compiled variant: the segment height of a split variant's row-walking
    energy kernel, 0 for the tiled energy kernel, -1 for the fused kinds."""
    n = lib().hlb_tile_variants(None, None, None, 0)
    return [int(lib().hlb_variant_energy_rows(k)) for k in range(n)]


def _autotune(fn, handle, steps, stream):
    import torch
    torch.cuda.current_stream().synchronize()
    n = lib().hlb_tile_variants(None, None, None, 0)
    ms = (C.c_float * n)()
    chosen = C.c_int()
    check("autotune", fn(handle, int(steps), C.byref(chosen), ms, n))
    return chosen.value, [ms[k] for k in range(n)]


class Domain:
    """One lattice domain living in a caller-owned (torch) device workspace."""

    def __init__(self, params: hlb_params, stream=None):
        import torch
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        nbytes = workspace_bytes(params)
        if nbytes == 0:
            raise ValueError("invalid hlb_params")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        aligned = (base + 255) & ~255
        self._h = C.c_void_p()
        check("hlb_init", lib().hlb_init(C.byref(self._h), C.byref(params), C.c_void_p(aligned), nbytes,
                                         C.c_void_p(self.stream.cuda_stream)))

    def _enter(self):
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())

    def _leave(self):
        import torch
        torch.cuda.current_stream().wait_stream(self.stream)

    def set_fields(self, rho, T):
        self._enter()
        check("hlb_set_fields", lib().hlb_set_fields(self._h, _ptr(rho), _ptr(T)))
        rho.record_stream(self.stream)
        T.record_stream(self.stream)
        self._leave()

    def set_wall(self, T_bottom: float):
        check("hlb_set_wall", lib().hlb_set_wall(self._h, float(T_bottom)))

    def set_nucleation_sites(self, sites):
        arr = (hlb_site * max(len(sites), 1))()
        for i, (xc, w, g) in enumerate(sites):
            arr[i] = hlb_site(float(xc), float(w), float(g))
        check("hlb_set_nucleation_sites", lib().hlb_set_nucleation_sites(self._h, len(sites), arr))

    def step(self, n: int = 1):
        self._enter()
        check("hlb_step", lib().hlb_step(self._h, int(n)))
        self._leave()

    def read(self):
        """(rho, ux, uy, T) as new float32 CUDA tensors of shape (ny, nx)."""
        import torch
        out = [torch.empty((self.ny, self.nx), dtype=torch.float32, device="cuda") for _ in range(4)]
        self._enter()
        check("hlb_read", lib().hlb_read(self._h, *[_ptr(t) for t in out]))
        for t in out:
            t.record_stream(self.stream)
        self._leave()
        return tuple(out)

    def diag(self, check_flags: bool = True) -> Diag:
        rec = hlb_diag_record()
        st = lib().hlb_diag(self._h, C.byref(rec))
        if st not in (HLB_OK, HLB_EUNSTABLE, HLB_ETIMEOUT) or (check_flags and st != HLB_OK):
            check("hlb_diag", st)
        return Diag(rec.step, rec.mass, rec.energy, rec.q_bottom, rec.q_top, rec.q_interface, rec.rho_ave,
                    rec.u_top, rec.q_bottom_timeavg, rec.error_flags, rec.vapour_coverage,
                    rec.vapour_coverage_timeavg)

    def reset_timeavg(self):
        check("hlb_reset_timeavg", lib().hlb_reset_timeavg(self._h))

    def flux_history(self, max_len=65536):
        """The per-step wall heat flux q_bottom since set_fields (FP64)."""
        import numpy as np
        buf = np.zeros(max_len, dtype=np.float64)
        n = C.c_int()
        check("hlb_flux_history", lib().hlb_flux_history(
            self._h, buf.ctypes.data_as(C.POINTER(C.c_double)), max_len, C.byref(n)))
        return buf[:n.value].copy()

    def checkpoint(self) -> bytes:
        """Byte image of the state after the last step (see hlb_checkpoint_save)."""
        self._enter()
        return _save_checkpoint(lib().hlb_checkpoint_save, "hlb_checkpoint_save", self.params, self._h)

    def restore(self, blob: bytes):
        """Replace the state by a checkpoint taken with checkpoint()."""
        self._enter()
        check("hlb_checkpoint_load", lib().hlb_checkpoint_load(self._h, blob, len(blob)))

    def autotune(self, steps_per_variant=8):
        """Time every compiled tile variant on this domain and keep the fastest."""
        return _autotune(lib().hlb_autotune, self._h, steps_per_variant, self.stream)

    def set_tile_variant(self, v):
        """Use compiled tile variant v (an index into tile_variants()) for later steps."""
        check("hlb_set_tile_variant", lib().hlb_set_tile_variant(self._h, int(v)))

    def close(self):
        if self._h:
            lib().hlb_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _sites_array(sites):
    arr = (hlb_site * max(len(sites), 1))()
    for i, (xc, w, g) in enumerate(sites):
        arr[i] = hlb_site(float(xc), float(w), float(g))
    return arr


def _event_handle(ev) -> C.c_void_p:
    """cudaEvent_t of a torch.cuda.Event (created on first use)."""
    if ev is None:
        return C.c_void_p(None)
    return C.c_void_p(ev.cuda_event)


class Batch:
    """Independent domains stepped together by one launch per step (boiling-curve sweep)."""

    def __init__(self, params_list, stream=None):
        import torch
        n = len(params_list)
        self.params = (hlb_params * n)(*params_list)
        self.n = n
        self.shapes = [(p.ny, p.nx) for p in params_list]
        nbytes = int(lib().hlb_batch_workspace_bytes(n, self.params))
        if nbytes == 0:
            raise ValueError("invalid hlb_params in batch")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        aligned = (self._ws.data_ptr() + 255) & ~255
        self._h = C.c_void_p()
        check("hlb_batch_init", lib().hlb_batch_init(C.byref(self._h), n, self.params, C.c_void_p(aligned), nbytes,
                                                     C.c_void_p(self.stream.cuda_stream)))

    def _enter(self):
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())

    def _leave(self):
        import torch
        torch.cuda.current_stream().wait_stream(self.stream)

    def set_fields(self, i, rho, T):
        self._enter()
        check("hlb_batch_set_fields", lib().hlb_batch_set_fields(self._h, i, _ptr(rho), _ptr(T)))
        rho.record_stream(self.stream)
        T.record_stream(self.stream)
        self._leave()

    def set_wall(self, i, T_bottom):
        check("hlb_batch_set_wall", lib().hlb_batch_set_wall(self._h, i, float(T_bottom)))

    def set_nucleation_sites(self, i, sites):
        check("hlb_batch_set_nucleation_sites",
              lib().hlb_batch_set_nucleation_sites(self._h, i, len(sites), _sites_array(sites)))

    def step(self, n=1):
        self._enter()
        check("hlb_batch_step", lib().hlb_batch_step(self._h, int(n)))
        self._leave()

    def step_profiled(self, ev_before, ev_after):
        """One step with torch.cuda.Event objects recorded around the step kernel
        (on the batch stream); no stream hand-off, for timing loops."""
        check("hlb_batch_step_profiled",
              lib().hlb_batch_step_profiled(self._h, _event_handle(ev_before), _event_handle(ev_after)))

    def step_phases(self, ev_before, ev_flow, ev_after):
        """One step with events before the step kernels, between the flow and
        the energy kernels of a split step, and after the step kernels."""
        check("hlb_batch_step_phases",
              lib().hlb_batch_step_phases(self._h, _event_handle(ev_before), _event_handle(ev_flow),
                                          _event_handle(ev_after)))

    def set_lanes(self, lanes):
        """Run the split step in 1 or 2 lanes (see hlb_batch_set_lanes)."""
        check("hlb_batch_set_lanes", lib().hlb_batch_set_lanes(self._h, int(lanes)))

    def read(self, i):
        import torch
        ny, nx = self.shapes[i]
        out = [torch.empty((ny, nx), dtype=torch.float32, device="cuda") for _ in range(4)]
        self._enter()
        check("hlb_batch_read", lib().hlb_batch_read(self._h, i, *[_ptr(t) for t in out]))
        for t in out:
            t.record_stream(self.stream)
        self._leave()
        return tuple(out)

    def read_into(self, i, rho=None, ux=None, uy=None, T=None):
        check("hlb_batch_read", lib().hlb_batch_read(self._h, i, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T)))

    def diag(self, i, check_flags=True) -> Diag:
        rec = hlb_diag_record()
        st = lib().hlb_batch_diag(self._h, i, C.byref(rec))
        if st not in (HLB_OK, HLB_EUNSTABLE, HLB_ETIMEOUT) or (check_flags and st != HLB_OK):
            check("hlb_batch_diag", st)
        return Diag(rec.step, rec.mass, rec.energy, rec.q_bottom, rec.q_top, rec.q_interface, rec.rho_ave,
                    rec.u_top, rec.q_bottom_timeavg, rec.error_flags, rec.vapour_coverage,
                    rec.vapour_coverage_timeavg)

    def flux_history(self, i, max_len=65536):
        import numpy as np
        buf = np.zeros(max_len, dtype=np.float64)
        n = C.c_int()
        check("hlb_batch_flux_history", lib().hlb_batch_flux_history(
            self._h, i, buf.ctypes.data_as(C.POINTER(C.c_double)), max_len, C.byref(n)))
        return buf[:n.value].copy()

    def stop(self, i):
        check("hlb_batch_stop", lib().hlb_batch_stop(self._h, i))

    def checkpoint(self, i) -> bytes:
        """Byte image of domain i's state after its last step."""
        self._enter()
        return _save_checkpoint(lib().hlb_batch_checkpoint_save, "hlb_batch_checkpoint_save", self.params[i],
                                self._h, int(i))

    def restore(self, i, blob: bytes):
        """Replace domain i's state by a checkpoint and make it active again."""
        self._enter()
        check("hlb_batch_checkpoint_load", lib().hlb_batch_checkpoint_load(self._h, int(i), blob, len(blob)))

    def autotune(self, steps_per_variant=8):
        """Time every compiled tile variant on this batch and keep the fastest."""
        return _autotune(lib().hlb_batch_autotune, self._h, steps_per_variant, self.stream)

    def set_tile_variant(self, v):
        """Use compiled tile variant v (an index into tile_variants()) for later steps."""
        check("hlb_batch_set_tile_variant", lib().hlb_batch_set_tile_variant(self._h, int(v)))

    def close(self):
        if self._h:
            lib().hlb_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
