"""Python binding of the C ABI in include/pflbm.h (ctypes).

Argument marshalling only: every step of the method runs in the CUDA
library ``_build/libpflbm.so``.  The functions keep the C names; a nonzero
status raises :class:`PflbmError`.  :class:`Domain` is a convenience owner
that takes its device workspace and stream from PyTorch (plumbing: PyTorch
provides memory and streams, never arithmetic of the method).

There is no fallback: if the library is missing or cannot be loaded every
call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

from . import build as _build

FORMS = ("STF1", "STF2", "CPF1", "CPF2", "PF1", "PF2", "CSF1", "CSF2")
FAMILY = {"STF": "STF1", "CPF": "CPF1", "PF": "PF1", "CSF": "CSF1"}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
FIELDS = ("phi", "rho", "ux", "uy", "P", "mu", "p_h", "Fx", "Fy")
NOALLOC_MAX_NODES = 8388608  # PFLBM_NOALLOC_MAX_NODES
PERIODIC, WALL, FREESLIP = 0, 1, 2

STATUS = {0: "PFLBM_OK", 1: "PFLBM_EINVAL", 2: "PFLBM_ENOMEM_WS", 3: "PFLBM_ECUDA",
          4: "PFLBM_EUNSTABLE", 5: "PFLBM_ETIMEOUT", 6: "PFLBM_ESTATE"}


class PflbmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {detail}".strip())


class pflbm_params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("W", ctypes.c_double), ("M", ctypes.c_double),
                ("tau_h", ctypes.c_double), ("rho1", ctypes.c_double), ("rho2", ctypes.c_double),
                ("nu1", ctypes.c_double), ("nu2", ctypes.c_double), ("gx", ctypes.c_double),
                ("gy", ctypes.c_double), ("rho0", ctypes.c_double),
                ("uw_bottom", ctypes.c_double), ("uw_top", ctypes.c_double),
                ("eps", ctypes.c_double), ("force", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("scale_f", ctypes.c_double),
                ("scale_h", ctypes.c_double)]


class pflbm_diag_geom(ctypes.Structure):
    _fields_ = [("xc", ctypes.c_double), ("yc", ctypes.c_double), ("r_in", ctypes.c_double),
                ("r_out", ctypes.c_double)]


class pflbm_diag(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "mass", "umax", "area1", "R_num", "p_in", "p_out", "dp", "sigma_num", "xc1", "yc1",
        "taylor_D", "nonfinite")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pflbm_bubble_diag(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "mass2", "xc2", "yc2", "uc2", "vc2", "area2", "perimeter", "circularity", "nonfinite")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every symbol include/pflbm.h declares, with its ctypes signature
_vp, _i, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
SIGNATURES = {
    "pflbm_workspace_bytes": (_sz, [_i, _i, _i]),
    "pflbm_create": (_i, [_i, _i, _i, _i, _i, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "pflbm_set_params": (_i, [_vp, ctypes.POINTER(pflbm_params)]),
    "pflbm_init_phi": (_i, [_vp, _vp, _i]),
    "pflbm_step": (_i, [_vp, _i]),
    "pflbm_set_graphs": (_i, [_vp, _i]),
    "pflbm_set_tma": (_i, [_vp, _i]),
    "pflbm_set_stage_mode": (_i, [_vp, _i]),
    "pflbm_get_stage_mode": (_i, [_vp]),
    "pflbm_autotune": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "pflbm_steps_done": (ctypes.c_longlong, [_vp]),
    "pflbm_read": (_i, [_vp, _i, _vp, _i]),
    "pflbm_read_fields": (_i, [_vp, _vp, _i]),
    "pflbm_read_populations": (_i, [_vp, _vp, _vp, _i]),
    "pflbm_diagnostics": (_i, [_vp, ctypes.POINTER(pflbm_diag_geom), ctypes.POINTER(pflbm_diag)]),
    "pflbm_bubble_diagnostics": (_i, [_vp, ctypes.POINTER(pflbm_bubble_diag)]),
    "pflbm_state_bytes": (_sz, [_vp]),
    "pflbm_save_state": (_i, [_vp, _vp, _i]),
    "pflbm_load_state": (_i, [_vp, _vp, _i]),
    "pflbm_destroy": (None, [_vp]),
    "pflbm_adjoint_scratch_bytes": (_sz, [_vp, _i, _i]),
    "pflbm_adjoint_run": (_i, [_vp, _vp, _i, _i, _vp, _vp, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), _vp, _sz]),
    "pflbm_batch_workspace_bytes": (_sz, [_i, ctypes.POINTER(_vp)]),
    "pflbm_batch_create": (_i, [_i, ctypes.POINTER(_vp), _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "pflbm_batch_step": (_i, [_vp, _i]),
    "pflbm_batch_set_graphs": (_i, [_vp, _i]),
    "pflbm_batch_set_config": (_i, [_vp, _i, _i]),
    "pflbm_batch_set_tile_rows": (_i, [_vp, _i]),
    "pflbm_batch_get_tile_rows": (_i, [_vp]),
    "pflbm_batch_autotune": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "pflbm_batch_items": (ctypes.c_longlong, [_vp]),
    "pflbm_batch_destroy": (None, [_vp]),
    "pflbm_field_diagnostics_noalloc": (_i, [_i, _i, _i, _i, _vp, ctypes.POINTER(pflbm_diag_geom),
                                         ctypes.POINTER(pflbm_diag), _vp]),
    "pflbm_status_str": (ctypes.c_char_p, [_i]),
    "pflbm_last_error": (ctypes.c_char_p, []),
    "pflbm_version": (ctypes.c_char_p, []),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpflbm.so (building it with nvcc first if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"CUDA library missing: {path}")
        _build.build()
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(st: int, where: str):
    if st != 0:
        L = load()
        raise PflbmError(st, where, L.pflbm_last_error().decode())


def _ptr(x) -> int:
    """Address of a torch tensor or numpy array (contiguous, float32 data)."""
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    assert x.flags["C_CONTIGUOUS"]
    return x.ctypes.data


def _on_device(x) -> int:
    return int(hasattr(x, "is_cuda") and x.is_cuda)


# ---------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------

def pflbm_workspace_bytes(nx: int, ny: int, storage: int) -> int:
    return int(load().pflbm_workspace_bytes(nx, ny, storage))


def pflbm_create(nx, ny, bc_x, bc_y, storage, workspace_ptr, ws_bytes, stream_ptr):
    h = ctypes.c_void_p()
    _check(load().pflbm_create(nx, ny, bc_x, bc_y, storage, workspace_ptr, ws_bytes,
                               stream_ptr, ctypes.byref(h)), "pflbm_create")
    return h


def pflbm_set_params(d, p: pflbm_params):
    _check(load().pflbm_set_params(d, ctypes.byref(p)), "pflbm_set_params")


def pflbm_init_phi(d, phi0):
    _check(load().pflbm_init_phi(d, _ptr(phi0), _on_device(phi0)), "pflbm_init_phi")


def pflbm_step(d, nsteps: int):
    _check(load().pflbm_step(d, int(nsteps)), "pflbm_step")


def pflbm_set_graphs(d, enable: bool):
    _check(load().pflbm_set_graphs(d, int(bool(enable))), "pflbm_set_graphs")


def pflbm_set_tma(d, enable: bool):
    _check(load().pflbm_set_tma(d, int(bool(enable))), "pflbm_set_tma")


STAGE_MODES = {"boxes": 0, "gather": 1, "march": 2, "gather8": 3}


def pflbm_set_stage_mode(d, mode: int):
    _check(load().pflbm_set_stage_mode(d, int(mode)), "pflbm_set_stage_mode")


def pflbm_get_stage_mode(d) -> int:
    return int(load().pflbm_get_stage_mode(d))


def pflbm_autotune(d, trial_steps: int) -> int:
    out = ctypes.c_int(-1)
    _check(load().pflbm_autotune(d, int(trial_steps), ctypes.byref(out)), "pflbm_autotune")
    return out.value


def pflbm_steps_done(d) -> int:
    return int(load().pflbm_steps_done(d))


def pflbm_read(d, field: int, dst):
    _check(load().pflbm_read(d, int(field), _ptr(dst), _on_device(dst)), "pflbm_read")


def pflbm_read_fields(d, dst):
    _check(load().pflbm_read_fields(d, _ptr(dst), _on_device(dst)), "pflbm_read_fields")


def pflbm_read_populations(d, f_out, h_out):
    dev = _on_device(f_out if f_out is not None else h_out)
    _check(load().pflbm_read_populations(d, None if f_out is None else _ptr(f_out),
                                         None if h_out is None else _ptr(h_out), dev),
           "pflbm_read_populations")


def pflbm_diagnostics(d, geom: Optional[pflbm_diag_geom]):
    out = pflbm_diag()
    st = load().pflbm_diagnostics(d, None if geom is None else ctypes.byref(geom),
                                  ctypes.byref(out))
    if st not in (0, 4):
        _check(st, "pflbm_diagnostics")
    return st, out


def pflbm_bubble_diagnostics(d):
    out = pflbm_bubble_diag()
    st = load().pflbm_bubble_diagnostics(d, ctypes.byref(out))
    if st not in (0, 4):
        _check(st, "pflbm_bubble_diagnostics")
    return st, out


def pflbm_field_diagnostics_noalloc(nx: int, ny: int, fields, geom: Optional[pflbm_diag_geom],
                                    stream=None, bc_x: int = 0, bc_y: int = 0):
    """FP64 diagnostics of device fields [PFLBM_NFIELDS][ny][nx] through the
    library's static scratch (no allocation); stream is a torch stream, a raw
    handle or None (legacy default stream); bc_x, bc_y the lattice's sides
    (pflbm_bc values).  Returns (status, pflbm_diag)."""
    out = pflbm_diag()
    handle = getattr(stream, "cuda_stream", stream)
    st = load().pflbm_field_diagnostics_noalloc(int(nx), int(ny), int(bc_x), int(bc_y),
                                                _ptr(fields),
                                                None if geom is None else ctypes.byref(geom),
                                                ctypes.byref(out), handle)
    if st not in (0, 4):
        _check(st, "pflbm_field_diagnostics_noalloc")
    return st, out


def pflbm_state_bytes(d) -> int:
    return int(load().pflbm_state_bytes(d))


def pflbm_save_state(d, dst):
    _check(load().pflbm_save_state(d, _ptr(dst), _on_device(dst)), "pflbm_save_state")


def pflbm_load_state(d, src):
    _check(load().pflbm_load_state(d, _ptr(src), _on_device(src)), "pflbm_load_state")


def pflbm_destroy(d):
    load().pflbm_destroy(d)


# ---------------------------------------------------------------------------
# convenience owner
# ---------------------------------------------------------------------------

def pflbm_adjoint_scratch_bytes(d, nsteps: int, ckpt_every: int) -> int:
    return int(load().pflbm_adjoint_scratch_bytes(d, int(nsteps), int(ckpt_every)))


def pflbm_adjoint_run(d, phi0, nsteps, ckpt_every, dJ_dphiT, dJ_dphi0, scratch):
    """All arrays are device tensors; returns (dJ/dsigma, dJ/dM)."""
    ds, dm = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().pflbm_adjoint_run(d, _ptr(phi0), int(nsteps), int(ckpt_every), _ptr(dJ_dphiT),
                                    _ptr(dJ_dphi0), ctypes.byref(ds), ctypes.byref(dm),
                                    _ptr(scratch), scratch.numel()), "pflbm_adjoint_run")
    return ds.value, dm.value


def _handles(doms):
    arr = (ctypes.c_void_p * len(doms))()
    for i, d in enumerate(doms):
        arr[i] = d.h.value if isinstance(d.h, ctypes.c_void_p) else d.h
    return arr


def pflbm_batch_workspace_bytes(handles) -> int:
    return int(load().pflbm_batch_workspace_bytes(len(handles), handles))


def pflbm_batch_create(handles, workspace_ptr, ws_bytes, stream_ptr):
    b = ctypes.c_void_p()
    _check(load().pflbm_batch_create(len(handles), handles, workspace_ptr, ws_bytes, stream_ptr,
                                     ctypes.byref(b)), "pflbm_batch_create")
    return b


def pflbm_batch_set_tile_rows(b, rows: int):
    _check(load().pflbm_batch_set_tile_rows(b, int(rows)), "pflbm_batch_set_tile_rows")


def pflbm_batch_get_tile_rows(b) -> int:
    return int(load().pflbm_batch_get_tile_rows(b))


def pflbm_batch_step(b, nsteps: int):
    _check(load().pflbm_batch_step(b, int(nsteps)), "pflbm_batch_step")


def pflbm_batch_set_graphs(b, enable: bool):
    _check(load().pflbm_batch_set_graphs(b, int(bool(enable))), "pflbm_batch_set_graphs")


def pflbm_batch_set_config(b, mode: int, ctas_per_sm: int):
    _check(load().pflbm_batch_set_config(b, int(mode), int(ctas_per_sm)), "pflbm_batch_set_config")


def pflbm_batch_autotune(b, trial_steps: int):
    m, c = ctypes.c_int(-1), ctypes.c_int(-1)
    _check(load().pflbm_batch_autotune(b, int(trial_steps), ctypes.byref(m), ctypes.byref(c)),
           "pflbm_batch_autotune")
    return m.value, c.value


def pflbm_batch_items(b) -> int:
    return int(load().pflbm_batch_items(b))


def pflbm_batch_destroy(b):
    load().pflbm_batch_destroy(b)


class Batch:
    """Many Domains (FP32, initialised) advanced by one launch per step."""

    def __init__(self, domains, stream=None):
        import torch
        self.domains = list(domains)
        self._handles = _handles(self.domains)
        nbytes = pflbm_batch_workspace_bytes(self._handles)
        dev = self.domains[0].device
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.Stream(dev)
        for d in self.domains:
            d.synchronize()
        self.h = pflbm_batch_create(self._handles, self.ws.data_ptr(), nbytes,
                                    self.stream.cuda_stream)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            pflbm_batch_destroy(h)
            self.h = None

    @property
    def items(self) -> int:
        return pflbm_batch_items(self.h)

    def step(self, n: int = 1) -> "Batch":
        pflbm_batch_step(self.h, n)
        return self

    def graphs(self, enable: bool = True) -> "Batch":
        pflbm_batch_set_graphs(self.h, enable)
        return self

    def config(self, mode, ctas_per_sm: int, rows: int = 16) -> "Batch":
        """Staging mode, CTAs per SM and tile rows (16, or 8 with gathers)."""
        mode = STAGE_MODES.get(mode, mode)
        if rows == 16:  # full tiles first: every mode accepts them
            pflbm_batch_set_tile_rows(self.h, 16)
            pflbm_batch_set_config(self.h, mode, ctas_per_sm)
        else:
            pflbm_batch_set_config(self.h, mode, ctas_per_sm)
            pflbm_batch_set_tile_rows(self.h, rows)
        return self

    @property
    def tile_rows(self) -> int:
        return pflbm_batch_get_tile_rows(self.h)

    def autotune(self, trial_steps: int = 5):
        """(mode, CTAs per SM, tile rows) of the fastest candidate, now set."""
        m, c = pflbm_batch_autotune(self.h, trial_steps)
        return {v: k for k, v in STAGE_MODES.items()}[m], c, self.tile_rows

    def synchronize(self):
        self.stream.synchronize()


def make_params(sigma=0.01, W=4.0, M=0.1, tau_h=1.0, rho1=1.0, rho2=1.0, nu1=0.1, nu2=0.1,
                gx=0.0, gy=0.0, rho0=float("nan"), uw_bottom=0.0, uw_top=0.0, eps=1e-6,
                form="STF1", scale_f=0.0, scale_h=0.0) -> pflbm_params:
    f = FORMS.index(FAMILY.get(form, form)) if isinstance(form, str) else int(form)
    return pflbm_params(sigma, W, M, tau_h, rho1, rho2, nu1, nu2, gx, gy, rho0, uw_bottom,
                        uw_top, eps, f, 0, scale_f, scale_h)


class Domain:
    """One lattice on the current CUDA device.  The workspace is a torch
    uint8 tensor; the stream is a torch stream (a new one by default)."""

    def __init__(self, nx: int, ny: int, wall_y: bool = False, storage: str = "fp32",
                 stream=None, device=None, wall_x: bool = False):
        import torch
        self.torch = torch
        self.nx, self.ny, self.wall = int(nx), int(ny), bool(wall_y)
        self.wall_x = bool(wall_x)  # free-slip side walls
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.device = torch.device(device or "cuda")
        nbytes = pflbm_workspace_bytes(nx, ny, self.storage)
        if nbytes == 0:
            raise PflbmError(1, "pflbm_workspace_bytes", f"invalid size {nx}x{ny}")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.h = pflbm_create(nx, ny, FREESLIP if wall_x else PERIODIC,
                              WALL if wall_y else PERIODIC, self.storage,
                              self.ws.data_ptr(), nbytes, self.stream.cuda_stream)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            pflbm_destroy(h)
            self.h = None

    def set_params(self, p: Optional[pflbm_params] = None, **kw) -> "Domain":
        pflbm_set_params(self.h, p if p is not None else make_params(**kw))
        return self

    def init_phi(self, phi0) -> "Domain":
        torch = self.torch
        if isinstance(phi0, np.ndarray):
            phi0 = np.ascontiguousarray(phi0, dtype=np.float32).reshape(self.ny, self.nx)
            pflbm_init_phi(self.h, phi0)
        else:
            phi0 = phi0.to(device=self.device, dtype=torch.float32).contiguous()
            with torch.cuda.stream(self.stream):
                pflbm_init_phi(self.h, phi0)
        return self

    def graphs(self, enable: bool = True) -> "Domain":
        pflbm_set_graphs(self.h, enable)
        return self

    def tma(self, enable: bool = True) -> "Domain":
        pflbm_set_tma(self.h, enable)
        return self

    def stage_mode(self, mode) -> "Domain":
        pflbm_set_stage_mode(self.h, STAGE_MODES.get(mode, mode))
        return self

    def stage(self) -> str:
        """Name of the stage mode the step kernel uses."""
        return {v: k for k, v in STAGE_MODES.items()}[pflbm_get_stage_mode(self.h)]

    def autotune(self, trial_steps: int = 20) -> str:
        m = pflbm_autotune(self.h, trial_steps)
        return {v: k for k, v in STAGE_MODES.items()}[m]

    def step(self, n: int = 1) -> "Domain":
        pflbm_step(self.h, n)
        return self

    @property
    def t(self) -> int:
        return pflbm_steps_done(self.h)

    def fields(self, device: bool = False):
        """All fields as a dict of [ny][nx] float32 arrays (numpy by default,
        torch tensors on the device with device=True)."""
        torch = self.torch
        if device:
            out = torch.empty((len(FIELDS), self.ny, self.nx), dtype=torch.float32,
                              device=self.device)
        else:
            out = np.empty((len(FIELDS), self.ny, self.nx), dtype=np.float32)
        pflbm_read_fields(self.h, out)
        if device:
            self.stream.synchronize()
        return {k: out[i] for i, k in enumerate(FIELDS)}

    def read(self, field: str) -> np.ndarray:
        out = np.empty((self.ny, self.nx), dtype=np.float32)
        pflbm_read(self.h, FIELDS.index(field), out)
        return out

    def populations(self):
        f = np.empty((9, self.ny, self.nx), dtype=np.float32)
        h = np.empty((9, self.ny, self.nx), dtype=np.float32)
        pflbm_read_populations(self.h, f, h)
        return f, h

    def diagnostics(self, xc=None, yc=None, r_in=None, r_out=None):
        geom = None
        if xc is not None:
            geom = pflbm_diag_geom(xc, yc, r_in, r_out)
        st, d = pflbm_diagnostics(self.h, geom)
        out = d.as_dict()
        out["status"] = STATUS[st]
        return out

    def bubble_diagnostics(self):
        """Rising-bubble quantities (Sec. 5.4) in lattice units."""
        st, d = pflbm_bubble_diagnostics(self.h)
        out = d.as_dict()
        out["status"] = STATUS[st]
        return out

    def save_state(self) -> np.ndarray:
        buf = np.empty(pflbm_state_bytes(self.h), dtype=np.uint8)
        pflbm_save_state(self.h, buf)
        return buf

    def load_state(self, buf: np.ndarray) -> "Domain":
        pflbm_load_state(self.h, np.ascontiguousarray(buf))
        return self

    def synchronize(self):
        self.stream.synchronize()
