"""Thin ctypes binding of libpond (include/pond.h).

Argument marshalling only: every step of the PonD path runs in the library's CUDA
kernels.  PyTorch supplies device memory (the workspace and device-side arrays) and the
CUDA stream.  There is no CPU fallback: if the shared library has not been built, or no
CUDA device is present, the calls raise.

The functions carry the C names (``pond_create``, ``pond_set_state``, ``pond_step``,
``pond_get_moments``, ``pond_get_populations``, ``pond_get_stats``, ``pond_destroy`` ...);
``Simulation`` wraps one ``pond_sim`` with its workspace.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("POND_LIB") or os.path.join(_HERE, "_build", "libpond.so")

POND_OK, POND_EINVAL, POND_ENOMEM, POND_ECUDA, POND_ENONPHYSICAL, POND_ENOCONV = 0, -1, -2, -3, -4, -5
POND_D2Q16, POND_D2Q25 = 16, 25
POND_SPLIT_TOTAL, POND_SPLIT_INTERNAL, POND_SPLIT_NT = 0, 1, 2
POND_FP64, POND_MIXED_FP32, POND_MIXED_FP16, POND_MIXED_BF16 = 0, 1, 2, 3
POND_BC_PERIODIC, POND_BC_OUTFLOW, POND_BC_WALL, POND_BC_INFLOW = 0, 1, 2, 3

PRECISIONS = {"fp64": POND_FP64, "fp32": POND_MIXED_FP32, "fp16": POND_MIXED_FP16,
              "bf16": POND_MIXED_BF16}
SPLITS = {"total": POND_SPLIT_TOTAL, "internal": POND_SPLIT_INTERNAL, "nt": POND_SPLIT_NT}
BCS = {"periodic": POND_BC_PERIODIC, "outflow": POND_BC_OUTFLOW, "wall": POND_BC_WALL,
       "inflow": POND_BC_INFLOW}
SIDES = {"x_low": 0, "x_high": 1, "y_low": 2, "y_high": 3}

# Symbols the header declares (checked by the ABI test).
EXPORTS = ("pond_config_default", "pond_workspace_bytes", "pond_create", "pond_set_state",
           "pond_set_populations", "pond_step", "pond_get_moments", "pond_get_populations",
           "pond_get_stats", "pond_sync", "pond_destroy", "pond_strerror", "pond_version",
           "pond_state_bytes", "pond_export_state", "pond_import_state", "pond_step_static",
           "pond_batch_workspace_bytes", "pond_batch_create", "pond_batch_step",
           "pond_batch_use_graph", "pond_batch_destroy", "pond_get_launch", "pond_set_launch",
           "pond_autotune", "pond_autotune_clear", "pond_set_boundary_profile",
           "pond_batch_set_state", "pond_batch_get_moments", "pond_alu_peak")
POND_TUNE_APPLY, POND_TUNE_RETIME = 1, 2


class pond_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("lattice", ctypes.c_int32),
                ("split", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("interp_order", ctypes.c_int32), ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("pc_tol", ctypes.c_double),
                ("pc_max_iter", ctypes.c_int32), ("pc_fixed_iters", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("halo", ctypes.c_int32),
                ("grad_order", ctypes.c_int32), ("wall", (ctypes.c_double * 4) * 4)]


class pond_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("node_updates", ctypes.c_int64),
                ("pc_iters_total", ctypes.c_int64), ("pc_iters_max", ctypes.c_int32),
                ("status", ctypes.c_int32), ("nonconv_updates", ctypes.c_int64),
                ("first_bad_node", ctypes.c_int64), ("halo_fallbacks", ctypes.c_int64)]


class pond_tuning(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("halo", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("ms_per_step", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PondError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (%d)" % (what, strerror(status), status))


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpond.so (raises if it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libpond is not built (%s missing): run "
                               "`python -m paper_2405_11489_gb300.build`" % path)
        lib = ctypes.CDLL(path)
        vp, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
        P = ctypes.POINTER
        lib.pond_config_default.argtypes = [P(pond_config), i32, i32]
        lib.pond_workspace_bytes.argtypes = [P(pond_config), P(sz)]
        lib.pond_create.argtypes = [P(pond_config), vp, sz, vp, P(vp)]
        lib.pond_set_state.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int]
        lib.pond_set_populations.argtypes = [vp] + [vp] * 5 + [ctypes.c_int]
        lib.pond_step.argtypes = [vp, i32]
        lib.pond_get_moments.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int]
        lib.pond_get_populations.argtypes = [vp] + [vp] * 5 + [ctypes.c_int]
        lib.pond_get_stats.argtypes = [vp, P(pond_stats)]
        lib.pond_sync.argtypes = [vp]
        lib.pond_destroy.argtypes = [vp]
        lib.pond_state_bytes.argtypes = [P(pond_config), P(sz), P(sz)]
        lib.pond_export_state.argtypes = [vp, vp, vp, ctypes.c_int]
        lib.pond_import_state.argtypes = [vp, vp, vp, ctypes.c_int]
        lib.pond_step_static.argtypes = [P(pond_config), vp, vp, i32, vp, P(pond_stats)]
        lib.pond_batch_workspace_bytes.argtypes = [i32, P(sz)]
        lib.pond_batch_create.argtypes = [P(vp), i32, vp, sz, vp, P(vp)]
        lib.pond_batch_step.argtypes = [vp, i32]
        lib.pond_batch_set_state.argtypes = [vp, P(vp), P(vp), P(vp), P(vp), ctypes.c_int]
        lib.pond_batch_get_moments.argtypes = [vp, P(vp), P(vp), P(vp), P(vp), ctypes.c_int]
        lib.pond_batch_use_graph.argtypes = [vp, i32]
        lib.pond_batch_destroy.argtypes = [vp]
        lib.pond_get_launch.argtypes = [vp, P(pond_tuning)]
        lib.pond_set_launch.argtypes = [vp, i32, i32, i32]
        lib.pond_autotune.argtypes = [vp, vp, sz, i32, i32, P(pond_tuning)]
        lib.pond_autotune_clear.argtypes = []
        lib.pond_set_boundary_profile.argtypes = [vp, i32, vp, ctypes.c_int]
        lib.pond_alu_peak.argtypes = [i32, i32, vp, P(ctypes.c_double), P(ctypes.c_float)]
        lib.pond_strerror.argtypes = [ctypes.c_int]
        lib.pond_strerror.restype = ctypes.c_char_p
        lib.pond_version.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("pond_strerror", "pond_version", "pond_autotune_clear"):
                getattr(lib, name).restype = ctypes.c_int
        lib.pond_autotune_clear.restype = None
        _lib = lib
        return lib


def strerror(status: int) -> str:
    try:
        return load_library().pond_strerror(status).decode()
    except RuntimeError:
        return "status %d" % status


def _check(rc, what, allow=()):
    if rc != POND_OK and rc not in allow:
        raise PondError(rc, what)
    return rc


# ---------------------------------------------------------------------------------------
# Functions with the C names (argument marshalling only)
# ---------------------------------------------------------------------------------------
def pond_config_default(nx: int, ny: int) -> pond_config:
    cfg = pond_config()
    _check(load_library().pond_config_default(ctypes.byref(cfg), nx, ny), "pond_config_default")
    return cfg


def pond_workspace_bytes(cfg: pond_config) -> int:
    n = ctypes.c_size_t(0)
    _check(load_library().pond_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)), "pond_workspace_bytes")
    return n.value


def pond_create(cfg: pond_config, workspace_ptr: int, nbytes: int, stream_ptr: int) -> int:
    h = ctypes.c_void_p(0)
    _check(load_library().pond_create(ctypes.byref(cfg), ctypes.c_void_p(workspace_ptr), nbytes,
                                      ctypes.c_void_p(stream_ptr), ctypes.byref(h)), "pond_create")
    return h.value


def pond_set_state(h, rho, ux, uy, T, on_device: int) -> int:
    return load_library().pond_set_state(h, rho, ux, uy, T, on_device)


def pond_set_populations(h, f, g, ux, uy, T, on_device: int) -> int:
    return load_library().pond_set_populations(h, f, g, ux, uy, T, on_device)


def pond_step(h, nsteps: int) -> int:
    return load_library().pond_step(h, nsteps)


def pond_get_moments(h, rho, ux, uy, T, on_device: int) -> int:
    return load_library().pond_get_moments(h, rho, ux, uy, T, on_device)


def pond_get_populations(h, f, g, ux, uy, T, on_device: int) -> int:
    return load_library().pond_get_populations(h, f, g, ux, uy, T, on_device)


def pond_get_stats(h):
    st = pond_stats()
    rc = load_library().pond_get_stats(h, ctypes.byref(st))
    return rc, st


def pond_state_bytes(cfg: pond_config):
    m, n = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(load_library().pond_state_bytes(ctypes.byref(cfg), ctypes.byref(m), ctypes.byref(n)),
           "pond_state_bytes")
    return m.value, n.value


def pond_export_state(h, mac, neq, on_device: int) -> int:
    return load_library().pond_export_state(h, mac, neq, on_device)


def pond_import_state(h, mac, neq, on_device: int) -> int:
    return load_library().pond_import_state(h, mac, neq, on_device)


def pond_step_static(cfg: pond_config, mac_ptr: int, neq_ptr: int, nsteps: int, stream_ptr: int,
                     want_stats: bool = True):
    """Advance a raw state held in the caller's device buffers in place, allocating nothing
    (the library's static device array holds the second state copy); returns (rc, stats)."""
    st = pond_stats()
    rc = load_library().pond_step_static(ctypes.byref(cfg), ctypes.c_void_p(mac_ptr),
                                         ctypes.c_void_p(neq_ptr), nsteps,
                                         ctypes.c_void_p(stream_ptr),
                                         ctypes.byref(st) if want_stats else None)
    return rc, st


def pond_alu_peak(fp64: bool, iters: int, stream_ptr: int = 0):
    """One launch of independent FMA chains on the current device (FP32, or FP64 with fp64);
    returns (flop executed, milliseconds)."""
    flop, ms = ctypes.c_double(0.0), ctypes.c_float(0.0)
    rc = load_library().pond_alu_peak(1 if fp64 else 0, iters, ctypes.c_void_p(stream_ptr),
                                      ctypes.byref(flop), ctypes.byref(ms))
    if rc != POND_OK:
        raise PondError(rc, "pond_alu_peak")
    return flop.value, ms.value


def pond_batch_workspace_bytes(count: int) -> int:
    n = ctypes.c_size_t(0)
    _check(load_library().pond_batch_workspace_bytes(count, ctypes.byref(n)), "pond_batch_workspace_bytes")
    return n.value


def pond_batch_create(handles, workspace_ptr: int, nbytes: int, stream_ptr: int) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    h = ctypes.c_void_p(0)
    _check(load_library().pond_batch_create(arr, len(handles), ctypes.c_void_p(workspace_ptr), nbytes,
                                            ctypes.c_void_p(stream_ptr), ctypes.byref(h)),
           "pond_batch_create")
    return h.value


def _ptr_array(ptrs):
    if ptrs is None:
        return None
    return (ctypes.c_void_p * len(ptrs))(*[p or None for p in ptrs])


def pond_batch_set_state(h, rho, ux, uy, T, on_device: int) -> int:
    """rho, ux, uy, T: sequences of member pointers (ints)."""
    return load_library().pond_batch_set_state(h, _ptr_array(rho), _ptr_array(ux), _ptr_array(uy),
                                               _ptr_array(T), on_device)


def pond_batch_get_moments(h, rho, ux, uy, T, on_device: int) -> int:
    return load_library().pond_batch_get_moments(h, _ptr_array(rho), _ptr_array(ux), _ptr_array(uy),
                                                 _ptr_array(T), on_device)


def pond_batch_step(h, nsteps: int) -> int:
    return load_library().pond_batch_step(h, nsteps)


def pond_batch_use_graph(h, steps_per_graph: int) -> int:
    return load_library().pond_batch_use_graph(h, steps_per_graph)


def pond_batch_destroy(h) -> int:
    return load_library().pond_batch_destroy(h)


def pond_get_launch(h) -> pond_tuning:
    t = pond_tuning()
    _check(load_library().pond_get_launch(h, ctypes.byref(t)), "pond_get_launch")
    return t


def pond_set_launch(h, tile_x: int, tile_y: int, halo: int) -> int:
    return load_library().pond_set_launch(h, tile_x, tile_y, halo)


def pond_autotune(h, scratch_ptr: int, nbytes: int, steps: int, flags: int):
    t = pond_tuning()
    rc = load_library().pond_autotune(h, ctypes.c_void_p(scratch_ptr), nbytes, steps, flags, ctypes.byref(t))
    return rc, t


def pond_autotune_clear() -> None:
    load_library().pond_autotune_clear()


def pond_set_boundary_profile(h, side: int, state, on_device: int) -> int:
    return load_library().pond_set_boundary_profile(h, side, state, on_device)


def pond_sync(h) -> int:
    return load_library().pond_sync(h)


def pond_destroy(h) -> int:
    return load_library().pond_destroy(h)


# ---------------------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------------------
@dataclass
class Config:
    nx: int
    ny: int
    lattice: int = 16
    split: str = "total"
    precision: str = "fp32"
    interp_order: int = 3
    bc_x: str = "periodic"
    bc_y: str = "periodic"
    gamma: float = 1.4
    mu: float = 1e-3
    pc_tol: float | None = None
    pc_max_iter: int = 20
    pc_fixed_iters: int = 0
    tile_x: int = 0
    tile_y: int = 0
    halo: int = 0
    grad_order: int = 0       # 0: the lattice's (3 on D2Q16, 4 on D2Q25)
    walls: tuple | None = None  # four (u_x, u_y, T, rho): x-low, x-high, y-low, y-high
    # boundaries per axis: "periodic", "outflow", "wall" (both sides prescribed) or "inflow"
    # (low side prescribed, high side outflow)

    def to_c(self) -> pond_config:
        tol = self.pc_tol if self.pc_tol is not None else (1e-12 if self.precision == "fp64" else 1e-6)
        return pond_config(nx=self.nx, ny=self.ny, lattice=self.lattice, split=SPLITS[self.split],
                           precision=PRECISIONS[self.precision], interp_order=self.interp_order,
                           bc_x=BCS[self.bc_x], bc_y=BCS[self.bc_y], gamma=self.gamma, mu=self.mu,
                           pc_tol=tol, pc_max_iter=self.pc_max_iter,
                           pc_fixed_iters=self.pc_fixed_iters, tile_x=self.tile_x,
                           tile_y=self.tile_y, halo=self.halo, grad_order=self.grad_order,
                           wall=self._walls())

    def _walls(self):
        w = ((ctypes.c_double * 4) * 4)()
        for k, state in enumerate(self.walls or [(0.0, 0.0, 1.0, 1.0)] * 4):
            for j in range(4):
                w[k][j] = float(state[j])
        return w

    @property
    def Q(self) -> int:
        return self.lattice


def _dptr(t) -> int:
    return int(t.data_ptr())


class Simulation:
    """One pond_sim with a caller-owned (PyTorch) device workspace."""

    def __init__(self, cfg: Config, device="cuda:0", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libpond needs a CUDA device")
        self.torch = torch
        self.cfg = cfg
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._c = cfg.to_c()
        with torch.cuda.device(self.device):
            self.ws_bytes = pond_workspace_bytes(self._c)
            self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
            base = _dptr(self.workspace)
            self._ws_ptr = (base + 255) // 256 * 256
            self.handle = pond_create(self._c, self._ws_ptr, self.ws_bytes, self.stream.cuda_stream)

    # -- state in -------------------------------------------------------------------------
    def set_state(self, rho, ux, uy, T):
        """Fields [ny][nx]: numpy (host copy inside the library) or CUDA tensors (float64)."""
        torch = self.torch
        shape = (self.cfg.ny, self.cfg.nx)
        if isinstance(rho, torch.Tensor):
            arrs = [a.to(device=self.device, dtype=torch.float64).contiguous().reshape(shape)
                    for a in (rho, ux, uy, T)]
            with torch.cuda.device(self.device):
                rc = pond_set_state(self.handle, *[_dptr(a) for a in arrs], 1)
                self._keep = arrs
        else:
            arrs = [np.ascontiguousarray(np.broadcast_to(a, shape), dtype=np.float64) for a in (rho, ux, uy, T)]
            with torch.cuda.device(self.device):
                rc = pond_set_state(self.handle, *[a.ctypes.data for a in arrs], 0)
        _check(rc, "pond_set_state")

    def set_boundary_profile(self, side, state=None):
        """Per-position states [n][4] (u_x, u_y, T, rho) of a prescribed side ("x_low",
        "x_high", "y_low", "y_high" or 0..3; n = ny for the x sides, nx for the y sides):
        numpy (checked and copied by the library) or a CUDA float64 tensor; None restores
        the side's uniform state."""
        torch = self.torch
        w = SIDES[side] if isinstance(side, str) else int(side)
        if not 0 <= w <= 3:
            raise ValueError("side %r" % (side,))
        n = self.cfg.ny if w < 2 else self.cfg.nx
        if state is not None and tuple(state.shape) != (n, 4):
            raise ValueError("profile of side %d: shape %s, expected (%d, 4)" % (w, tuple(state.shape), n))
        with torch.cuda.device(self.device):
            if state is None:
                rc = pond_set_boundary_profile(self.handle, w, None, 0)
            elif isinstance(state, torch.Tensor):
                t = state.to(device=self.device, dtype=torch.float64).contiguous()
                rc = pond_set_boundary_profile(self.handle, w, _dptr(t), 1)
                self.stream.synchronize()          # the copy has read t
            else:
                a = np.ascontiguousarray(state, dtype=np.float64)
                rc = pond_set_boundary_profile(self.handle, w, a.ctypes.data, 0)
        _check(rc, "pond_set_boundary_profile")

    def set_populations(self, f, g, ux, uy, T):
        """Populations [Q][ny][nx] in the frames (ux, uy, T) [ny][nx] (numpy or tensors)."""
        torch = self.torch
        Q = self.cfg.lattice
        shape = (self.cfg.ny, self.cfg.nx)
        def dev(a, s):
            return torch.as_tensor(np.asarray(a) if not isinstance(a, torch.Tensor) else a,
                                   dtype=torch.float64).to(self.device).contiguous().reshape(s)
        arrs = [dev(f, (Q,) + shape), dev(g, (Q,) + shape)] + [dev(a, shape) for a in (ux, uy, T)]
        with torch.cuda.device(self.device):
            rc = pond_set_populations(self.handle, *[_dptr(a) for a in arrs], 1)
            self.stream.synchronize()
        _check(rc, "pond_set_populations")

    # -- stepping -------------------------------------------------------------------------
    def step(self, n: int = 1):
        with self.torch.cuda.device(self.device):
            _check(pond_step(self.handle, n), "pond_step")

    # -- state out ------------------------------------------------------------------------
    def moments(self, on_device: bool = False, allow=(POND_ENOCONV,)):
        """(rho, ux, uy, T) as numpy arrays (host) or CUDA tensors (on_device)."""
        torch = self.torch
        shape = (self.cfg.ny, self.cfg.nx)
        with torch.cuda.device(self.device):
            if on_device:
                out = [torch.empty(shape, dtype=torch.float64, device=self.device) for _ in range(4)]
                rc = pond_get_moments(self.handle, *[_dptr(a) for a in out], 1)
            else:
                out = [np.empty(shape) for _ in range(4)]
                rc = pond_get_moments(self.handle, *[a.ctypes.data for a in out], 0)
        self.last_status = rc
        _check(rc, "pond_get_moments", allow)
        return tuple(out)

    def populations(self, allow=(POND_ENOCONV,)):
        """(f, g, ux, uy, T) as numpy arrays, each node in its own frame."""
        torch = self.torch
        Q = self.cfg.lattice
        ny, nx = self.cfg.ny, self.cfg.nx
        with torch.cuda.device(self.device):
            f = torch.empty((Q, ny, nx), dtype=torch.float64, device=self.device)
            g = torch.empty_like(f)
            fr = [torch.empty((ny, nx), dtype=torch.float64, device=self.device) for _ in range(3)]
            rc = pond_get_populations(self.handle, _dptr(f), _dptr(g), *[_dptr(a) for a in fr], 1)
        self.last_status = rc
        _check(rc, "pond_get_populations", allow)
        return tuple(a.cpu().numpy() for a in [f, g] + fr)

    def export_state(self, on_device: bool = True):
        """Raw state (checkpoint): (mac, neq) as uint8 CUDA tensors (or numpy arrays)."""
        torch = self.torch
        mb, nb = pond_state_bytes(self._c)
        with torch.cuda.device(self.device):
            if on_device:
                mac = torch.empty(mb, dtype=torch.uint8, device=self.device)
                neq = torch.empty(nb, dtype=torch.uint8, device=self.device)
                rc = pond_export_state(self.handle, _dptr(mac), _dptr(neq), 1)
            else:
                mac = np.empty(mb, dtype=np.uint8)
                neq = np.empty(nb, dtype=np.uint8)
                rc = pond_export_state(self.handle, mac.ctypes.data, neq.ctypes.data, 0)
        _check(rc, "pond_export_state", (POND_ENOCONV,))
        return mac, neq

    def import_state(self, mac, neq):
        torch = self.torch
        with torch.cuda.device(self.device):
            if isinstance(mac, torch.Tensor):
                rc = pond_import_state(self.handle, _dptr(mac), _dptr(neq), 1)
                self.stream.synchronize()
            else:
                mac = np.ascontiguousarray(mac)
                neq = np.ascontiguousarray(neq)
                rc = pond_import_state(self.handle, mac.ctypes.data, neq.ctypes.data, 0)
        _check(rc, "pond_import_state")

    def stats(self):
        with self.torch.cuda.device(self.device):
            rc, st = pond_get_stats(self.handle)
        return rc, st

    # -- launch shape ---------------------------------------------------------------------
    def launch(self) -> dict:
        """Current tile and halo of the step kernel."""
        t = pond_get_launch(self.handle)
        return {"tile_x": t.tile_x, "tile_y": t.tile_y, "halo": t.halo}

    def set_launch(self, tile_x: int, tile_y: int, halo: int):
        with self.torch.cuda.device(self.device):
            _check(pond_set_launch(self.handle, tile_x, tile_y, halo), "pond_set_launch")

    def autotune(self, steps: int = 3, apply: bool = True, retime: bool = False) -> dict:
        """Time the candidate launch shapes on a copy of the current state (pond_autotune)
        and, with apply, use the fastest; the result is cached per problem class."""
        torch = self.torch
        flags = (POND_TUNE_APPLY if apply else 0) | (POND_TUNE_RETIME if retime else 0)
        with torch.cuda.device(self.device):
            scratch = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
            ptr = (_dptr(scratch) + 255) // 256 * 256
            rc, t = pond_autotune(self.handle, ptr, self.ws_bytes, steps, flags)
            self.stream.synchronize()
            del scratch
        _check(rc, "pond_autotune")
        return t.as_dict()

    def sync(self):
        with self.torch.cuda.device(self.device):
            return pond_sync(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            with self.torch.cuda.device(self.device):
                pond_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several Simulations advanced together: one kernel launch per time step (pond_batch)."""

    def __init__(self, sims, stream=None):
        import torch
        self.torch = torch
        self.sims = list(sims)
        self.device = self.sims[0].device
        self.stream = stream if stream is not None else self.sims[0].stream
        with torch.cuda.device(self.device):
            nb = pond_batch_workspace_bytes(len(self.sims))
            self.workspace = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
            ptr = (int(self.workspace.data_ptr()) + 255) // 256 * 256
            self.handle = pond_batch_create([s.handle for s in self.sims], ptr, nb,
                                            self.stream.cuda_stream)

    def use_graph(self, steps_per_graph: int):
        with self.torch.cuda.device(self.device):
            _check(pond_batch_use_graph(self.handle, steps_per_graph), "pond_batch_use_graph")

    def step(self, n: int = 1):
        with self.torch.cuda.device(self.device):
            _check(pond_batch_step(self.handle, n), "pond_batch_step")

    def set_state(self, fields):
        """fields: one (rho, ux, uy, T) per member, numpy arrays (host input, checked) or CUDA
        float64 tensors (device input), shaped [ny][nx] of that member."""
        torch = self.torch
        cols, keep = [[], [], [], []], []
        on_device = isinstance(fields[0][0], torch.Tensor)
        for sim, f in zip(self.sims, fields):
            shape = (sim.cfg.ny, sim.cfg.nx)
            for k, a in enumerate(f):
                if on_device:
                    a = a.to(device=self.device, dtype=torch.float64).contiguous().reshape(shape)
                    cols[k].append(_dptr(a))
                else:
                    a = np.ascontiguousarray(np.broadcast_to(a, shape), dtype=np.float64)
                    cols[k].append(a.ctypes.data)
                keep.append(a)
        with torch.cuda.device(self.device):
            rc = pond_batch_set_state(self.handle, *cols, 1 if on_device else 0)
        self._keep = keep
        _check(rc, "pond_batch_set_state")

    def moments(self, allow=(POND_OK, POND_ENOCONV)):
        """Every member's (rho, ux, uy, T) as float64 numpy arrays, one synchronisation."""
        outs = [[np.empty((s.cfg.ny, s.cfg.nx)) for _ in range(4)] for s in self.sims]
        cols = [[o[k].ctypes.data for o in outs] for k in range(4)]
        with self.torch.cuda.device(self.device):
            rc = pond_batch_get_moments(self.handle, *cols, 0)
        _check(rc, "pond_batch_get_moments", allow=allow)
        return [tuple(o) for o in outs]

    def close(self):
        if getattr(self, "handle", None):
            with self.torch.cuda.device(self.device):
                pond_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
