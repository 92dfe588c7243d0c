"""FP64 CPU oracle for the PonD double-distribution BGK step (arXiv 2405.11489).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product library (``paper_2405_11489_gb300``) never imports it and shares no code,
header or constant with it.

The arithmetic lives in ``pond_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module builds it with gcc and wraps it with ctypes.
``riemann.py`` holds the exact Riemann solver used to pin the Sod problem.

Pins (each in ``tests/test_oracle_*.py``): Table I nodes/weights and quadrature
exactness (closed forms), frame-transform moment invariance to order 3 and the
expanded coefficient formulas of Sec. III.A.1, equilibrium moments to round-off,
uniform supersonic flow invariance, per-node and global conservation, exact cubic
reproduction of the interpolation, Sod against the exact Riemann solution, and the
shear/thermal decay rates and sound speed set by tau (Sec. III.B).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "pond_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile pond_oracle.c into oracle/_build/liboracle.so (gcc, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("q1", ctypes.c_int32),
        ("split", ctypes.c_int32), ("interp_order", ctypes.c_int32),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("pc_tol", ctypes.c_double),
        ("pc_max_iter", ctypes.c_int32), ("pc_fixed_iters", ctypes.c_int32),
        ("grad_order", ctypes.c_int32),
        ("wall", (ctypes.c_double * 4) * 4),
        ("profile", ctypes.c_void_p * 4),
    ]


def make_config(nx, ny, lattice=16, split="total", interp_order=3, bc_x="periodic",
                bc_y="periodic", gamma=1.4, mu=1e-4, pc_tol=1e-12, pc_max_iter=20,
                pc_fixed_iters=0, grad_order=0, walls=None, profiles=None) -> Config:
    """split: "total", "internal" or "nt" (non-translational); grad_order: N = 3 or 4
    (0: the lattice's, 3 on D2Q16 and 4 on D2Q25).  Boundaries per axis: "periodic",
    "outflow", "wall" (both sides prescribed) or "inflow" (low side prescribed, high side
    outflow).  walls = four uniform states (u_x, u_y, T, rho) of the sides x-low, x-high,
    y-low, y-high; profiles = four arrays [n][4] of per-position states along the sides
    (n = ny for the x sides, nx for the y sides) or None each."""
    bc = {"periodic": 0, "outflow": 1, "wall": 2, "inflow": 3}
    w = ((ctypes.c_double * 4) * 4)()
    for k, state in enumerate(walls or [(0.0, 0.0, 1.0, 1.0)] * 4):
        for j in range(4):
            w[k][j] = float(state[j])
    prof = (ctypes.c_void_p * 4)()
    keep = []
    for k, arr in enumerate(profiles or [None] * 4):
        if arr is not None:
            arr = np.ascontiguousarray(arr, dtype=np.float64)
            if arr.shape != ((ny if k < 2 else nx), 4):
                raise ValueError("profile %d: shape %s" % (k, arr.shape))
            keep.append(arr)
            prof[k] = arr.ctypes.data
    cfg = Config(nx=nx, ny=ny, q1={16: 4, 25: 5}[lattice], wall=w, profile=prof,
                 split={"total": 0, "internal": 1, "nt": 2}[split], interp_order=interp_order,
                 bc_x=bc[bc_x], bc_y=bc[bc_y], gamma=gamma, mu=mu, pc_tol=pc_tol,
                 pc_max_iter=pc_max_iter, pc_fixed_iters=pc_fixed_iters, grad_order=grad_order)
    cfg._profiles = keep          # the C side reads the arrays through the pointers
    return cfg


_D = ctypes.POINTER(ctypes.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.or_lattice_1d.argtypes = [ctypes.c_int, _D, _D]
            lib.or_set_threads.argtypes = [ctypes.c_int]
            lib.or_set_threads.restype = ctypes.c_int
            lib.or_grad_transform.argtypes = [ctypes.c_int, _D] + [ctypes.c_double] * 6 + [_D]
            lib.or_grad_coefficients.argtypes = [ctypes.c_int, _D] + [ctypes.c_double] * 6 + [_D]
            lib.or_grad_transform_n.argtypes = [ctypes.c_int, ctypes.c_int, _D] + [ctypes.c_double] * 6 + [_D]
            lib.or_init.argtypes = [P(Config)] + [_D] * 8
            lib.or_moments_field.argtypes = [P(Config)] + [_D] * 10
            lib.or_stream_node.argtypes = ([P(Config)] + [_D] * 5 + [ctypes.c_int] * 2
                                           + [ctypes.c_double] * 3 + [_D] * 2)
            lib.or_stream_node_kept.argtypes = ([P(Config)] + [_D] * 5 + [ctypes.c_int] * 2
                                                + [ctypes.c_double] * 6 + [_D] * 2)
            lib.or_step.argtypes = ([P(Config)] + [_D] * 10
                                    + [P(ctypes.c_int32), P(ctypes.c_int64)])
            lib.or_collide_node.argtypes = [P(Config), _D, _D] + [ctypes.c_double] * 3 + [_D] * 3
            lib.or_step_nodes.argtypes = ([P(Config)] + [_D] * 5 + [ctypes.c_int]
                                          + [P(ctypes.c_int32)] * 2 + [_D] * 3 + [P(ctypes.c_int32)])
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's node loops (n > 0 sets them); returns the count in effect."""
    return _lib_handle().or_set_threads(n)


def lattice_1d(q1: int):
    c = np.zeros(q1)
    w = np.zeros(q1)
    _lib_handle().or_lattice_1d(q1, _p(c), _p(w))
    return c, w


def lattice_2d(lattice: int = 16):
    """(cx, cy, w) of the tensor-product lattice; population i = b*q1 + a."""
    q1 = {16: 4, 25: 5}[lattice]
    c, w = lattice_1d(q1)
    a = np.tile(np.arange(q1), q1)
    b = np.repeat(np.arange(q1), q1)
    return c[a], c[b], w[a] * w[b]


def grad_transform(pops, src_frame, dst_frame, lattice=16):
    q1 = {16: 4, 25: 5}[lattice]
    src = np.ascontiguousarray(pops, dtype=np.float64)
    out = np.zeros_like(src)
    _lib_handle().or_grad_transform(q1, _p(src), *map(float, src_frame), *map(float, dst_frame),
                                    _p(out))
    return out


def grad_transform_n(pops, src_frame, dst_frame, lattice=25, order=4):
    """The frame transformation with Grad order N = order (3 or 4)."""
    q1 = {16: 4, 25: 5}[lattice]
    src = np.ascontiguousarray(pops, dtype=np.float64)
    out = np.zeros_like(src)
    _lib_handle().or_grad_transform_n(q1, order, _p(src), *map(float, src_frame),
                                      *map(float, dst_frame), _p(out))
    return out


def grad_coefficients(pops, src_frame, dst_frame, lattice=16):
    """a0, a1 (2), a2 (2x2), a3 (2x2x2) of the populations in the target frame."""
    q1 = {16: 4, 25: 5}[lattice]
    src = np.ascontiguousarray(pops, dtype=np.float64)
    out = np.zeros(15)
    _lib_handle().or_grad_coefficients(q1, _p(src), *map(float, src_frame),
                                       *map(float, dst_frame), _p(out))
    return out[0], out[1:3].copy(), out[3:7].reshape(2, 2).copy(), out[7:15].reshape(2, 2, 2).copy()


class State:
    """Populations f, g (Q, ny, nx) in each node's own frame (ux, uy, T)."""

    def __init__(self, f, g, ux, uy, T):
        self.f, self.g, self.ux, self.uy, self.T = f, g, ux, uy, T

    def copy(self):
        return State(self.f.copy(), self.g.copy(), self.ux.copy(), self.uy.copy(), self.T.copy())


def init_state(cfg: Config, rho, ux, uy, T) -> State:
    ny, nx = cfg.ny, cfg.nx
    Q = cfg.q1 * cfg.q1
    arrs = [np.ascontiguousarray(np.broadcast_to(a, (ny, nx)), dtype=np.float64)
            for a in (rho, ux, uy, T)]
    f = np.zeros((Q, ny, nx))
    g = np.zeros((Q, ny, nx))
    fux, fuy, fT = (np.zeros((ny, nx)) for _ in range(3))
    _lib_handle().or_init(ctypes.byref(cfg), *map(_p, arrs), _p(f), _p(g), _p(fux), _p(fuy), _p(fT))
    return State(f, g, fux, fuy, fT)


def moments(cfg: Config, st: State):
    """rho, ux, uy, T, E of every node from its populations."""
    ny, nx = cfg.ny, cfg.nx
    out = [np.zeros((ny, nx)) for _ in range(5)]
    _lib_handle().or_moments_field(ctypes.byref(cfg), _p(st.f), _p(st.g), _p(st.ux), _p(st.uy),
                                   _p(st.T), *map(_p, out))
    return tuple(out)


def stream_node(cfg: Config, st: State, x: int, y: int, frame, stencil_frame=None):
    """Populations streamed to node (x, y) on the lattice of frame; the stencils are those the
    departure points of stencil_frame select (default: of frame itself)."""
    Q = cfg.q1 * cfg.q1
    P = np.zeros(Q)
    G = np.zeros(Q)
    if stencil_frame is None:
        _lib_handle().or_stream_node(ctypes.byref(cfg), _p(st.f), _p(st.g), _p(st.ux), _p(st.uy),
                                     _p(st.T), x, y, *map(float, frame), _p(P), _p(G))
    else:
        _lib_handle().or_stream_node_kept(ctypes.byref(cfg), _p(st.f), _p(st.g), _p(st.ux), _p(st.uy),
                                          _p(st.T), x, y, *map(float, frame), *map(float, stencil_frame),
                                          _p(P), _p(G))
    return P, G


def collide_node(cfg: Config, P, G, frame):
    """BGK collision of streamed populations P, G on the lattice of `frame`; returns
    (f*, g*, frame*) with frame* = (ux, uy, T) of their moments, or raises on a
    non-physical moment set."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    fo = np.zeros_like(P)
    go = np.zeros_like(G)
    fr = np.zeros(3)
    rc = _lib_handle().or_collide_node(ctypes.byref(cfg), _p(P), _p(G), *map(float, frame),
                                       _p(fo), _p(go), _p(fr))
    if rc != 0:
        raise ValueError("non-physical moments")
    return fo, go, fr


def step_nodes(cfg: Config, st: State, xs, ys):
    """One time step at the listed nodes only, from the full state st (the internal-split
    source pass, which needs every node's new frame, is not applied).  Returns
    (f [Q][count], g [Q][count], (ux, uy, T), iters)."""
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    count = len(xs)
    Q = cfg.q1 * cfg.q1
    fo = np.zeros((Q, count))
    go = np.zeros((Q, count))
    fr = np.zeros((3, count))
    it = np.zeros(count, dtype=np.int32)
    I32 = ctypes.POINTER(ctypes.c_int32)
    rc = _lib_handle().or_step_nodes(ctypes.byref(cfg), _p(st.f), _p(st.g), _p(st.ux), _p(st.uy),
                                     _p(st.T), count, xs.ctypes.data_as(I32), ys.ctypes.data_as(I32),
                                     _p(fo), _p(go), _p(fr), it.ctypes.data_as(I32))
    if rc == -1:
        raise ValueError("step_nodes: a node lies outside the %d x %d grid" % (cfg.nx, cfg.ny))
    return fo, go, (fr[0], fr[1], fr[2]), it


class StepResult:
    def __init__(self, state, status, iters, first_bad):
        self.state, self.status, self.iters, self.first_bad = state, status, iters, first_bad


def step(cfg: Config, st: State) -> StepResult:
    """One PonD time step n -> n+1 (returns a new state; the input is not modified)."""
    ny, nx = cfg.ny, cfg.nx
    Q = cfg.q1 * cfg.q1
    fo = np.zeros((Q, ny, nx))
    go = np.zeros((Q, ny, nx))
    oux, ouy, oT = (np.zeros((ny, nx)) for _ in range(3))
    iters = np.zeros((ny, nx), dtype=np.int32)
    bad = ctypes.c_int64(-1)
    rc = _lib_handle().or_step(ctypes.byref(cfg), _p(st.f), _p(st.g), _p(st.ux), _p(st.uy),
                               _p(st.T), _p(fo), _p(go), _p(oux), _p(ouy), _p(oT),
                               iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               ctypes.byref(bad))
    return StepResult(State(fo, go, oux, ouy, oT), rc, iters, bad.value)


def run(cfg: Config, st: State, nsteps: int):
    """Advance nsteps; returns (state, list of per-step status codes, total PC iterations)."""
    statuses = []
    total_iters = 0
    for _ in range(nsteps):
        r = step(cfg, st)
        st = r.state
        statuses.append(r.status)
        total_iters += int(r.iters.sum())
    return st, statuses, total_iters
