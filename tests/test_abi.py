"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/pond.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pond.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2405_11489_gb300 import build, pond
    build.build()
    return pond.load_library()


def _declared():
    text = open(HEADER).read()
    decl = r"^\s*(?:int|void|const\s+char\s*\*)\s*(pond_[a-z_]+)\s*\("
    return sorted(set(re.findall(decl, text, flags=re.MULTILINE)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pond_create", "pond_set_state", "pond_step", "pond_get_moments", "pond_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2405_11489_gb300 import pond
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(pond.EXPORTS)


def test_host_side_calls_without_gpu(lib):
    from paper_2405_11489_gb300 import pond
    cfg = pond.pond_config_default(64, 32)
    assert cfg.lattice == 16 and cfg.precision == pond.POND_MIXED_FP32
    n16 = pond.pond_workspace_bytes(cfg)
    # two states of 4 FP64 frame planes + 19 FP32 coefficient planes, plus a status block
    assert n16 >= 2 * 64 * 32 * (4 * 8 + 19 * 4)
    cfg.precision = pond.POND_FP64
    assert pond.pond_workspace_bytes(cfg) > n16
    assert lib.pond_version().decode().startswith("libpond")
    assert "non-physical" in lib.pond_strerror(-4).decode()


@pytest.mark.parametrize("field,value", [("nx", 0), ("lattice", 9), ("gamma", 2.5), ("gamma", 1.0),
                                         ("mu", 0.0), ("interp_order", 5), ("pc_max_iter", 0),
                                         ("bc_x", 7), ("precision", 9), ("tile_x", 48), ("split", 3),
                                         ("grad_order", 4), ("grad_order", 2)])
def test_invalid_configs_are_rejected(lib, field, value):
    from paper_2405_11489_gb300 import pond
    cfg = pond.pond_config_default(16, 16)
    setattr(cfg, field, value)
    n = ctypes.c_size_t(0)
    assert lib.pond_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)) == pond.POND_EINVAL
    h = ctypes.c_void_p(0)
    assert lib.pond_create(ctypes.byref(cfg), ctypes.c_void_p(256), 1 << 20, None, ctypes.byref(h)) == pond.POND_EINVAL


@pytest.mark.parametrize("ny,tile,ok", [(1, (128, 1), True), (1, (256, 1), False), (1, (64, 2), False),
                                         (16, (32, 8), True), (16, (128, 2), True), (16, (128, 1), False)])
def test_tiles_hold_the_kernels_threads(lib, ny, tile, ok):
    """A tile holds one CTA's threads: 256 nodes on 2-D grids, 128 x 1 on quasi-1-D ones."""
    from paper_2405_11489_gb300 import pond
    cfg = pond.pond_config_default(400, ny)
    cfg.tile_x, cfg.tile_y = tile
    n = ctypes.c_size_t(0)
    rc = lib.pond_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n))
    assert rc == (pond.POND_OK if ok else pond.POND_EINVAL)


def test_null_handles_are_rejected(lib):
    from paper_2405_11489_gb300 import pond
    assert lib.pond_step(None, 1) == pond.POND_EINVAL
    assert lib.pond_sync(None) == pond.POND_EINVAL
    assert lib.pond_destroy(None) == pond.POND_EINVAL


def test_prescribed_sides_are_validated_and_sized(lib):
    from paper_2405_11489_gb300 import pond
    n = ctypes.c_size_t(0)
    base = pond.pond_config_default(40, 24)
    b0 = pond.pond_workspace_bytes(base)
    # inflow on x: the x-low side is prescribed and carries a profile of ny states
    cfg = pond.pond_config_default(40, 24)
    cfg.bc_x = pond.POND_BC_INFLOW
    cfg.wall[0][2], cfg.wall[0][3] = 1.0, 1.0
    assert pond.pond_workspace_bytes(cfg) >= b0 + 24 * 4 * 8
    cfg.wall[0][2] = 0.0                                  # T <= 0 on a prescribed side
    assert lib.pond_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)) == pond.POND_EINVAL
    cfg.wall[0][2] = 1.0
    cfg.wall[1][2] = 0.0                                  # x-high is outflow: not checked
    assert lib.pond_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)) == pond.POND_OK
    # no prescribed y sides on quasi-1-D grids
    cfg1 = pond.pond_config_default(40, 1)
    cfg1.bc_y = pond.POND_BC_INFLOW
    assert lib.pond_workspace_bytes(ctypes.byref(cfg1), ctypes.byref(n)) == pond.POND_EINVAL
    cfg1.bc_y = 4
    assert lib.pond_workspace_bytes(ctypes.byref(cfg1), ctypes.byref(n)) == pond.POND_EINVAL
    assert lib.pond_set_boundary_profile(None, 0, None, 0) == pond.POND_EINVAL
