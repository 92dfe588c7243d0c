"""Launch-shape autotuning (pond_autotune): it times candidate tiles and halos on a copy of
the state, leaves the simulation's own state untouched, caches the choice per problem class,
and a tuned shape gives the same results as the default one (up to rounding: the tile's
centre node is the reference of the deviation arithmetic)."""
import numpy as np
import pytest

from paper_2405_11489_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pond():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_11489_gb300 import build, pond as P
    build.build()
    P.load_library()
    return P


def _sim(pond, case, precision, **kw):
    s = pond.Simulation(pond.Config(nx=case.nx, ny=case.ny, precision=precision, gamma=case.gamma,
                                    mu=case.mu, bc_x=case.bc_x, bc_y=case.bc_y, **kw))
    s.set_state(case.rho, case.ux, case.uy, case.T)
    return s


def test_autotune_picks_a_valid_shape_caches_it_and_keeps_the_state(pond):
    import torch
    pond.pond_autotune_clear()
    case = W.shear_wave(n=96, ny=80, ma=1.0, mu=0.05)
    s = _sim(pond, case, "fp32")
    s.step(2)
    mac0, neq0 = s.export_state()
    _, st0 = s.stats()
    t = s.autotune(steps=2, apply=True)
    assert t["candidates"] >= 5 and t["ms_per_step"] > 0
    assert t["tile_x"] * t["tile_y"] == 256 and t["tile_x"] % 2 == 0 and t["halo"] in (4, 5, 6, 8)
    assert s.launch() == {"tile_x": t["tile_x"], "tile_y": t["tile_y"], "halo": t["halo"]}
    mac1, neq1 = s.export_state()
    assert torch.equal(mac0, mac1) and torch.equal(neq0, neq1)
    _, st1 = s.stats()
    assert st1.steps == st0.steps and st1.pc_iters_total == st0.pc_iters_total
    s.step(2)                  # the trials' shapes left the kernel launchable for this one
    assert s.stats()[1].steps == st0.steps + 2
    # same class: served from the cache without timing
    s2 = _sim(pond, W.shear_wave(n=100, ny=70, ma=0.5, mu=0.05), "fp32")
    t2 = s2.autotune(steps=2, apply=True)
    assert t2["candidates"] == 0
    assert (t2["tile_x"], t2["tile_y"], t2["halo"]) == (t["tile_x"], t["tile_y"], t["halo"])
    t3 = s2.autotune(steps=1, apply=False, retime=True)
    assert t3["candidates"] >= 5
    s.close()
    s2.close()


def test_quasi_1d_grids_keep_the_row_tile(pond):
    pond.pond_autotune_clear()
    case = W.tube_batch(count=1, seed=3, nmin=600, nmax=600)[0]
    s = _sim(pond, case, "fp32", interp_order=2)
    t = s.autotune(steps=2)
    assert (t["tile_x"], t["tile_y"]) == (128, 1) and t["candidates"] >= 1
    s.close()


def test_autotune_times_states_whose_nodes_do_not_converge(pond):
    pond.pond_autotune_clear()
    case = W.riemann2d(n=64, seed=0)
    s = _sim(pond, case, "fp32", interp_order=2, pc_max_iter=1)
    s.step(1)
    assert s.stats()[0] == pond.POND_ENOCONV
    t = s.autotune(steps=1)
    assert t["candidates"] >= 5
    s.close()


def test_quasi_1d_grids_take_only_the_row_tile(pond):
    case = W.tube_batch(count=1, seed=3, nmin=500, nmax=500)[0]
    s = _sim(pond, case, "fp32")
    s.set_launch(128, 1, 6)
    assert s.launch() == {"tile_x": 128, "tile_y": 1, "halo": 6}
    for shape in ((256, 1, 5), (64, 2, 5)):
        with pytest.raises(pond.PondError):
            s.set_launch(*shape)
    assert s.launch() == {"tile_x": 128, "tile_y": 1, "halo": 6}
    s.step(3)
    assert s.stats()[1].steps == 3
    s.close()


# shapes whose staged box fits shared memory (FP64 records are twice as large)
SHAPES = [("fp64", 1e-12, (16, 16, 4)), ("fp64", 1e-12, (64, 4, 5)), ("fp64", 1e-12, (8, 32, 5)),
          ("fp32", 2e-6, (16, 16, 4)), ("fp32", 2e-6, (64, 4, 8)), ("fp32", 2e-6, (128, 2, 5)),
          ("fp32", 2e-6, (8, 32, 5))]


@pytest.mark.parametrize("precision,tol,shape", SHAPES)
def test_every_shape_gives_the_default_shapes_result(pond, precision, tol, shape):
    case = W.thermal_pulse(n=72, amp=1e-2, width=5.0, mu=0.05, ma=0.8)
    a = _sim(pond, case, precision, pc_fixed_iters=3)
    b = _sim(pond, case, precision, pc_fixed_iters=3)
    b.set_launch(*shape)
    assert b.launch() == {"tile_x": shape[0], "tile_y": shape[1], "halo": shape[2]}
    a.step(6)
    b.step(6)
    for x, y, scale in zip(a.moments(), b.moments(), (1.0, 1.0, 1.0, 1.0)):
        assert np.max(np.abs(x - y)) <= tol * max(np.max(np.abs(x)), scale)
    _, sa = a.stats()
    _, sb = b.stats()
    assert sa.halo_fallbacks == 0 and sb.halo_fallbacks == 0
    a.close()
    b.close()


# (FP32 128 x 2 with halo 6: the box's records and the y-weight table exceed the shared memory
# of a block, as the FP64 boxes below do with their 8-byte records)
@pytest.mark.parametrize("precision,shape", [("fp32", (30, 8, 5)), ("fp32", (32, 4, 5)),
                                             ("fp32", (16, 16, 65)), ("fp32", (7, 0, 5)),
                                             ("fp32", (128, 2, 6)), ("fp64", (128, 2, 6)),
                                             ("fp64", (64, 4, 8))])
def test_invalid_shapes_are_rejected(pond, precision, shape):
    case = W.shear_wave(n=40, ny=24, ma=0.5, mu=0.05)
    s = _sim(pond, case, precision)
    with pytest.raises(pond.PondError):
        s.set_launch(*shape)
    assert s.launch() == {"tile_x": 32, "tile_y": 8, "halo": 5}
    s.close()
