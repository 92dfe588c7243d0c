"""Mixed precision against the FP64 oracle, and sampled parity at the full configuration
sizes.

Mixed modes compute in FP32 on deviations from a per-tile reference equilibrium, with rho,
u, T in FP64 and the non-equilibrium Hermite coefficients stored in FP32, FP16 or BF16.
Stated bounds (per-field relative L1 error against the oracle, fixed-K mode):

  FP32 storage:  rho, T <= 5e-8 relative; u <= 1e-7 of the velocity scale
  FP16 storage:  rho, T <= 2e-6;          u <= 2e-5
  BF16 storage:  rho, T <= 2e-5;          u <= 2e-4

The rounding acts on deviations from the tile's reference node, so it grows with the
contrast inside a tile.  For a jet of Mach 1.5 over a Mach 0.3 co-flow (velocity
deviations of 1.2 sound speeds instead of a few per cent) the bounds are four times the
ones above (FP32 2e-7, BF16 8e-5 for every field); at the jet's full configuration, where a
tile can straddle the jet (rho, T) = (5, 0.005) and the ambient (50, 0.0005), a contrast of
10 in both rho and T scales the rounding relative to a node's own values by up to 100
(2e-5): sampled moments within 3e-5 relative, populations within 1e-4 of their scale
(measured: T 4.3e-6 to 1.07e-5, populations up to 2.0e-5, over two builds of the kernel).

Full sizes (256 x 256 decay configuration, 1024 x 1024 four-quadrant Riemann problem with the
3-point interpolation of Sec. III.A.2, in the launch configuration the benchmark uses): after a few GPU steps the state is exported as
FP64 populations, the GPU takes one more step and the oracle computes that step node by
node at sampled nodes (corners, edges, the quadrant interfaces, random nodes).
"""
import math

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


def _l1(a, b, scale):
    return float(np.mean(np.abs(a - b)) / scale)


BOUNDS = {"fp32": (5e-8, 1e-7), "fp16": (2e-6, 2e-5), "bf16": (2e-5, 2e-4)}


# Errors relative to the physical signal of the 256^2 decay configuration after 200 steps
# (mean |mixed - FP64| over the mean |FP64 - its own mean|): the shear wave's u_y and the
# thermal pulse's T and rho.  Measured on one GB300: u_y 4.7e-7 / 1.9e-6 / 2.0e-5, T 1.9e-5 /
# 7.0e-4 / 5.1e-3, rho 2.9e-5 / 7.4e-4 / 5.5e-3 (FP32 / FP16 / BF16 storage).  The pulse
# also induces a second-order u_x perturbation that the reduced storages do not resolve
# (error 1.3 times that perturbation with BF16, 0.19 with FP16, 0.011 with FP32 storage);
# it is not bounded here.
SIGNAL_BOUNDS = {"fp32": {"uy": 2e-6, "T": 1e-4, "rho": 1e-4},
                 "fp16": {"uy": 1e-5, "T": 3e-3, "rho": 3e-3},
                 "bf16": {"uy": 1e-4, "T": 2e-2, "rho": 2e-2}}


def test_reduced_storage_errors_against_the_signal(pond):
    """The decay configuration's perturbations (shear wave u_y, thermal pulse T and rho) in
    the mixed modes stay within stated bounds relative to their own size, against the FP64
    path, after 200 steps."""
    sh = W.shear_wave(n=256, ma=1.0, amp=0.05, mu=0.05)
    pu = W.thermal_pulse(n=256, amp=1e-3, width=16.0, mu=0.05, ma=1.0)
    res = {}
    for prec in ("fp64", "fp32", "fp16", "bf16"):
        s = pond.Simulation(pond.Config(nx=256, ny=256, precision=prec, gamma=1.4, mu=0.05))
        s.set_state(pu.rho, sh.ux, sh.uy, pu.T)
        s.step(200)
        res[prec] = dict(zip(("rho", "ux", "uy", "T"), s.moments()))
        s.close()
    ref = res["fp64"]
    for prec in ("fp32", "fp16", "bf16"):
        errs = {}
        for k in ("uy", "T", "rho"):
            signal = np.mean(np.abs(ref[k] - ref[k].mean()))
            errs[k] = float(np.mean(np.abs(res[prec][k] - ref[k])) / signal)
        print(prec, errs)
        assert all(errs[k] <= SIGNAL_BOUNDS[prec][k] for k in errs), (prec, errs)


MIXED_CASES = [(prec, 16, split) for prec in ("fp32", "fp16", "bf16")
               for split in ("total", "internal", "nt")] + \
              [("fp32", 25, "total"), ("fp32", 25, "nt"), ("bf16", 25, "nt")]


@pytest.mark.parametrize("precision,lattice,split", MIXED_CASES)
def test_mixed_precision_l1_bounds(pond, orc, precision, lattice, split):
    nx, ny, steps = 48, 40, 20
    y, x = np.mgrid[0:ny, 0:nx]
    rho = 1.0 + 0.02 * np.sin(2 * math.pi * x / nx) * np.cos(2 * math.pi * y / ny)
    ux = 0.6 + 0.03 * np.cos(2 * math.pi * y / ny)
    uy = -0.2 + 0.03 * np.sin(2 * math.pi * x / nx)
    T = 0.8 * (1.0 + 0.02 * np.cos(2 * math.pi * (x / nx + y / ny)))
    ocfg = orc.make_config(nx, ny, lattice=lattice, split=split, mu=0.04, pc_fixed_iters=2)
    st = orc.init_state(ocfg, rho, ux, uy, T)
    for _ in range(steps):
        st = orc.step(ocfg, st).state
    o = orc.moments(ocfg, st)
    sim = pond.Simulation(pond.Config(nx=nx, ny=ny, lattice=lattice, precision=precision, split=split,
                                      mu=0.04, pc_fixed_iters=2))
    sim.set_state(rho, ux, uy, T)
    sim.step(steps)
    g = sim.moments()
    brt, bu = BOUNDS[precision]
    speed = max(np.abs(o[1]).max(), np.abs(o[2]).max(), math.sqrt(o[3].max()))
    errs = {"rho": _l1(g[0], o[0], np.mean(np.abs(o[0]))), "T": _l1(g[3], o[3], np.mean(o[3])),
            "ux": _l1(g[1], o[1], speed), "uy": _l1(g[2], o[2], speed)}
    print(precision, lattice, split, errs)
    assert errs["rho"] <= brt and errs["T"] <= brt, errs
    assert errs["ux"] <= bu and errs["uy"] <= bu, errs
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_mixed_precision_jet_inflow_l1_bounds(pond, orc, precision):
    """A jet entering through a profiled inlet (x-low inflow, tanh jet of Ma 1.5 over a
    Ma 0.3 co-flow at equal pressure), outflow elsewhere, in the mixed modes: the stated
    bounds hold."""
    nx, ny, steps, gamma = 48, 40, 20, 1.4
    yc = np.arange(ny) - (ny - 1) / 2.0
    jet = 0.5 * (1.0 - np.tanh((np.abs(yc) - 6.0) / 2.0))
    T_in = 0.8 * (1.0 + 0.1 * jet)
    prof = np.stack([(0.3 + 1.2 * jet) * np.sqrt(gamma * T_in), np.zeros(ny), T_in, 0.8 / T_in], 1)
    walls = [tuple(prof[0])] * 4
    rho = np.full((ny, nx), 1.0)
    ux = np.full((ny, nx), 0.3 * math.sqrt(gamma * 0.8))
    uy = np.zeros((ny, nx))
    T = np.full((ny, nx), 0.8)
    ocfg = orc.make_config(nx, ny, bc_x="inflow", bc_y="outflow", mu=0.04, pc_fixed_iters=2,
                           walls=walls, profiles=[prof, None, None, None])
    st = orc.init_state(ocfg, rho, ux, uy, T)
    for _ in range(steps):
        st = orc.step(ocfg, st).state
    o = orc.moments(ocfg, st)
    sim = pond.Simulation(pond.Config(nx=nx, ny=ny, precision=precision, bc_x="inflow",
                                      bc_y="outflow", mu=0.04, pc_fixed_iters=2, walls=tuple(walls)))
    sim.set_boundary_profile("x_low", prof)
    sim.set_state(rho, ux, uy, T)
    sim.step(steps)
    g = sim.moments()
    brt = bu = {"fp32": 2e-7, "bf16": 8e-5}[precision]     # four times the small-amplitude bounds
    speed = max(np.abs(o[1]).max(), np.abs(o[2]).max(), math.sqrt(o[3].max()))
    errs = {"rho": _l1(g[0], o[0], np.mean(np.abs(o[0]))), "T": _l1(g[3], o[3], np.mean(o[3])),
            "ux": _l1(g[1], o[1], speed), "uy": _l1(g[2], o[2], speed)}
    print(precision, "jet", errs)
    assert errs["rho"] <= brt and errs["T"] <= brt, errs
    assert errs["ux"] <= bu and errs["uy"] <= bu, errs
    # the jet has entered: the centre row is faster than the co-flow
    assert g[1][ny // 2, nx // 4] > 1.5 * g[1][2, nx // 4]
    sim.close()


def _sample_nodes(nx, ny, rng, n_random=48):
    pts = {(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (nx // 2, ny // 2),
           (nx // 2 - 1, ny // 2 - 1), (nx // 2, 0), (0, ny // 2), (nx - 1, ny // 2 + 1)}
    for _ in range(n_random):
        pts.add((int(rng.integers(nx)), int(rng.integers(ny))))
    pts = sorted({(min(max(x, 0), nx - 1), min(max(y, 0), ny - 1)) for x, y in pts})   # one-row grids
    return np.array([p[0] for p in pts]), np.array([p[1] for p in pts])


def _sampled_step(pond, orc, case, precision, split, warm, tol_m, tol_f, seed, order=3):
    walls = case.meta.get("walls")
    prof = case.meta.get("profile")
    cfg = pond.Config(nx=case.nx, ny=case.ny, precision=precision, split=split, gamma=case.gamma,
                      mu=case.mu, bc_x=case.bc_x, bc_y=case.bc_y, interp_order=order,
                      walls=tuple(walls) if walls else None)
    sim = pond.Simulation(cfg)
    if prof is not None:
        sim.set_boundary_profile("x_low", prof)
    sim.set_state(case.rho, case.ux, case.uy, case.T)
    sim.step(warm)
    f, g, fux, fuy, fT = sim.populations()
    sim.step(1)
    gf, gg, gux, guy, gT = sim.populations()
    ocfg = orc.make_config(case.nx, case.ny, split=split, gamma=case.gamma, mu=case.mu,
                           bc_x=case.bc_x, bc_y=case.bc_y, pc_tol=1e-13, pc_max_iter=40,
                           interp_order=order, walls=walls,
                           profiles=[prof, None, None, None] if prof is not None else None)
    st = orc.State(f, g, fux, fuy, fT)
    xs, ys = _sample_nodes(case.nx, case.ny, np.random.default_rng(seed))
    of, og, (oux, ouy, oT), _ = orc.step_nodes(ocfg, st, xs, ys)
    speed = max(np.abs(oux).max(), np.abs(ouy).max(), math.sqrt(oT.max()))
    errs = {"T": np.max(np.abs(gT[ys, xs] - oT) / oT),
            "ux": np.max(np.abs(gux[ys, xs] - oux)) / speed,
            "uy": np.max(np.abs(guy[ys, xs] - ouy)) / speed,
            "f": np.max(np.abs(gf[:, ys, xs] - of)) / np.max(np.abs(of))}
    if split == "total":
        errs["g"] = np.max(np.abs(gg[:, ys, xs] - og)) / np.max(np.abs(og))
    sim.close()
    print("sampled %s %s %s" % (case.name if hasattr(case, "name") else "", precision, errs))
    bad = {k: v for k, v in errs.items() if not v <= (tol_f if k in ("f", "g") else tol_m)}
    assert not bad, errs


@pytest.mark.parametrize("precision,tol_m,tol_f", [("fp32", 2e-6, 2e-5), ("fp64", 1e-9, 1e-8)])
def test_decay_256_sampled_parity(pond, orc, precision, tol_m, tol_f):
    rho = W.thermal_pulse(n=256, amp=1e-3, width=16.0, mu=0.05, ma=1.0).rho
    sh = W.shear_wave(n=256, ma=1.0, amp=0.05, mu=0.05)
    case = W.Case("decay", rho, sh.ux, sh.uy, 1.0 / rho, mu=0.05)
    _sampled_step(pond, orc, case, precision, "total", 3, tol_m, tol_f, seed=1)


@pytest.mark.parametrize("split", ["total", "internal"])
def test_riemann_1024_sampled_parity(pond, orc, split):
    case = W.riemann2d(n=1024, seed=0)
    _sampled_step(pond, orc, case, "fp32", split, 4, 5e-6, 5e-5, seed=2, order=2)


@pytest.mark.parametrize("split", ["total", "internal"])
def test_riemann_1024_runs_500_steps_physical(pond, split):
    """The four-quadrant configuration (1024^2, 500 steps, mixed FP32) stays physical."""
    case = W.riemann2d(n=1024, seed=0)
    sim = pond.Simulation(pond.Config(nx=case.nx, ny=case.ny, precision="fp32", split=split,
                                      gamma=case.gamma, mu=case.mu, bc_x=case.bc_x, bc_y=case.bc_y,
                                      interp_order=2))
    sim.set_state(case.rho, case.ux, case.uy, case.T)
    sim.step(case.steps)
    rc, st = sim.stats()
    assert rc in (pond.POND_OK, pond.POND_ENOCONV) and st.first_bad_node == -1
    rho, ux, uy, T = sim.moments()
    assert np.all(rho > 0) and np.all(T > 0) and np.all(np.isfinite(ux))
    sim.close()


def test_tube_batch_runs_physical(pond):
    """The 256 uneven tubes (N ~ logU[200, 4000]) advanced together for 600 steps."""
    cases = W.tube_batch(count=256, seed=1)
    sims = []
    for c in cases:
        s = pond.Simulation(pond.Config(nx=c.nx, ny=c.ny, precision="fp32", gamma=c.gamma, mu=c.mu,
                                        bc_x=c.bc_x, bc_y=c.bc_y, interp_order=2))
        s.set_state(c.rho, c.ux, c.uy, c.T)
        sims.append(s)
    batch = pond.Batch(sims)
    batch.step(600)
    for s in sims:
        rc, st = s.stats()
        assert rc in (pond.POND_OK, pond.POND_ENOCONV) and st.first_bad_node == -1, pond.strerror(rc)
    batch.close()


def test_tube_batch_256_sampled_parity(pond, orc):
    """The 256 uneven tubes advanced in one batched launch per step, in the benchmark's launch
    configuration (3-point stencil, FP32, halo tuned on the longest tube, convergence mode):
    after 20 batched steps, one more batched step of four members (the shortest, the longest
    and two drawn) is checked node by node against the oracle at every sampled node where the
    oracle's predictor-corrector converges (to 1e-13) within the GPU's iteration cap.  At the
    shocks, which fill much of a short tube, some nodes do not converge; there the iterate at
    the cap is not a result that two precisions share, and those nodes are counted instead
    (at most a fifth of the sample)."""
    cases = W.tube_batch(count=256, seed=1)
    sims = []
    for c in cases:
        s = pond.Simulation(pond.Config(nx=c.nx, ny=c.ny, precision="fp32", gamma=c.gamma, mu=c.mu,
                                        bc_x=c.bc_x, bc_y=c.bc_y, interp_order=2))
        s.set_state(c.rho, c.ux, c.uy, c.T)
        sims.append(s)
    big = max(range(len(cases)), key=lambda i: cases[i].nx)
    halo = sims[big].autotune(steps=2, apply=True)["halo"]
    for s in sims:
        s.set_launch(0, 0, halo)
    batch = pond.Batch(sims)
    batch.step(20)
    rng = np.random.default_rng(5)
    pick = [min(range(len(cases)), key=lambda i: cases[i].nx), big] + [int(v) for v in rng.integers(len(cases), size=2)]
    before = {i: sims[i].populations() for i in pick}
    batch.step(1)
    for i in pick:
        c = cases[i]
        gf, gg, gux, guy, gT = sims[i].populations()
        ocfg = orc.make_config(c.nx, c.ny, gamma=c.gamma, mu=c.mu, bc_x=c.bc_x, bc_y=c.bc_y,
                               pc_tol=1e-13, pc_max_iter=40, interp_order=2)
        xs, ys = _sample_nodes(c.nx, c.ny, rng)
        of, og, (oux, ouy, oT), oit = orc.step_nodes(ocfg, orc.State(*before[i]), xs, ys)
        ok = oit < 20                                   # converged within the GPU's cap
        print("tube %d (%d cells): %d of %d sampled nodes converge within the cap" % (i, c.nx, int(ok.sum()), len(xs)))
        # with the stencils carried between iterations every sampled node converges (measured:
        # 192 of 192 over the four tubes); before, up to a fifth of them cycled at the shocks
        assert ok.all(), (i, c.nx, int(ok.sum()), len(xs))
        xs, ys, of, og, oux, oT = xs[ok], ys[ok], of[:, ok], og[:, ok], oux[ok], oT[ok]
        speed = max(np.abs(oux).max(), math.sqrt(oT.max()))
        errs = {"T": np.max(np.abs(gT[ys, xs] - oT) / oT), "ux": np.max(np.abs(gux[ys, xs] - oux)) / speed,
                "f": np.max(np.abs(gf[:, ys, xs] - of)) / np.max(np.abs(of)),
                "g": np.max(np.abs(gg[:, ys, xs] - og)) / np.max(np.abs(og))}
        print("tube %d errors %s" % (i, errs))
        assert errs["T"] <= 5e-6 and errs["ux"] <= 5e-6 and errs["f"] <= 5e-5 and errs["g"] <= 5e-5, (i, c.nx, errs)
    batch.close()
    for s in sims:
        s.close()


def test_sod_400x4_fp32_matches_exact_riemann(pond):
    from oracle.riemann import RiemannSolution
    c = W.sod(nx=400, ny=4)
    sim = pond.Simulation(pond.Config(nx=c.nx, ny=c.ny, precision="fp32", gamma=c.gamma, mu=c.mu,
                                      bc_x=c.bc_x, bc_y=c.bc_y))
    sim.set_state(c.rho, c.ux, c.uy, c.T)
    sim.step(c.steps)
    rho, ux, uy, T = sim.moments()
    sol = RiemannSolution((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    t = c.steps * 0.2 / c.nx
    re, ue, pe = sol.sample((np.arange(c.nx) - c.meta["x0"] + 0.5) / c.nx / t)
    for row in range(c.ny):
        assert np.mean(np.abs(rho[row] - re)) < 4e-3
        assert np.mean(np.abs(rho[row] * T[row] / 0.04 - pe)) < 4e-3
    sim.close()


def test_jet_2000x1000_sampled_parity(pond, orc):
    """The jet configuration of Sec. III.C at its resolution (2000 x 1000, D = 100, the paper's
    jet and ambient states, profiled x-low inflow) at Mach 1.5, in mixed FP32."""
    case = W.jet(ma=1.5)
    # the FP32 rounding, scaled by the contrast inside a tile (10 in rho and in T: up to 100 times
    # the co-flow jet's 2e-7), bounds the moments by 2e-5; 3e-5 and 1e-4 here.  Measured on one
    # GB300 with two builds of the same arithmetic (differing only in the compiler's
    # scheduling and contraction): T 4.3e-6 / 1.07e-5, f 5.0e-6 / 5.2e-6, g 6.4e-6 / 2.0e-5
    _sampled_step(pond, orc, case, "fp32", "total", 3, 3e-5, 1e-4, seed=4)


# Moments handed to the caller from populations far from their frame's equilibrium: the
# mixed modes form the stored coefficients' contribution in FP32 and add it to the FP64
# frame (the moment definitions of Sec. II rearranged relative to the frame), so the
# corrections u - u_frame and T - T_frame are large here (5 % non-equilibrium parts).  On
# these fields a wrong sign on a term of a rearrangement gives errors from 6e-4 (the |d|^2
# term) to 3e-2 (u_frame . d, the A_20 + A_02 term), above the FP32 and FP16 bounds; the
# bounds are the storage rounding of the coefficients.
@pytest.mark.parametrize("split,lattice", [("total", 16), ("internal", 16), ("nt", 16), ("nt", 25),
                                           ("total", 25)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6), ("fp16", 3e-4),
                                           ("bf16", 3e-3)])
def test_moments_of_non_equilibrium_populations(pond, orc, split, lattice, precision, tol):
    nx, ny = 23, 9
    rng = np.random.default_rng(lattice + len(split))
    ocfg = orc.make_config(nx, ny, lattice=lattice, split=split, gamma=1.4, mu=0.02)
    y, x = np.mgrid[0:ny, 0:nx]
    rho = 1.0 + 0.1 * np.sin(2 * np.pi * x / nx) + 0.02 * rng.standard_normal((ny, nx))
    ux = 0.9 + 0.2 * np.cos(2 * np.pi * y / ny)
    uy = -0.4 + 0.1 * np.sin(2 * np.pi * (x + y) / nx)
    T = 0.7 * (1 + 0.1 * np.cos(2 * np.pi * x / nx))
    st = orc.init_state(ocfg, rho, ux, uy, T)
    Q = ocfg.q1 * ocfg.q1
    st.f = st.f * (1 + 0.05 * rng.standard_normal((Q, ny, nx)))
    st.g = st.g * (1 + 0.05 * rng.standard_normal((Q, ny, nx)))
    o_rho, o_ux, o_uy, o_T, _ = orc.moments(ocfg, st)
    assert np.max(np.abs(o_ux - st.ux)) > 1e-3
    # the internal split reports the frame's temperature (its g carries U + sum G / 2); the
    # others recover T from the perturbed populations
    if split == "internal":
        assert np.array_equal(o_T, st.T)
    else:
        assert np.max(np.abs(o_T - st.T)) > 1e-3
    sim = pond.Simulation(pond.Config(nx=nx, ny=ny, lattice=lattice, split=split, precision=precision,
                                      gamma=1.4, mu=0.02))
    sim.set_populations(st.f, st.g, st.ux, st.uy, st.T)
    g_rho, g_ux, g_uy, g_T = sim.moments(allow=(pond.POND_OK,))
    speed = max(np.max(np.abs(o_ux)), np.max(np.abs(o_uy)), np.sqrt(np.max(o_T)))
    assert np.max(np.abs(g_rho - o_rho)) <= tol * np.max(o_rho)
    assert np.max(np.abs(g_ux - o_ux)) <= tol * speed
    assert np.max(np.abs(g_uy - o_uy)) <= tol * speed
    assert np.max(np.abs(g_T - o_T)) <= tol * np.max(o_T)
    sim.close()
