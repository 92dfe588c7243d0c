"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

FP64 mode in fixed-iteration predictor-corrector mode must match the oracle to a relative
L-infinity error of 1e-12 per field (rel = max|gpu - oracle| / max|oracle|), on grids that
span several tiles and leave ragged tails, with every boundary type (periodic, outflow,
walls, inflow, per-position side profiles), both lattices, the three energy splits, both
interpolation orders, the shared-memory and the global-gather (halo fallback) paths and
degenerate grid shapes.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def pond():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_11489_gb300 import build, pond as P
    build.build()
    P.load_library()
    return P


def rel_linf(a, b):
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0))


def random_state(orc, ocfg, seed, amp=0.05, ux0=0.3, uy0=-0.2, T0=0.8, neq=0.01):
    """Smooth random fields plus a random non-equilibrium part in each node's own frame."""
    rng = np.random.default_rng(seed)
    ny, nx = ocfg.ny, ocfg.nx
    y, x = np.mgrid[0:ny, 0:nx]
    def smooth(phase):
        return (np.sin(2 * math.pi * (x / max(nx, 1) + phase[0])) *
                np.cos(2 * math.pi * (y / max(ny, 1) + phase[1])))
    rho = 1.0 + amp * smooth(rng.uniform(0, 1, 2)) + 0.2 * amp * rng.standard_normal((ny, nx))
    ux = ux0 + amp * smooth(rng.uniform(0, 1, 2))
    uy = uy0 + amp * smooth(rng.uniform(0, 1, 2))
    T = T0 * (1 + amp * smooth(rng.uniform(0, 1, 2)))
    st = orc.init_state(ocfg, rho, ux, uy, T)
    Q = ocfg.q1 * ocfg.q1
    st.f = st.f * (1 + neq * rng.standard_normal((Q, ny, nx)))
    st.g = st.g * (1 + neq * rng.standard_normal((Q, ny, nx)))
    return st


# wall states (u_x, u_y, T, rho) for x-low, x-high, y-low, y-high, used where a bc is "wall"
WALLS = [(0.2, 0.05, 0.75, 1.0), (0.45, -0.1, 0.9, 1.1), (0.3, 0.0, 0.85, 0.95), (-0.2, 0.0, 0.7, 1.05)]


def make_pair(pond, orc, nx, ny, lattice=16, split="total", order=3, bc=("periodic", "periodic"),
              K=2, tol=1e-12, precision="fp64", halo=0, gamma=1.4, mu=0.02, maxit=20):
    ocfg = orc.make_config(nx, ny, lattice=lattice, split=split, interp_order=order, bc_x=bc[0],
                           bc_y=bc[1], gamma=gamma, mu=mu, pc_tol=tol, pc_max_iter=maxit,
                           pc_fixed_iters=K, walls=WALLS)
    gcfg = pond.Config(nx=nx, ny=ny, lattice=lattice, split=split, precision=precision,
                       interp_order=order, bc_x=bc[0], bc_y=bc[1], gamma=gamma, mu=mu, pc_tol=tol,
                       pc_max_iter=maxit, pc_fixed_iters=K, halo=halo, walls=tuple(WALLS))
    return ocfg, pond.Simulation(gcfg)


def vel_err(a, b, speed):
    """Velocity components are compared on the flow's velocity scale (a component that is
    zero in exact arithmetic has no relative error of its own)."""
    return float(np.max(np.abs(a - b)) / speed)


def compare(orc, ocfg, sim, st, tol, what=""):
    rho, ux, uy, T, E = orc.moments(ocfg, st)
    g_rho, g_ux, g_uy, g_T = sim.moments()
    speed = max(np.max(np.abs(ux)), np.max(np.abs(uy)), np.sqrt(np.max(T)))
    errs = {"rho": rel_linf(g_rho, rho), "ux": vel_err(g_ux, ux, speed),
            "uy": vel_err(g_uy, uy, speed), "T": rel_linf(g_T, T)}
    f, g, fux, fuy, fT = sim.populations()
    errs["f"] = rel_linf(f, st.f)
    errs["g"] = rel_linf(g, st.g)
    errs["frame"] = max(vel_err(fux, st.ux, speed), vel_err(fuy, st.uy, speed), rel_linf(fT, st.T))
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, "%s: %s" % (what, errs)
    return errs


def run_both(orc, ocfg, sim, st, nsteps):
    sim.set_populations(st.f, st.g, st.ux, st.uy, st.T)
    for _ in range(nsteps):
        st = orc.step(ocfg, st).state
    sim.step(nsteps)
    return st


CASES = [
    # nx, ny, lattice, split, order, bcs
    (37, 11, 16, "total", 3, ("periodic", "periodic")),
    (45, 9, 16, "total", 3, ("outflow", "outflow")),
    (33, 6, 16, "internal", 3, ("periodic", "outflow")),
    (29, 10, 25, "total", 3, ("periodic", "periodic")),
    (26, 7, 25, "internal", 3, ("outflow", "periodic")),
    (31, 9, 16, "total", 2, ("periodic", "periodic")),
    (27, 8, 25, "nt", 3, ("periodic", "periodic")),
    (30, 7, 16, "nt", 3, ("outflow", "periodic")),
    (25, 9, 25, "nt", 2, ("outflow", "outflow")),
    (28, 10, 16, "total", 3, ("periodic", "wall")),
    (24, 11, 25, "nt", 3, ("wall", "wall")),
    (30, 8, 16, "internal", 3, ("wall", "outflow")),
    (33, 9, 16, "total", 3, ("inflow", "outflow")),
    (26, 10, 25, "internal", 3, ("inflow", "inflow")),
    (29, 8, 16, "nt", 2, ("periodic", "inflow")),
    (300, 1, 16, "total", 3, ("inflow", "periodic")),
]


@pytest.mark.parametrize("nx,ny,lattice,split,order,bc", CASES)
def test_fp64_fixed_k_matches_oracle(pond, orc, nx, ny, lattice, split, order, bc):
    ocfg, sim = make_pair(pond, orc, nx, ny, lattice, split, order, bc, K=3)
    st = random_state(orc, ocfg, seed=nx * ny)
    st = run_both(orc, ocfg, sim, st, 3)
    compare(orc, ocfg, sim, st, FP64_TOL, "case %s" % ((nx, ny, lattice, split, order, bc),))
    sim.close()


def test_fp64_set_state_equilibrium_start(pond, orc):
    ocfg, sim = make_pair(pond, orc, 40, 12, K=2)
    rng = np.random.default_rng(5)
    rho = 1 + 0.05 * rng.standard_normal((12, 40))
    ux = 0.5 + 0.05 * rng.standard_normal((12, 40))
    uy = -0.1 + 0.05 * rng.standard_normal((12, 40))
    T = 0.7 + 0.02 * rng.standard_normal((12, 40))
    st = orc.init_state(ocfg, rho, ux, uy, T)
    sim.set_state(rho, ux, uy, T)
    compare(orc, ocfg, sim, st, 1e-15, "init")
    for _ in range(4):
        st = orc.step(ocfg, st).state
    sim.step(4)
    compare(orc, ocfg, sim, st, FP64_TOL, "4 steps")
    sim.close()


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2), (1, 7), (6, 1), (2, 33), (130, 1)])
def test_fp64_degenerate_grids(pond, orc, nx, ny):
    ocfg, sim = make_pair(pond, orc, nx, ny, K=2, bc=("periodic", "outflow"))
    st = random_state(orc, ocfg, seed=7 + nx + ny)
    st = run_both(orc, ocfg, sim, st, 2)
    compare(orc, ocfg, sim, st, FP64_TOL, "grid %dx%d" % (nx, ny))
    sim.close()


def test_fp64_global_gather_fallback(pond, orc):
    """A staged box too small for the stencils sends every population to the global-memory
    gather path; the result must not change."""
    ocfg, sim = make_pair(pond, orc, 40, 12, K=2, halo=1)
    st = random_state(orc, ocfg, seed=3, ux0=1.5, T0=1.0)
    st = run_both(orc, ocfg, sim, st, 2)
    compare(orc, ocfg, sim, st, FP64_TOL, "fallback")
    rc, stats = sim.stats()
    assert stats.halo_fallbacks > 0
    sim.close()


def test_fp64_convergence_mode(pond, orc):
    """Iterating to the tolerance: iteration counts may differ at the margin, results agree
    to ~tolerance."""
    ocfg, sim = make_pair(pond, orc, 36, 10, K=0, tol=1e-12, maxit=30)
    st = random_state(orc, ocfg, seed=9)
    sim.set_populations(st.f, st.g, st.ux, st.uy, st.T)
    iters = 0
    for _ in range(3):
        r = orc.step(ocfg, st)
        st = r.state
        iters += int(r.iters.sum())
    sim.step(3)
    compare(orc, ocfg, sim, st, 1e-10, "converged")
    rc, stats = sim.stats()
    assert rc == 0
    assert abs(stats.pc_iters_total - iters) <= 0.02 * iters
    sim.close()


def test_fp64_sod_400x4_matches_oracle(pond, orc):
    """The Sod configuration (400 x 4, y periodic, x outflow), 400 steps, FP64."""
    from paper_2405_11489_gb300 import workloads as W
    c = W.sod(nx=400, ny=4, mu=1e-4 * 0.2 * 400)
    ocfg = orc.make_config(c.nx, c.ny, gamma=c.gamma, mu=c.mu, bc_x=c.bc_x, bc_y=c.bc_y,
                           pc_fixed_iters=3)
    st = orc.init_state(ocfg, c.rho, c.ux, c.uy, c.T)
    sim = pond.Simulation(pond.Config(nx=c.nx, ny=c.ny, precision="fp64", gamma=c.gamma, mu=c.mu,
                                      bc_x=c.bc_x, bc_y=c.bc_y, pc_fixed_iters=3))
    sim.set_state(c.rho, c.ux, c.uy, c.T)
    done = 0
    for upto in (50, 100, 200, c.steps):
        for _ in range(upto - done):
            st = orc.step(ocfg, st).state
        sim.step(upto - done)
        done = upto
        # rounding differences accumulate about linearly (measured on one GB300: 6.1e-14,
        # 2.0e-13, 5.6e-13, 1.8e-12 after 50, 100, 200, 400 steps, about 4.4e-15 per step);
        # the bound is 1e-12 for the first 160 steps and 6.25e-15 per step beyond
        errs = compare(orc, ocfg, sim, st, max(FP64_TOL, 6.25e-15 * done), "sod")
        print("sod fp64 step %d: max rel err %.2e %s" % (done, max(errs.values()), errs))
    sim.close()


def test_nonphysical_state_is_reported(pond, orc):
    ocfg, sim = make_pair(pond, orc, 12, 8, K=2)
    st = random_state(orc, ocfg, seed=4)
    sim.set_populations(st.f, -st.g, st.ux, st.uy, st.T)   # negative energy -> T < 0
    sim.step(1)
    rc, stats = sim.stats()
    assert rc == pond.POND_ENONPHYSICAL and stats.first_bad_node >= 0
    with pytest.raises(pond.PondError):
        sim.set_state(np.ones((8, 12)), np.zeros((8, 12)), np.zeros((8, 12)), -np.ones((8, 12)))
    # every kind of bad host field, at one node each
    for field, value in ((0, 0.0), (0, np.inf), (0, np.nan), (1, np.nan), (1, np.inf), (2, -np.inf),
                         (3, 0.0), (3, np.inf), (3, np.nan)):
        f = [np.ones((8, 12)), np.zeros((8, 12)), np.zeros((8, 12)), np.ones((8, 12))]
        f[field][5, 7] = value
        with pytest.raises(pond.PondError):
            sim.set_state(*f)
    sim.set_state(np.ones((8, 12)), np.full((8, 12), -3.0), np.zeros((8, 12)), np.ones((8, 12)))
    sim.close()


def test_nonconvergence_is_reported(pond, orc):
    ocfg, sim = make_pair(pond, orc, 12, 8, K=0, tol=0.0, maxit=2)
    st = random_state(orc, ocfg, seed=6)
    sim.set_populations(st.f, st.g, st.ux, st.uy, st.T)
    sim.step(1)
    rc, stats = sim.stats()
    assert rc == pond.POND_ENOCONV and stats.nonconv_updates == 12 * 8
    assert stats.pc_iters_max == 2
    sim.close()


@pytest.mark.parametrize("precision,lattice,split", [("fp64", 16, "total"), ("fp32", 16, "total"),
                                                    ("fp32", 25, "nt"), ("fp64", 25, "total")])
def test_checkpoint_resume_is_bit_identical(pond, orc, precision, lattice, split):
    """Export after 3 steps, import into a fresh simulation, 3 more steps: identical to 6
    straight steps (device and host checkpoints)."""
    from paper_2405_11489_gb300 import workloads as W
    c = W.shear_wave(n=48, ny=20, ma=1.0, amp=0.05, mu=0.05)
    cfg = pond.Config(nx=c.nx, ny=c.ny, precision=precision, mu=c.mu, lattice=lattice, split=split)
    a = pond.Simulation(cfg)
    a.set_state(c.rho, c.ux, c.uy, c.T)
    a.step(6)
    ref = a.moments()
    for on_device in (True, False):
        b = pond.Simulation(cfg)
        b.set_state(c.rho, c.ux, c.uy, c.T)
        b.step(3)
        mac, neq = b.export_state(on_device=on_device)
        b.close()
        d = pond.Simulation(cfg)
        d.import_state(mac, neq)
        d.step(3)
        for x, y in zip(d.moments(), ref):
            assert np.array_equal(x, y)
        d.close()
    a.close()


def test_couette_flow_on_the_gpu(pond):
    """Thermal Couette flow (Sec. III.B) between walls in both precisions on 32 cells: the
    steady temperature follows the analytic profile, the velocity is linear."""
    import math
    gamma, cp, T0, T1, Ec, mu, ny = 1.4, 3.5, 1.0, 1.005, 8.0, 0.1, 32
    u0 = math.sqrt(Ec * cp * (T1 - T0))
    walls = ((0, 0, 1, 1), (0, 0, 1, 1), (0.0, 0.0, T0, 1.0), (u0, 0.0, T1, 1.0 / T1))
    eta = (np.arange(ny) + 0.5) / ny
    exact = eta + 0.5 * Ec * eta * (1.0 - eta)
    for precision in ("fp64", "fp32"):
        sim = pond.Simulation(pond.Config(nx=1, ny=ny, precision=precision, bc_y="wall", walls=walls,
                                          gamma=gamma, mu=mu))
        sim.set_state(np.ones((ny, 1)), (u0 * eta)[:, None], np.zeros((ny, 1)), (T0 + (T1 - T0) * eta)[:, None])
        sim.step(int(2.5 * ny * ny / mu))
        rho, ux, uy, T = sim.moments()
        theta = (T[:, 0] - T0) / (T1 - T0)
        assert np.max(np.abs(theta - exact)) < 0.05, precision
        assert np.max(np.abs(ux[:, 0] / u0 - eta)) < 0.02, precision
        sim.close()


def _profiles(rng, nx, ny, sides):
    """Random per-position states (u_x, u_y, T, rho) along the given sides."""
    out = [None] * 4
    for w in sides:
        n = ny if w < 2 else nx
        out[w] = np.stack([0.3 + 0.1 * rng.standard_normal(n), 0.05 * rng.standard_normal(n),
                           0.8 + 0.05 * rng.standard_normal(n), 1.0 + 0.05 * rng.standard_normal(n)], 1)
    return out


@pytest.mark.parametrize("split,lattice,bc,sides", [
    ("total", 16, ("inflow", "wall"), (0, 2, 3)),
    ("internal", 16, ("inflow", "inflow"), (0, 2)),
    ("nt", 25, ("wall", "periodic"), (0, 1)),
])
def test_fp64_side_profiles_match_oracle(pond, orc, split, lattice, bc, sides):
    """Per-position side states (pond_set_boundary_profile), changed between steps, and
    restored to the uniform state, against the oracle with the same profiles."""
    nx, ny = 35, 19
    rng = np.random.default_rng(7)
    ocfg, sim = make_pair(pond, orc, nx, ny, lattice, split, 3, bc, K=3)
    st = random_state(orc, ocfg, seed=11)
    sim.set_populations(st.f, st.g, st.ux, st.uy, st.T)
    for phase in range(3):
        prof = _profiles(rng, nx, ny, sides) if phase < 2 else [None] * 4
        for w in sides:
            sim.set_boundary_profile(w, prof[w])
        pcfg = orc.make_config(nx, ny, lattice=lattice, split=split, bc_x=bc[0], bc_y=bc[1],
                               mu=0.02, pc_fixed_iters=3, walls=WALLS, profiles=prof)
        for _ in range(2):
            st = orc.step(pcfg, st).state
        sim.step(2)
        compare(orc, pcfg, sim, st, FP64_TOL, "phase %d" % phase)
    sim.close()


def test_fp64_batched_members_keep_their_profiles(pond, orc):
    """A batch of two inflow grids with different inlet profiles (one launch per step)."""
    nx, ny = 30, 14
    rng = np.random.default_rng(3)
    sims, pairs = [], []
    for k in range(2):
        ocfg, sim = make_pair(pond, orc, nx, ny, 16, "total", 3, ("inflow", "outflow"), K=2)
        prof = _profiles(rng, nx, ny, (0,))
        sim.set_boundary_profile("x_low", prof[0])
        pcfg = orc.make_config(nx, ny, bc_x="inflow", bc_y="outflow", mu=0.02, pc_fixed_iters=2,
                               walls=WALLS, profiles=prof)
        st = random_state(orc, ocfg, seed=20 + k)
        sim.set_populations(st.f, st.g, st.ux, st.uy, st.T)
        sims.append(sim)
        pairs.append((pcfg, st))
    batch = pond.Batch(sims)
    batch.step(3)
    for sim, (pcfg, st) in zip(sims, pairs):
        for _ in range(3):
            st = orc.step(pcfg, st).state
        compare(orc, pcfg, sim, st, FP64_TOL, "batched")
    batch.close()
    for s in sims:
        s.close()


def test_profile_shape_and_side_are_checked(pond):
    sim = pond.Simulation(pond.Config(nx=20, ny=10, bc_x="inflow", walls=tuple(WALLS)))
    with pytest.raises(ValueError):
        sim.set_boundary_profile("x_low", np.ones((20, 4)))      # x sides take ny states
    with pytest.raises(pond.PondError):
        sim.set_boundary_profile("x_high", np.ones((10, 4)))     # outflow side: not prescribed
    bad = np.ones((10, 4))
    bad[3, 2] = -1.0                                             # T <= 0
    with pytest.raises(pond.PondError):
        sim.set_boundary_profile("x_low", bad)
    sim.close()
