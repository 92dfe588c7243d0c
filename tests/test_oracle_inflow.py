"""Pins of the oracle's prescribed inflow (boundary type "inflow": the low side of the axis
holds ghost equilibria at a prescribed state, the high side is outflow; the paper imposes
prescribed conditions on the jet's inlet side, Sec. III.C, without a discretisation) and of
per-position boundary profiles:

- a supersonic inflow into a gas moving the same way is the Riemann problem between the
  inflow state (for x < 0) and the interior: with every wave moving into the domain the
  exact solution (gas-dynamics textbook) holds at the boundary too;
- a uniform flow entering at its own state stays uniform (all three energy splits: the
  internal split's gradients take the prescribed velocity beyond the side);
- a profile that equals the side's uniform state gives the same result as no profile, and
  rows far from a profile's edge (further than the domain of dependence) follow the run with
  that row's state on the whole side.
"""
import math

import numpy as np
import pytest

GAMMA = 1.4


def test_supersonic_inflow_matches_the_exact_riemann_solution(orc):
    from oracle.riemann import RiemannSolution
    nx, kappa, steps = 200, 0.2, 150
    a = math.sqrt(GAMMA)
    left = (1.0, 2.0 * a, 1.0)                 # Ma 2 inflow
    right = (0.5, 1.0 * a, 0.4)                # interior: slower, thinner, cooler
    sol = RiemannSolution(left, right, GAMMA)
    assert min(sol.wave_speeds()) > 0          # every wave enters the domain
    walls = [(kappa * left[1], 0.0, kappa ** 2 * left[2] / left[0], left[0])] + [(0.0, 0.0, 1.0, 1.0)] * 3
    cfg = orc.make_config(nx, 1, gamma=GAMMA, mu=1e-4 * kappa * nx, pc_tol=1e-10, bc_x="inflow",
                          walls=walls)
    st = orc.init_state(cfg, np.full((1, nx), right[0]), np.full((1, nx), kappa * right[1]),
                        np.zeros((1, nx)), np.full((1, nx), kappa ** 2 * right[2] / right[0]))
    for _ in range(steps):
        r = orc.step(cfg, st)
        assert r.status in (0, -5)
        st = r.state
    rho, ux, uy, T, E = orc.moments(cfg, st)
    t = steps * kappa / nx                     # unit length = nx cells, dt = kappa / nx
    xi = (np.arange(nx) + 0.5) / nx / t        # the inlet face lies half a cell before node 0
    re, ue, pe = sol.sample(xi)
    assert np.mean(np.abs(rho[0] - re)) < 1e-2
    assert np.mean(np.abs(ux[0] / kappa - ue)) < 1.3e-2
    assert np.mean(np.abs(rho[0] * T[0] / kappa ** 2 - pe)) < 1.4e-2
    # right shock within 2 cells of the exact front
    mid = 0.5 * (sol.rho_star_R + right[0])
    shock = -0.5 + sol.wave_speeds()[1] * t * nx
    assert abs(np.where(rho[0] > mid)[0].max() - shock) <= 2.0
    # star-left plateau (between the left shock and the contact) at the exact density
    xl = -0.5 + 0.5 * (sol.wave_speeds()[0] + sol.u_star) * t * nx
    assert abs(rho[0][int(xl)] / sol.rho_star_L - 1.0) < 0.025
    # the inlet region keeps the inflow state
    assert abs(rho[0][2] - left[0]) < 1e-3 and abs(ux[0][2] / kappa - left[1]) < 1e-3


@pytest.mark.parametrize("split", ["total", "internal", "nt"])
def test_uniform_flow_through_inflow_and_outflow_stays_uniform(orc, split):
    rho, ux, uy, T = 0.9, 0.45, 0.2, 0.7
    state = (ux, uy, T, rho)
    # x: inflow at x-low, outflow at x-high; y: inflow at y-low (u_y > 0), outflow at y-high
    cfg = orc.make_config(10, 8, split=split, bc_x="inflow", bc_y="inflow", walls=[state] * 4,
                          mu=0.02)
    st = orc.init_state(cfg, np.full((8, 10), rho), np.full((8, 10), ux), np.full((8, 10), uy),
                        np.full((8, 10), T))
    for _ in range(4):
        r = orc.step(cfg, st)
        assert r.status == 0
        st = r.state
    m = orc.moments(cfg, st)
    for got, want in zip(m[:4], (rho, ux, uy, T)):
        assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, abs(want))


def _jet_fields(nx, ny):
    rho = np.full((ny, nx), 1.0)
    return rho, np.full((ny, nx), 0.2), np.zeros((ny, nx)), np.full((ny, nx), 1.0)


def test_uniform_profile_equals_the_uniform_side_state(orc):
    nx, ny = 12, 9
    inflow = (0.5, 0.05, 1.2, 1.3)
    walls = [inflow, (0, 0, 1, 1), (0.0, 0.0, 1.0, 1.0), (0.1, 0.0, 0.9, 1.1)]
    prof = [np.tile(inflow, (ny, 1)), None, np.tile(walls[2], (nx, 1)), np.tile(walls[3], (nx, 1))]
    out = []
    for profiles in (None, prof):
        cfg = orc.make_config(nx, ny, bc_x="inflow", bc_y="wall", walls=walls, profiles=profiles,
                              mu=0.05)
        st = orc.init_state(cfg, *_jet_fields(nx, ny))
        for _ in range(3):
            st = orc.step(cfg, st).state
        out.append(st)
    for a, b in zip((out[0].f, out[0].g, out[0].ux, out[0].uy, out[0].T),
                    (out[1].f, out[1].g, out[1].ux, out[1].uy, out[1].T)):
        assert np.array_equal(a, b)


def test_profile_rows_follow_their_own_inflow_state(orc):
    """Upper half of the inlet at state A, lower half at state B (y periodic): after a few
    steps, rows further from the profile's edges than the domain of dependence equal the
    runs with A, respectively B, on the whole side."""
    nx, ny, steps = 16, 64, 3
    A = (0.6, 0.0, 1.3, 1.2)
    B = (0.3, 0.0, 0.8, 0.9)
    prof = np.array([B if y < ny // 2 else A for y in range(ny)], dtype=float)
    res = {}
    for name, walls, profiles in (("mix", [A] * 4, [prof, None, None, None]),
                                  ("A", [A] * 4, None), ("B", [B] * 4, None)):
        cfg = orc.make_config(nx, ny, bc_x="inflow", walls=walls, profiles=profiles, mu=0.05)
        st = orc.init_state(cfg, *_jet_fields(nx, ny))
        for _ in range(steps):
            st = orc.step(cfg, st).state
        res[name] = orc.moments(cfg, st)
    # the fastest population moves < 2.7 cells per step and the stencil reaches 2 more: rows
    # 16 (B) and 48 (A) lie 16 rows from both edges (0 / 32, periodic)
    for row, ref in ((16, "B"), (48, "A")):
        for k in range(4):
            got, want = res["mix"][k][row], res[ref][k][row]
            assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))
    # and the two halves differ: the profile is seen
    assert np.max(np.abs(res["mix"][0][16] - res["mix"][0][48])) > 1e-3
