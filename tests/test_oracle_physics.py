"""Whole-step pins of the oracle against the hydrodynamic limit of Sec. II and the
measurements of Sec. III.B:

- Sod's shock tube against the exact Riemann solution (gas-dynamics textbook);
- shear-wave decay rate k^2 nu with nu = tau T (Sec. III.B, shear viscosity), independent
  of the background Mach number (Galilean invariance the paper reports);
- entropy-wave decay rate k^2 alpha with alpha = tau T (Pr = 1, Eq. therm_cond);
- speed of a weak pressure front sqrt(gamma T) for gamma = 1.4 and 1.8 (Sec. III.B).
Each tolerance is far below the error a dropped term or a wrong factor would cause
(e.g. omega = 1/tau instead of 1/(tau + 1/2) changes nu by T/2, a factor 11 here).
"""
import math

import numpy as np
import pytest

from paper_2405_11489_gb300 import workloads as W


def _run(orc, case, **kw):
    cfg = orc.make_config(case.nx, case.ny, gamma=case.gamma, mu=case.mu, bc_x=case.bc_x,
                          bc_y=case.bc_y, **kw)
    st = orc.init_state(cfg, case.rho, case.ux, case.uy, case.T)
    return cfg, st


def _mode(field, n):
    x = np.arange(n)
    return 2.0 * abs(np.mean(field * np.exp(-2j * math.pi * x / n)))


def test_sod_matches_exact_riemann(orc):
    from oracle.riemann import RiemannSolution
    nx, kappa = 200, 0.2
    # viscosity 1e-4 in the units of the stated states, i.e. mu_lat = 1e-4 * kappa * nx
    case = W.sod(nx=nx, ny=1, kappa=kappa, mu=1e-4 * kappa * nx)
    cfg, st = _run(orc, case, pc_tol=1e-10)
    for _ in range(case.steps):
        r = orc.step(cfg, st)
        assert r.status in (0, -5)
        st = r.state
    rho, ux, uy, T, E = orc.moments(cfg, st)
    sol = RiemannSolution((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    t = case.steps * kappa / nx
    xi = (np.arange(nx) - case.meta["x0"] + 0.5) / nx / t
    re, ue, pe = sol.sample(xi)
    assert np.mean(np.abs(rho[0] - re)) < 6e-3
    assert np.mean(np.abs(ux[0] / kappa - ue)) < 1.2e-2
    assert np.mean(np.abs(rho[0] * T[0] / kappa ** 2 - pe)) < 5e-3
    # shock position: last node above the mid density, within 2 cells of the exact front
    mid = 0.5 * (sol.rho_star_R + 0.125)
    shock = case.meta["x0"] - 0.5 + sol.wave_speeds()[1] * t * nx
    assert abs(np.where(rho[0] > mid)[0].max() - shock) <= 2.0
    # plateau between contact and shock at the exact star-right density
    plate = rho[0][int(case.meta["x0"] + 0.5 * (sol.u_star + sol.wave_speeds()[1]) * t * nx)]
    assert abs(plate / sol.rho_star_R - 1.0) < 0.02


@pytest.mark.parametrize("ma", [0.0, 1.5])
def test_shear_wave_decay_rate(orc, ma):
    case = W.shear_wave(n=64, ny=1, ma=ma, amp=1e-3, mu=0.05, steps=300)
    cfg, st = _run(orc, case)
    ts, amps = [], []
    for s in range(case.steps):
        st = orc.step(cfg, st).state
        if s % 50 == 49:
            ts.append(s + 1)
            amps.append(_mode(orc.moments(cfg, st)[2][0], case.nx))
    nu = -np.polyfit(ts, np.log(amps), 1)[0] / case.meta["k"] ** 2
    assert abs(nu / case.mu - 1.0) < 0.02        # nu = tau T = mu / rho with rho = 1


@pytest.mark.parametrize("split", ["total", "internal"])
def test_thermal_wave_decay_rate(orc, split):
    case = W.thermal_wave(n=128, amp=1e-3, mu=0.05, steps=600)
    cfg, st = _run(orc, case, split=split)
    ts, amps = [], []
    for s in range(case.steps):
        st = orc.step(cfg, st).state
        if s >= 199 and s % 50 == 49:
            ts.append(s + 1)
            amps.append(_mode(orc.moments(cfg, st)[3][0] - 1.0, case.nx))
    alpha = -np.polyfit(ts, np.log(amps), 1)[0] / case.meta["k"] ** 2
    assert abs(alpha / case.mu - 1.0) < 0.01     # alpha = tau T, Pr = 1


@pytest.mark.parametrize("gamma", [1.4, 1.8])
def test_sound_speed(orc, gamma):
    T0 = 0.5
    case = W.pressure_step(n=300, dp=1e-3, T0=T0, gamma=gamma, mu=1e-3, steps=80)
    cfg, st = _run(orc, case)
    ts, xs = [], []
    for s in range(case.steps):
        st = orc.step(cfg, st).state
        if s >= 19 and s % 10 == 9:
            rho, ux, uy, T, E = orc.moments(cfg, st)
            p = (rho * T)[0, case.meta["x0"]:]
            pmid = T0 * (1.0 + case.meta["dp"] / 4.0)   # half-way up the right-moving front
            k = np.where(p > pmid)[0].max()
            ts.append(s + 1)
            xs.append(k + (p[k] - pmid) / (p[k] - p[k + 1]))
    cs = np.polyfit(ts, xs, 1)[0]
    assert abs(cs / math.sqrt(gamma * T0) - 1.0) < 0.01


def test_d2q25_shear_decay(orc):
    case = W.shear_wave(n=48, ny=1, ma=0.5, amp=1e-3, mu=0.05, steps=200)
    cfg, st = _run(orc, case, lattice=25)
    ts, amps = [], []
    for s in range(case.steps):
        st = orc.step(cfg, st).state
        if s % 50 == 49:
            ts.append(s + 1)
            amps.append(_mode(orc.moments(cfg, st)[2][0], case.nx))
    nu = -np.polyfit(ts, np.log(amps), 1)[0] / case.meta["k"] ** 2
    assert abs(nu / case.mu - 1.0) < 0.03


def test_internal_split_source_is_pdv_work(orc):
    """The internal-split source (Eq. int_g_evolution with f -> f_eq) adds sum_i G_i =
    -p div u to the internal energy: for a uniform-T compression u_x = -e (x - x0) the
    internal energy after one step grows by ~ p e per unit time relative to the
    total split, to first order."""
    nx = 32
    x = np.arange(nx, dtype=float)
    e = 1e-4
    rho = np.ones((1, nx))
    ux = (-e * (x - nx / 2))[None, :]
    uy = np.zeros((1, nx))
    T = np.ones((1, nx))
    res = {}
    for split in ("total", "internal"):
        cfg = orc.make_config(nx, 1, split=split, gamma=1.4, mu=0.05, bc_x="outflow",
                              pc_tol=1e-13)
        st = orc.init_state(cfg, rho, ux, uy, T)
        for _ in range(2):
            st = orc.step(cfg, st).state
        res[split] = orc.moments(cfg, st)[3][0]
    # both splits agree on the temperature in the interior (same hydrodynamics)
    mid = slice(8, 24)
    assert np.allclose(res["total"][mid], res["internal"][mid], rtol=2e-6, atol=0)
    # and the compression heats the gas: dT/dt = (gamma - 1) T e for an ideal gas
    dT = res["total"][nx // 2] - 1.0
    assert abs(dT / (2 * 0.4 * e) - 1.0) < 0.05
