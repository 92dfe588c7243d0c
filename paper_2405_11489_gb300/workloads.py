"""Seeded synthetic initial conditions shaped like the paper's test cases (Sec. III.B).

This module holds no arithmetic of the PonD method: it only produces macroscopic
fields (rho, u_x, u_y, T) on a grid, in lattice units (r = 1), which both the CUDA
library and the FP64 oracle then turn into equilibrium populations themselves.
Every generator is deterministic given its arguments (numpy ``default_rng(seed)``).

Fields are float64 arrays of shape (ny, nx), row-major, x fastest.

Velocity scale: a shock tube stated in gas-dynamics units (rho, u, p) is mapped to
lattice units with a velocity scale kappa = dt/dx:  u_lat = kappa u,  T_lat = kappa^2 p/rho.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Largest |c_a| of the D1Q4 quadrature, sqrt(3 + sqrt 6) (Table I); a population moves
# at most |u| + C_MAX sqrt(T) cells per step.  Used only to choose velocity scales.
C_MAX_Q16 = math.sqrt(3.0 + math.sqrt(6.0))


@dataclass
class Case:
    """One initial-value problem: fields plus the configuration it is meant to run with."""
    name: str
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray
    gamma: float = 1.4
    mu: float = 1e-4
    bc_x: str = "periodic"
    bc_y: str = "periodic"
    steps: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def ny(self) -> int:
        return self.rho.shape[0]

    @property
    def nx(self) -> int:
        return self.rho.shape[1]


def _fields(ny, nx):
    return (np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), np.ones((ny, nx)))


def _blend(xs, x0, width):
    """Weight of the left state: a step at x0 - 1/2, or a tanh profile of the given width."""
    if width <= 0:
        return (xs < x0).astype(float)
    return 0.5 * (1.0 - np.tanh((xs - (x0 - 0.5)) / width))


def shock_tube(nx, ny, left, right, gamma=1.4, kappa=0.2, mu=1e-4, steps=None, x0=None,
               name="tube", width=0.0):
    """Left/right states (rho, u, p) in gas-dynamics units, split at x0 (default nx/2);
    x outflow, y periodic.  kappa = lattice velocity scale.  width > 0 resolves the initial
    discontinuity over a tanh profile of that many cells (density, velocity and pressure
    blended, T = p/rho)."""
    rho, ux, uy, T = _fields(ny, nx)
    x0 = nx // 2 if x0 is None else x0
    xs = np.arange(nx, dtype=float)[None, :].repeat(ny, 0)
    wl = _blend(xs, x0, width)
    r = wl * left[0] + (1 - wl) * right[0]
    u = wl * left[1] + (1 - wl) * right[1]
    p = wl * left[2] + (1 - wl) * right[2]
    rho[:] = r
    ux[:] = kappa * u
    T[:] = kappa * kappa * p / r
    return Case(name, rho, ux, uy, T, gamma=gamma, mu=mu, bc_x="outflow", bc_y="periodic",
                steps=steps if steps is not None else nx,
                meta={"kappa": kappa, "left": left, "right": right, "x0": x0, "width": width})


def sod(nx=400, ny=4, kappa=0.2, mu=None):
    """Sod's problem: (1, 0, 1) | (0.125, 0, 0.1), gamma = 1.4.  With nx cells over the unit
    length and kappa = 0.2, nx steps reach t = 0.2 in gas-dynamics units (dt = kappa/nx).
    Default viscosity: 1e-4 in the units of the states, i.e. mu_lat = 1e-4 kappa nx."""
    mu = 1e-4 * kappa * nx if mu is None else mu
    return shock_tube(nx, ny, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), gamma=1.4, kappa=kappa, mu=mu,
                      steps=nx, name="sod")


def shear_wave(n=256, ny=None, ma=1.0, amp=0.05, gamma=1.4, mu=0.05, steps=2000):
    """Transverse shear wave u_y = amp sin(2 pi x / n) on rho = 1, T = 1, with a uniform
    background u_x = Ma sqrt(gamma T) (Sec. III.B, shear viscosity)."""
    ny = n if ny is None else ny
    rho, ux, uy, T = _fields(ny, n)
    x = np.arange(n)[None, :]
    ux[:] = ma * math.sqrt(gamma)
    uy[:] = amp * np.sin(2.0 * math.pi * x / n)
    return Case("shear", rho, ux, uy, T, gamma=gamma, mu=mu, steps=steps,
                meta={"ma": ma, "amp": amp, "k": 2 * math.pi / n})


def thermal_wave(n=64, ny=1, amp=1e-3, gamma=1.4, mu=0.05, ma=0.0, steps=400):
    """Isobaric entropy wave rho = 1 + amp sin(2 pi x/n), T = 1/rho (Sec. III.B, thermal
    diffusivity), optional background u_x = Ma sqrt(gamma)."""
    rho, ux, uy, T = _fields(ny, n)
    x = np.arange(n)[None, :]
    rho[:] = 1.0 + amp * np.sin(2.0 * math.pi * x / n)
    T[:] = 1.0 / rho
    ux[:] = ma * math.sqrt(gamma)
    return Case("thermal_wave", rho, ux, uy, T, gamma=gamma, mu=mu, steps=steps,
                meta={"amp": amp, "k": 2 * math.pi / n, "ma": ma})


def thermal_pulse(n=256, amp=1e-3, width=16.0, gamma=1.4, mu=0.05, ma=0.0, steps=2000):
    """Gaussian isobaric temperature pulse T = 1 + amp exp(-r^2 / (2 width^2)) at the box
    centre, rho = 1/T, on a periodic n x n box."""
    rho, ux, uy, T = _fields(n, n)
    y, x = np.mgrid[0:n, 0:n]
    r2 = (x - n / 2.0) ** 2 + (y - n / 2.0) ** 2
    T[:] = 1.0 + amp * np.exp(-r2 / (2.0 * width * width))
    rho[:] = 1.0 / T
    ux[:] = ma * math.sqrt(gamma)
    return Case("thermal_pulse", rho, ux, uy, T, gamma=gamma, mu=mu, steps=steps,
                meta={"amp": amp, "width": width, "ma": ma})


def pressure_step(n=200, dp=1e-3, T0=1.0, gamma=1.4, mu=1e-3, steps=60):
    """Freely travelling pressure front (Sec. III.B, speed of sound): left half at
    p = (1 + dp) rho T0 by a density step, uniform temperature T0, u = 0; x outflow."""
    rho, ux, uy, T = _fields(1, n)
    T[:] = T0
    rho[:, : n // 2] = 1.0 + dp
    return Case("pressure_step", rho, ux, uy, T, gamma=gamma, mu=mu, bc_x="outflow",
                steps=steps, meta={"dp": dp, "T0": T0, "x0": n // 2})


def riemann2d(n=1024, seed=0, gamma=1.4, max_disp=2.0, mu=1e-3, steps=500, width=4.0, mu_lat=None):
    """Four-quadrant 2-D Riemann problem: per quadrant rho ~ U[0.1, 1.5], p ~ U[0.03, 1.5],
    flow direction ~ U[0, 2 pi), |u| ~ U[0, 1.2 sqrt(gamma p / rho)]; outflow on all sides.
    The lattice velocity scale makes the largest population displacement max_disp cells.
    mu is given in the units of the states on the unit square (mu_lat = mu kappa n) unless
    mu_lat is given.  width > 0 blends the quadrants over tanh profiles of that many cells."""
    rng = np.random.default_rng(seed)
    states = []
    for _ in range(4):
        r = rng.uniform(0.1, 1.5)
        p = rng.uniform(0.03, 1.5)
        th = rng.uniform(0.0, 2.0 * math.pi)
        um = rng.uniform(0.0, 1.2 * math.sqrt(gamma * p / r))
        states.append((r, um * math.cos(th), um * math.sin(th), p))
    vmax = max(math.hypot(ux, uy) + C_MAX_Q16 * math.sqrt(p / r) for r, ux, uy, p in states)
    kappa = max_disp / vmax
    rho, ux, uy, T = _fields(n, n)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    wr = 1.0 - _blend(x, n // 2, width)        # weight of the x >= n/2 side
    wt = 1.0 - _blend(y, n // 2, width)        # weight of the y >= n/2 side
    quads = [wr * wt, (1 - wr) * wt, (1 - wr) * (1 - wt), wr * (1 - wt)]
    pres = np.zeros((n, n))
    rho[:] = 0.0
    for (r, vx, vy, p), w in zip(states, quads):
        rho += w * r
        ux += w * kappa * vx
        uy += w * kappa * vy
        pres += w * kappa * kappa * p
    T[:] = pres / rho
    ma = max(math.hypot(vx, vy) / math.sqrt(gamma * p / r) for r, vx, vy, p in states)
    mul = mu * kappa * n if mu_lat is None else mu_lat
    return Case("riemann2d", rho, ux, uy, T, gamma=gamma, mu=mul, bc_x="outflow",
                bc_y="outflow", steps=steps,
                meta={"seed": seed, "kappa": kappa, "states": states, "max_ma": ma, "width": width})


def jet(nx=2000, ny=1000, diameter=100.0, ma=1.5, jet_state=(5.0, 0.005), ambient=(50.0, 0.0005),
        gamma=1.4, mu=1e-3, width=2.0, steps=240):
    """The jet of Sec. III.C: a semicircle of diameter `diameter` on the left side holds the
    jet state (rho, T) = jet_state moving at Mach `ma` along x; the rest of the domain is at
    rest at `ambient` (the paper: Ma 80, (5, 0.005) into (50, 0.0005), 2000 x 1000, D = 100).
    The left side is an inflow side whose profile is the jet state inside the jet's diameter
    and the ambient state outside; outflow elsewhere.  width > 0 blends jet and ambient over
    a tanh profile of that many cells (density and pressure blended, T = p/rho).  The inlet
    profile is meta["profile"] ([ny][4]: u_x, u_y, T, rho) and meta["walls"] the four side
    states (the x-low one is the profile's first entry)."""
    rho_j, T_j = jet_state
    rho_a, T_a = ambient
    u_j = ma * math.sqrt(gamma * T_j)
    yc = np.arange(ny, dtype=float) - (ny - 1) / 2.0

    def inside(r):
        if width <= 0:
            return (r <= diameter / 2.0).astype(float)
        return 0.5 * (1.0 - np.tanh((r - diameter / 2.0) / width))

    def state(s):
        rho = rho_a + (rho_j - rho_a) * s
        p = rho_a * T_a + (rho_j * T_j - rho_a * T_a) * s
        return rho, u_j * s, p / rho

    r_in, u_in, T_in = state(inside(np.abs(yc)))
    prof = np.stack([u_in, np.zeros(ny), T_in, r_in], 1)
    x = np.arange(nx, dtype=float)[None, :]
    rho, ux, T = state(inside(np.sqrt((x + 0.5) ** 2 + yc[:, None] ** 2)))
    walls = [tuple(prof[0])] * 4
    return Case("jet", rho, ux, np.zeros((ny, nx)), T, gamma=gamma, mu=mu, bc_x="inflow",
                bc_y="outflow", steps=steps,
                meta={"ma": ma, "u_jet": u_j, "diameter": diameter, "profile": prof, "walls": walls,
                      "jet_state": jet_state, "ambient": ambient, "width": width})


def tube_batch(count=256, seed=1, nmin=200, nmax=4000, gamma=1.4, mu=1e-3, width=4.0):
    """Uneven quasi-1-D shock tubes: N ~ logU[nmin, nmax] cells (ny = 1), p_L/p_R ~ logU[2, 100],
    rho_L/rho_R ~ logU[1, 10] (right state rho = 0.125, p = 0.1 as in Sod).  Each tube's
    velocity scale keeps its fastest wave inside the tube over N steps and bounds the
    population displacement by 2 cells per step.  mu is given in the units of the states on a
    tube of unit length: mu_lat = mu kappa N; the discontinuity is resolved over a tanh
    profile of `width` cells.  With the 3-point interpolation of Sec. III.A.2 these tubes stay
    physical over their N steps at the strongest pressure and temperature jumps."""
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(count):
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        pr_ratio = math.exp(rng.uniform(math.log(2.0), math.log(100.0)))
        rho_ratio = math.exp(rng.uniform(0.0, math.log(10.0)))
        right = (0.125, 0.0, 0.1)
        left = (0.125 * rho_ratio, 0.0, 0.1 * pr_ratio)
        aL = math.sqrt(gamma * left[2] / left[0])
        aR = math.sqrt(gamma * right[2] / right[0])
        # Upper bound of the right-moving shock speed (p* <= p_L) and the left rarefaction head.
        s_shock = aR * math.sqrt((gamma + 1) / (2 * gamma) * pr_ratio + (gamma - 1) / (2 * gamma))
        smax = max(aL, s_shock)
        vmax = C_MAX_Q16 * max(math.sqrt(left[2] / left[0]), math.sqrt(right[2] / right[0])) + smax
        kappa = min(0.45 / smax, 2.0 / vmax)
        c = shock_tube(N, 1, left, right, gamma=gamma, kappa=kappa, mu=mu * kappa * N, steps=N,
                       name="tube%03d" % k, width=width)
        cases.append(c)
    return cases


@dataclass
class Request:
    """One simulation request of the serving workload."""
    rid: int
    arrival: float              # seconds after the start of the stream
    case: Case
    precision: str              # "fp32" or "fp64"
    split: str                  # "total" or "internal"
    interp_order: int
    steps: int


def serving_requests(count=10000, rate=50.0, seed=2, step_scale=1.0, max_side=1024):
    """Poisson request stream: exponential inter-arrival times of mean 1/rate; the type is
    uniform over shock tubes (N ~ logU[400, 4000], N steps), 2-D Riemann problems
    (n ~ logU[128, 1024] squared, 100 steps) and periodic decay cases (n ~ logU[64, 512]
    squared, 200 steps); Ma ~ U[0.5, 3] (background flow of decay cases); split and precision
    Bernoulli(1/2).  step_scale multiplies the step counts (to set the offered load)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        kind = int(rng.integers(3))
        ma = rng.uniform(0.5, 3.0)
        split = "internal" if rng.random() < 0.5 else "total"
        precision = "fp64" if rng.random() < 0.5 else "fp32"
        if kind == 0:
            N = int(round(math.exp(rng.uniform(math.log(400), math.log(4000)))))
            pr = math.exp(rng.uniform(math.log(2.0), math.log(100.0)))
            rr = math.exp(rng.uniform(0.0, math.log(10.0)))
            right = (0.125, 0.0, 0.1)
            left = (0.125 * rr, 0.0, 0.1 * pr)
            aR = math.sqrt(1.4 * right[2] / right[0])
            aL = math.sqrt(1.4 * left[2] / left[0])
            smax = max(aL, aR * math.sqrt(1.2 / 1.4 * pr + 0.2 / 1.4))
            vmax = C_MAX_Q16 * max(math.sqrt(left[2] / left[0]), math.sqrt(right[2] / right[0])) + smax
            kappa = min(0.45 / smax, 2.0 / vmax)
            case = shock_tube(N, 1, left, right, kappa=kappa, mu=1e-3 * kappa * N, width=4.0,
                              name="tube")
            order, steps = 2, N
        elif kind == 1:
            n = int(round(math.exp(rng.uniform(math.log(128), math.log(max_side)))))
            case = riemann2d(n=n, seed=int(rng.integers(1 << 30)))
            order, steps = 2, 100
        else:
            n = int(round(math.exp(rng.uniform(math.log(64), math.log(min(512, max_side))))))
            case = shear_wave(n=n, ma=ma, amp=0.05, mu=0.05)
            order, steps = 3, 200
        out.append(Request(k, t, case, precision, split, order,
                           max(1, int(round(steps * step_scale)))))
    return out
