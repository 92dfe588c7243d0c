"""Whole-step physics of the CUDA path in the mixed precisions, against the hydrodynamic
limit of Sec. II and the measurements of Sec. III.B (the same closed forms that pin the
FP64 oracle, here on the GPU without the oracle in the loop):

- shear-wave decay rate nu k^2, nu = tau T (Sec. III.B, shear viscosity), at rest and under
  a Mach 1.5 background flow;
- entropy-wave decay rate alpha k^2 with alpha = tau T (Pr = 1), total and internal split;
- speed of a weak pressure front sqrt(gamma T) (Sec. III.B, speed of sound);
- attenuation of a standing sound wave nu k^2, the value that the bulk viscosity
  eta = (2/D - r/c_v) mu of Sec. II gives in D = 2 with Pr = 1 (without it: gamma nu k^2 / 2),
  for the total and internal splits on D2Q16 and the non-translational split on D2Q25.
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


def _sim(pond, case, precision="fp32", **kw):
    s = pond.Simulation(pond.Config(nx=case.nx, ny=case.ny, precision=precision, gamma=case.gamma,
                                    mu=case.mu, bc_x=case.bc_x, bc_y=case.bc_y, **kw))
    s.set_state(case.rho, case.ux, case.uy, case.T)
    return s


def _mode(field, n):
    x = np.arange(n)
    return 2.0 * abs(np.mean(field * np.exp(-2j * math.pi * x / n)))


@pytest.mark.parametrize("ma", [0.0, 1.5])
def test_shear_wave_decay_rate(pond, ma):
    case = W.shear_wave(n=64, ny=1, ma=ma, amp=1e-3, mu=0.05, steps=300)
    s = _sim(pond, case)
    ts, amps = [], []
    for k in range(6):
        s.step(50)
        ts.append(50 * (k + 1))
        amps.append(_mode(s.moments()[2][0], case.nx))
    nu = -np.polyfit(ts, np.log(amps), 1)[0] / case.meta["k"] ** 2
    assert abs(nu / case.mu - 1.0) < 0.02
    s.close()


@pytest.mark.parametrize("split,precision", [("total", "fp32"), ("internal", "fp32"), ("internal", "fp64")])
def test_thermal_wave_decay_rate(pond, split, precision):
    case = W.thermal_wave(n=128, amp=1e-3, mu=0.05, steps=600)
    s = _sim(pond, case, precision=precision, split=split)
    s.step(150)
    ts, amps = [], []
    for k in range(9):
        s.step(50)
        ts.append(200 + 50 * k)
        amps.append(_mode(s.moments()[3][0] - 1.0, case.nx))
    alpha = -np.polyfit(ts, np.log(amps), 1)[0] / case.meta["k"] ** 2
    assert abs(alpha / case.mu - 1.0) < 0.01
    s.close()


@pytest.mark.parametrize("gamma", [1.4, 1.8])
def test_sound_speed(pond, gamma):
    T0 = 0.5
    case = W.pressure_step(n=300, dp=1e-3, T0=T0, gamma=gamma, mu=1e-3, steps=80)
    s = _sim(pond, case)
    s.step(10)
    ts, xs = [], []
    for k in range(7):
        s.step(10)
        rho, ux, uy, T = s.moments()
        p = (rho * T)[0, case.meta["x0"]:]
        pmid = T0 * (1.0 + case.meta["dp"] / 4.0)
        j = np.where(p > pmid)[0].max()
        ts.append(20 + 10 * k)
        xs.append(j + (p[j] - pmid) / (p[j] - p[j + 1]))
    cs = np.polyfit(ts, xs, 1)[0]
    assert abs(cs / math.sqrt(gamma * T0) - 1.0) < 0.01
    s.close()


@pytest.mark.parametrize("split,lattice,gamma", [("total", 16, 1.4), ("total", 16, 1.8), ("nt", 25, 1.8),
                                                 ("internal", 16, 1.4), ("internal", 16, 1.8)])
def test_sound_attenuation_gives_the_bulk_viscosity(pond, split, lattice, gamma):
    n, mu, A = 64, 0.05, 1e-4
    x = np.arange(n)[None, :]
    k = 2 * math.pi / n
    rho = 1.0 + A * np.sin(k * x)
    s = pond.Simulation(pond.Config(nx=n, ny=1, lattice=lattice, split=split, precision="fp32",
                                    gamma=gamma, mu=mu))
    s.set_state(rho, np.zeros((1, n)), np.zeros((1, n)), rho ** (gamma - 1.0))
    ts, es = [], []
    for step in range(120):
        s.step(4)
        r, ux, uy, T = s.moments()
        ts.append(4 * (step + 1))
        es.append(np.mean(r * ux * ux + gamma * (r - 1.0) ** 2))   # acoustic energy
    rate = -np.polyfit(ts, np.log(es), 1)[0] / 2.0
    assert abs(rate / (mu * k * k) - 1.0) < 0.02
    s.close()
