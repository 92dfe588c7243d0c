"""Pin of the FP64 oracle's rounding: a 3x3 and a 4x3 periodic grid stepped twice by the
oracle and by a separate 50-digit implementation (tests/mp_reference.py) with the same
readings agree to FP64 round-off in every population and frame value, for the three energy
splits and both lattices (Grad order N = 3 on D2Q16, 4 on D2Q25)."""
import math

import numpy as np
import pytest

import mp_reference as M


def _fields(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx]
    rho = 1.0 + 0.05 * np.sin(2 * math.pi * (x / nx + 0.3)) * np.cos(2 * math.pi * y / ny)
    ux = 0.3 + 0.05 * np.cos(2 * math.pi * y / ny + 0.4)
    uy = -0.2 + 0.04 * np.sin(2 * math.pi * x / nx)
    T = 0.9 + 0.05 * np.cos(2 * math.pi * (x / nx - y / ny))
    return rho, ux, uy, T


@pytest.mark.parametrize("nx,ny,lattice,split", [(3, 3, 16, "total"), (3, 3, 16, "internal"),
                                                 (4, 3, 25, "total"), (3, 3, 25, "nt"),
                                                 (3, 3, 16, "nt")])
def test_oracle_matches_50_digit_step(orc, nx, ny, lattice, split):
    gamma, mu, K, steps = 1.4, 0.05, 2, 2
    fields = _fields(nx, ny)
    cfg = orc.make_config(nx, ny, lattice=lattice, split=split, gamma=gamma, mu=mu, pc_fixed_iters=K)
    st = orc.init_state(cfg, *fields)
    lat = M.Lattice({16: 4, 25: 5}[lattice])
    ref = M.init(lat, nx, ny, *fields, split=split, gamma=gamma)
    for _ in range(steps):
        st = orc.step(cfg, st).state
        ref = M.step(lat, ref, nx, ny, split, gamma, mu, K)
    f_ref = np.array([[float(v) for v in ref["f"][n]] for n in range(nx * ny)]).T.reshape(-1, ny, nx)
    g_ref = np.array([[float(v) for v in ref["g"][n]] for n in range(nx * ny)]).T.reshape(-1, ny, nx)
    fr_ref = np.array([[float(v) for v in ref["fr"][n]] for n in range(nx * ny)]).T.reshape(3, ny, nx)
    tol = 2e-13
    assert np.max(np.abs(st.f - f_ref)) <= tol * np.max(np.abs(f_ref))
    assert np.max(np.abs(st.g - g_ref)) <= tol * np.max(np.abs(g_ref))
    for a, b in zip((st.ux, st.uy, st.T), fr_ref):
        assert np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(b)), 1.0)
    # the step did something: non-equilibrium content well above the tolerance
    feq = np.array([[float(lat.w[i]) for i in range(lat.Q)]]).T.reshape(-1, 1, 1) * f_ref.sum(axis=0)
    assert np.max(np.abs(f_ref - feq)) > 1e-4
