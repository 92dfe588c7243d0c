"""Pins of the oracle's lattice (Table I) and equilibria (Sec. II, Sec. III.A).

The lattice is checked against the printed Table I expressions, against numpy's
Gauss-Hermite (probabilists') rule, and against the closed-form quadrature exactness
sum_a w_a c_a^k = (k-1)!! that fixes the order of each rule.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_quadratures.txt")


def _table1():
    rows = {}
    env = {"sqrt": math.sqrt}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, node, weight = line.split()
            rows.setdefault(name, []).append((eval(node, env), eval(weight, env)))
    return rows


@pytest.mark.parametrize("q1,name", [(4, "D1Q4"), (5, "D1Q5")])
def test_lattice_matches_table1(orc, q1, name):
    c, w = orc.lattice_1d(q1)
    table = sorted(_table1()[name])
    got = sorted(zip(c, w))
    assert len(got) == len(table)
    for (c0, w0), (c1, w1) in zip(table, got):
        assert abs(c0 - c1) < 1e-15 and abs(w0 - w1) < 1e-15


@pytest.mark.parametrize("q1", [4, 5])
def test_lattice_is_gauss_hermite(orc, q1):
    """Table I rules are the probabilists' Gauss-Hermite rules (weights normalised to 1)."""
    c, w = orc.lattice_1d(q1)
    xg, wg = np.polynomial.hermite_e.hermegauss(q1)
    wg = wg / math.sqrt(2.0 * math.pi)
    order = np.argsort(c)
    assert np.allclose(c[order], xg, atol=1e-14)
    assert np.allclose(w[order], wg, atol=1e-14)


def _double_factorial(k):
    return 1 if k <= 0 else k * _double_factorial(k - 2)


@pytest.mark.parametrize("q1,exact_to", [(4, 7), (5, 9)])
def test_quadrature_exactness(orc, q1, exact_to):
    """An n-point Gauss-Hermite rule integrates the Gaussian moments exactly up to degree
    2n - 1 and fails at 2n: E[X^k] = (k-1)!! for even k, 0 for odd k."""
    c, w = orc.lattice_1d(q1)
    for k in range(exact_to + 1):
        exact = 0.0 if k % 2 else float(_double_factorial(k - 1))
        assert abs(np.sum(w * c ** k) - exact) < 1e-12 * max(1.0, exact)
    k = exact_to + 1
    assert abs(np.sum(w * c ** k) - _double_factorial(k - 1)) > 1.0


def _gauss_moment(k, mean, var):
    """E[X^k] for X ~ N(mean, var), from the binomial expansion and the central moments."""
    return sum(math.comb(k, j) * mean ** (k - j) * (var ** (j // 2)) * _double_factorial(j - 1)
               for j in range(0, k + 1, 2))


@pytest.mark.parametrize("lattice,pmax", [(16, 7), (25, 9)])
def test_feq_moments_exact(orc, lattice, pmax):
    """f_eq_i = rho w_i at C_i = sqrt(T) c_i + u (Sec. III.A) reproduces the Maxwellian's
    moments rho E[vx^p] E[vy^q] exactly for p, q up to the quadrature degree."""
    cx, cy, w = orc.lattice_2d(lattice)
    rho, ux, uy, T = 1.3, 2.1, -0.7, 0.45
    Cx, Cy = math.sqrt(T) * cx + ux, math.sqrt(T) * cy + uy
    f = rho * w
    for p in range(pmax + 1):
        for q in range(pmax + 1):
            exact = rho * _gauss_moment(p, ux, T) * _gauss_moment(q, uy, T)
            got = np.sum(f * Cx ** p * Cy ** q)
            assert abs(got - exact) <= 1e-11 * max(1.0, abs(exact)), (p, q)


@pytest.mark.parametrize("split", ["total", "internal"])
def test_geq_moments_exact(orc, split):
    """g_eq (Sec. II, per split) on the local lattice reproduces the continuous moments of
    (U'/rho + v^2/2) f_eq, resp. (U'/rho + (v-u)^2/2) f_eq, up to total degree 5 (D2Q16)."""
    gamma, rho, ux, uy, T = 1.4, 0.8, 1.7, 0.4, 0.6
    cv = 1.0 / (gamma - 1.0)
    cfg = orc.make_config(1, 1, lattice=16, split=split, gamma=gamma)
    st = orc.init_state(cfg, rho, ux, uy, T)
    cx, cy, w = orc.lattice_2d(16)
    Cx, Cy = math.sqrt(T) * cx + ux, math.sqrt(T) * cy + uy
    g = st.g[:, 0, 0]
    Up = (cv - 1.0) * T
    for p in range(4):
        for q in range(4):
            if p + q > 5:
                continue
            m = lambda a, b: _gauss_moment(a, ux, T) * _gauss_moment(b, uy, T)
            if split == "total":   # (U'/rho + (vx^2 + vy^2)/2) f_eq
                exact = rho * (Up * m(p, q) + 0.5 * (m(p + 2, q) + m(p, q + 2)))
            else:                   # (U'/rho + ((vx-ux)^2 + (vy-uy)^2)/2) f_eq
                exact = rho * (Up * m(p, q) + 0.5 * (m(p + 2, q) - 2 * ux * m(p + 1, q)
                                                     + ux * ux * m(p, q) + m(p, q + 2)
                                                     - 2 * uy * m(p, q + 1) + uy * uy * m(p, q)))
            got = np.sum(g * Cx ** p * Cy ** q)
            assert abs(got - exact) <= 1e-11 * max(1.0, abs(exact)), (p, q)


@pytest.mark.parametrize("split", ["total", "internal"])
@pytest.mark.parametrize("lattice", [16, 25])
def test_equilibrium_returns_its_moments(orc, split, lattice):
    """Equilibria built from (rho, u, T) give back (rho, u, T) to round-off, up to Ma 3."""
    rng = np.random.default_rng(3)
    ny, nx = 3, 5
    gamma = 1.4
    rho = rng.uniform(0.1, 2.0, (ny, nx))
    T = rng.uniform(0.05, 2.0, (ny, nx))
    ma = rng.uniform(0.0, 3.0, (ny, nx))
    th = rng.uniform(0, 2 * math.pi, (ny, nx))
    ux = ma * np.sqrt(gamma * T) * np.cos(th)
    uy = ma * np.sqrt(gamma * T) * np.sin(th)
    cfg = orc.make_config(nx, ny, lattice=lattice, split=split, gamma=gamma)
    st = orc.init_state(cfg, rho, ux, uy, T)
    r, vx, vy, TT, E = orc.moments(cfg, st)
    assert np.allclose(r, rho, rtol=1e-14, atol=0)
    assert np.allclose(vx, ux, rtol=0, atol=1e-13 * np.max(np.abs(ux)))
    assert np.allclose(vy, uy, rtol=0, atol=1e-13 * np.max(np.abs(uy)))
    assert np.allclose(TT, T, rtol=1e-12, atol=0)
    cv = 1.0 / (gamma - 1.0)
    assert np.allclose(E, rho * (cv * T + 0.5 * (ux ** 2 + uy ** 2)), rtol=1e-13)
