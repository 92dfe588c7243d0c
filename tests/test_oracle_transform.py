"""Pins of the oracle's frame transformation (Sec. III.A.1, Eq. gradGeneralTransform and
the expanded coefficients a_0 .. a_3 that follow it).

- moment matching (Eq. genericMomentUptoO3): the transformed populations carry every raw
  moment sum_i f_i C_x^p C_y^q of total order <= 3 of the source, in any pair of frames;
  order 4 is not kept (reduced Grad expansion, N = 3);
- the transform is a projection: applying it twice changes nothing;
- the Grad coefficients computed by direct Hermite-tensor summation equal the paper's
  expanded formulas in terms of raw moments M_0..M_3 (with the overline read as the sum
  over the distinct index permutations).
"""
import itertools
import math

import numpy as np
import pytest


def _raw_moments(pops, frame, lattice, pmax):
    from oracle import lattice_2d
    cx, cy, _ = lattice_2d(lattice)
    ux, uy, T = frame
    Cx, Cy = math.sqrt(T) * cx + ux, math.sqrt(T) * cy + uy
    return {(p, q): float(np.sum(pops * Cx ** p * Cy ** q))
            for p in range(pmax + 1) for q in range(pmax + 1) if p + q <= pmax}


def _random_case(rng, Q):
    pops = rng.uniform(0.0, 1.0, Q)
    src = (rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(0.2, 3.0))
    dst = (src[0] + rng.uniform(-1.5, 1.5), src[1] + rng.uniform(-1.5, 1.5),
           src[2] * rng.uniform(0.4, 2.5))
    return pops, src, dst


@pytest.mark.parametrize("lattice", [16, 25])
def test_transform_keeps_moments_to_order_3(orc, lattice):
    rng = np.random.default_rng(11)
    for _ in range(20):
        pops, src, dst = _random_case(rng, lattice)
        out = orc.grad_transform(pops, src, dst, lattice)
        m_src = _raw_moments(pops, src, lattice, 3)
        m_dst = _raw_moments(out, dst, lattice, 3)
        scale = max(abs(v) for v in m_src.values())
        for k in m_src:
            assert abs(m_src[k] - m_dst[k]) <= 1e-12 * scale, k


def test_transform_drops_order_4(orc):
    rng = np.random.default_rng(12)
    pops, src, dst = _random_case(rng, 16)
    out = orc.grad_transform(pops, src, dst, 16)
    m_src = _raw_moments(pops, src, 16, 4)
    m_dst = _raw_moments(out, dst, 16, 4)
    assert max(abs(m_src[(p, 4 - p)] - m_dst[(p, 4 - p)]) for p in range(5)) > 1e-3


@pytest.mark.parametrize("lattice", [16, 25])
def test_transform_is_a_projection(orc, lattice):
    rng = np.random.default_rng(13)
    for _ in range(10):
        pops, src, dst = _random_case(rng, lattice)
        once = orc.grad_transform(pops, src, dst, lattice)
        twice = orc.grad_transform(once, dst, dst, lattice)
        assert np.allclose(once, twice, rtol=0, atol=1e-13 * np.abs(once).max())
        # transforming onward to a third frame equals transforming directly
        third = (dst[0] - 0.3, dst[1] + 0.2, dst[2] * 1.3)
        a = orc.grad_transform(once, dst, third, lattice)
        b = orc.grad_transform(pops, src, third, lattice)
        assert np.allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())


def test_equilibrium_is_frame_independent(orc):
    """rho w_i in frame lambda, moved to another frame and back, is rho w_i again
    (its moments to order 3 are those of the same Maxwellian)."""
    _, _, w = orc.lattice_2d(16)
    f = 0.7 * w
    src, dst = (1.2, -0.4, 0.8), (0.3, 0.5, 1.7)
    there = orc.grad_transform(f, src, dst)
    back = orc.grad_transform(there, dst, src)
    assert np.allclose(back, f, rtol=0, atol=1e-14)


def _sym_u_B(u, B):
    """overline(u (x) B) for symmetric rank-2 B: u_a B_bc + u_b B_ac + u_c B_ab."""
    return (np.einsum("a,bc->abc", u, B) + np.einsum("b,ac->abc", u, B)
            + np.einsum("c,ab->abc", u, B))


def test_paper_expanded_coefficients(orc):
    """Sec. III.A.1: a_0 = M_0; a_1 = (M_1 - M_0 u)/sqrt(T);
    a_2 = (M_2 - M_0 T I - sqrt(T) overline(u a_1) - M_0 u u) / T;
    a_3 = (M_3 - T overline(u (M_0 I + a_2)) - T^{3/2} overline(a_1 I)
           - sqrt(T) overline(a_1 u u) - M_0 u u u) / T^{3/2}
    (T_L = 1), with raw moments M_n of the source populations at their own velocities."""
    from oracle import lattice_2d
    rng = np.random.default_rng(14)
    cx, cy, _ = lattice_2d(16)
    I = np.eye(2)
    for _ in range(10):
        pops, src, dst = _random_case(rng, 16)
        C = np.stack([math.sqrt(src[2]) * cx + src[0], math.sqrt(src[2]) * cy + src[1]], 1)
        M0 = pops.sum()
        M1 = np.einsum("j,ja->a", pops, C)
        M2 = np.einsum("j,ja,jb->ab", pops, C, C)
        M3 = np.einsum("j,ja,jb,jc->abc", pops, C, C, C)
        u = np.array(dst[:2])
        T = dst[2]
        sT = math.sqrt(T)
        a1 = (M1 - M0 * u) / sT
        a2 = (M2 - M0 * T * I - sT * (np.outer(u, a1) + np.outer(a1, u)) - M0 * np.outer(u, u)) / T
        a1I = (np.einsum("a,bc->abc", a1, I) + np.einsum("b,ac->abc", a1, I)
               + np.einsum("c,ab->abc", a1, I))
        a1uu = (np.einsum("a,b,c->abc", a1, u, u) + np.einsum("a,b,c->abc", u, a1, u)
                + np.einsum("a,b,c->abc", u, u, a1))
        a3 = (M3 - T * _sym_u_B(u, M0 * I + a2) - T ** 1.5 * a1I - sT * a1uu
              - M0 * np.einsum("a,b,c->abc", u, u, u)) / T ** 1.5
        g0, g1, g2, g3 = orc.grad_coefficients(pops, src, dst)
        scale = max(abs(M0), 1.0)
        assert abs(g0 - M0) <= 1e-13 * scale
        assert np.allclose(g1, a1, rtol=0, atol=1e-11 * scale)
        assert np.allclose(g2, a2, rtol=0, atol=1e-10 * scale)
        assert np.allclose(g3, a3, rtol=0, atol=1e-9 * scale)


def test_grad_reconstruction_contraction(orc):
    """f_i = w_i sum_n a_n : H^(n)(c_i) / n! with the full Frobenius product: on the
    lattice, the reconstructed populations' Hermite moments sum_i f_i H^(n)(c_i) are the
    coefficients a_n again (discrete orthogonality of the Hermite tensors up to n = 3)."""
    from oracle import lattice_2d
    cx, cy, _ = lattice_2d(16)
    rng = np.random.default_rng(15)
    pops, src, dst = _random_case(rng, 16)
    out = orc.grad_transform(pops, src, dst)
    g0, g1, g2, g3 = orc.grad_coefficients(pops, src, dst)
    h0, h1, h2, h3 = orc.grad_coefficients(out, dst, dst)
    for a, b in ((g0, h0), (g1, h1), (g2, h2), (g3, h3)):
        assert np.allclose(a, b, rtol=0, atol=1e-12 * max(1.0, abs(g0)))
    # a_2 and a_3 are symmetric tensors
    assert np.allclose(g2, g2.T, atol=1e-14)
    for perm in itertools.permutations(range(3)):
        assert np.allclose(g3, np.transpose(g3, perm), atol=1e-13)
