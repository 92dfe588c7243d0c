"""Power of the oracle's pins: each plausible mistake below is planted in a copy of
oracle/pond_oracle.c, compiled on the CPU into a separate library, and the pins of the
oracle (the same test functions, called on that library) run cheapest first until one fails.
Every mistake must make at least one pin fail; the test reports which.  The oracle under
test is never modified: the copies live in a temporary directory.

The mistakes cover each part of the step the pins are meant to guard: the Gauss-Hermite
rules of Table I, the Hermite tensors and the Grad reconstruction (Eq. gradGeneralTransform),
the departure points, Lagrange weights and the stencils carried between iterations
(Sec. III.A.2), the BGK relaxation (omega, tau of
Eq. kin_visc), the equilibria and the moment recovery of Sec. II, the collision frame, the
outflow map, and the internal split's source (Eq. int_g_evolution) with its trapezoidal
reading."""
import importlib.util
import os
import subprocess

import numpy as np
import pytest

import test_oracle_lattice as TL
import test_oracle_nt as TN
import test_oracle_physics as TP
import test_oracle_step as TS
import test_oracle_transform as TT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pond_oracle.c")

# (name, text in the oracle, planted replacement); each text occurs exactly once
MISTAKES = [
    ("D1Q4 outer weight perturbed",
     "wout = (3.0 - sqrt(6.0)) / 12.0;", "wout = (3.0 - sqrt(6.0)) / 12.1;"),
    ("D1Q4 weights swapped",
     "w[0] = wout;  w[1] = win;  w[2] = win; w[3] = wout;\n        return 4;",
     "w[0] = win;  w[1] = wout;  w[2] = wout; w[3] = win;\n        return 4;"),
    ("rank-3 Hermite tensor misses a term",
     "- xi[a] * kron(b, g) - xi[b] * kron(a, g) - xi[g] * kron(a, b);",
     "- xi[a] * kron(b, g) - xi[b] * kron(a, g);"),
    ("third-order Grad term dropped",
     "s2 / 2.0 + s3 / 6.0", "s2 / 2.0 + 0.0 * s3 / 6.0"),
    ("departure point reversed",
     "double xd = (double)x - Cx * 1.0", "double xd = (double)x + Cx * 1.0"),
    ("cubic Lagrange weight wrong",
     "wts[1] = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;", "wts[1] = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.1;"),
    ("omega = 1/tau",
     "double omega = 1.0 / (tau + 0.5);\n    for (int i = 0; i < L->Q; ++i) {",
     "double omega = 1.0 / tau;\n    for (int i = 0; i < L->Q; ++i) {"),
    ("tau = mu/T",
     "double tau = cfg->mu / (rho * m.T);", "double tau = cfg->mu / m.T;"),
    ("kinetic energy of g_eq doubled",
     "kin = 0.5 * (Cx * Cx + Cy * Cy);", "kin = (Cx * Cx + Cy * Cy);"),
    ("temperature recovery keeps the whole kinetic energy",
     "m.T = (G / rho - 0.5 * u2) / cv;", "m.T = (G / rho - u2) / cv;"),
    ("collision in the streaming frame, not the frame of the moments",
     "grad_coefficients(L, P, 1, grad_order_of(cfg), bar, star, &Af);",
     "grad_coefficients(L, P, 1, grad_order_of(cfg), bar, bar, &Af);"),
    ("outflow wraps around",
     "    if (j < 0) return 0;        /* outflow", "    if (j < 0) return n - 1;    /* outflow"),
    ("internal split: sign of G",
     "double Gi = -rho1 * L->w[i]", "double Gi = rho1 * L->w[i]"),
    ("internal split: full G instead of (1 - omega/2) G",
     "                        1.0 - 0.5 * omega);", "                        1.0 + 0.0 * omega);"),
    ("internal split: U without the half source",
     "m.T = G / (rho * (cv + 0.5 * div));", "m.T = G / (rho * cv);"),
    ("3-point Lagrange middle weight wrong",
     "wts[1] = (1.0 - t) * (1.0 + t);", "wts[1] = (1.0 - t) * (1.0 + 0.9 * t);"),
    ("g_eq's internal energy with c_v instead of c_v - 1 (D = 2)",
     "double Uprime_over_rho = (cv - 1.0) * fr.T;", "double Uprime_over_rho = cv * fr.T;"),
    ("stencils chosen again at every iteration",
     "return order == 3 ? (t >= -0.25 && t < 1.25) : (t >= -0.75 && t < 0.75);", "return 0;"),
    ("internal split: initial state g_eq - G/2",
     "node_source(cfg, &L, g, x, y, ux, uy, T[n], rho[n], 0.0, 0.0, 0.5);",
     "node_source(cfg, &L, g, x, y, ux, uy, T[n], rho[n], 0.0, 0.0, -0.5);"),
]

# The oracle's pins, cheapest first: (name, call on an oracle module).
PINS = [
    ("lattice matches Table I", lambda o: (TL.test_lattice_matches_table1(o, 4, "D1Q4"),
                                          TL.test_lattice_matches_table1(o, 5, "D1Q5"))),
    ("quadrature exactness", lambda o: (TL.test_quadrature_exactness(o, 4, 7), TL.test_quadrature_exactness(o, 5, 9))),
    ("equilibria return their moments", lambda o: [TL.test_equilibrium_returns_its_moments(o, s, q)
                                                   for s in ("total", "internal") for q in (16, 25)]),
    ("g_eq moments exact", lambda o: [TL.test_geq_moments_exact(o, s) for s in ("total", "internal")]),
    ("transform keeps moments to order 3", lambda o: [TT.test_transform_keeps_moments_to_order_3(o, q)
                                                      for q in (16, 25)]),
    ("transform is a projection", lambda o: [TT.test_transform_is_a_projection(o, q) for q in (16, 25)]),
    ("paper's expanded coefficients", lambda o: TT.test_paper_expanded_coefficients(o)),
    ("interpolation reproduces polynomials", lambda o: [TS.test_interpolation_reproduces_polynomials(o, 3, 3),
                                                        TS.test_interpolation_reproduces_polynomials(o, 2, 2)]),
    ("collision conserves per node", lambda o: [TS.test_collision_conserves_per_node(o, s)
                                                for s in ("total", "internal")]),
    ("uniform supersonic flow stays uniform", lambda o: [TS.test_uniform_supersonic_flow_stays_uniform(o, q, s)
                                                         for q in (16, 25) for s in ("total", "internal")]),
    ("predictor-corrector fixed point", lambda o: TS.test_predictor_corrector_fixed_point(o)),
    ("conservation drift is second order", lambda o: TS.test_conservation_drift_is_second_order(o)),
    ("kept stencils let the iteration converge", lambda o: TS.test_kept_stencils_let_the_iteration_converge(o)),
    ("internal split: pdV work", lambda o: TP.test_internal_split_source_is_pdv_work(o)),
    ("Sod vs the exact Riemann solution", lambda o: TP.test_sod_matches_exact_riemann(o)),
    ("sound speed", lambda o: TP.test_sound_speed(o, 1.4)),
    ("shear-wave decay", lambda o: TP.test_shear_wave_decay_rate(o, 0.0)),
    ("sound attenuation, internal split", lambda o: TN.test_sound_attenuation_gives_the_bulk_viscosity(
        o, "internal", 16, 1.4)),
    ("entropy-wave decay", lambda o: [TP.test_thermal_wave_decay_rate(o, s) for s in ("total", "internal")]),
]


def _oracle_from(source_text, workdir, tag):
    """A separate instance of the oracle package bound to a library built from source_text."""
    src = os.path.join(workdir, "pond_oracle_%s.c" % tag)
    so = os.path.join(workdir, "liboracle_%s.so" % tag)
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    src, "-o", so, "-lm"], check=True)
    spec = importlib.util.spec_from_file_location(
        "oracle_planted_%s" % tag, os.path.join(ROOT, "oracle", "__init__.py"),
        submodule_search_locations=[os.path.join(ROOT, "oracle")])
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build = lambda *a, **k: so
    mod._lib = None
    return mod


def _first_failing_pin(mod):
    with np.errstate(all="ignore"):
        for name, pin in PINS:
            try:
                pin(mod)
            except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError):
                return name
    return None


def test_unmodified_oracle_passes_the_pin_list(tmp_path):
    """The pin list itself holds on the oracle as it stands (built the same way)."""
    mod = _oracle_from(open(SRC).read(), str(tmp_path), "clean")
    assert _first_failing_pin(mod) is None


@pytest.mark.parametrize("name,old,new", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, "the planted text must occur exactly once: %r" % old
    mod = _oracle_from(text.replace(old, new), str(tmp_path), "planted")
    failed = _first_failing_pin(mod)
    print("%s -> fails: %s" % (name, failed))
    assert failed is not None, "no pin caught: " + name
