"""Strength of the oracle's pins: each case plants one plausible mistake in a
copy of the oracle's C source (on the CPU), builds it, points the oracle's
wrappers at that build, and checks that the named pins reject it.

The mistakes are the slips a restatement of Eq. 1, the leapfrog update, the
source and receivers, the stability limit, the CPML layer and the adjoint
gradient could plausibly contain. A pin set that let one of them through
would not be evidence that the oracle computes the method.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_cpml as cpml_pins
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "wave_oracle.c")

# name: (text in wave_oracle.c, replacement, pins that must fail)
MUTANTS = {
    "last weight mistyped": (
        "-1.0 / 560.0};", "-1.0 / 506.0};",
        [pins.test_weights_match_exact_solve, pins.test_polynomial_exactness_up_to_degree_9]),
    "centre counted twice": (
        "c[0] = ORACLE_W[0] / (2.0 * h * h);", "c[0] = ORACLE_W[0] / (h * h);",
        [pins.test_polynomial_exactness_up_to_degree_9]),
    "y coefficients from dx": (
        "oracle_axis_coeffs(dy, cy);", "oracle_axis_coeffs(dx, cy);",
        [pins.test_polynomial_exactness_up_to_degree_9]),
    "one-sided y neighbour": (
        "oracle_at(u, nx, ny, nz, i, j - m, k, periodic)",
        "oracle_at(u, nx, ny, nz, i, j - m + (m == 4), k, periodic)",
        [pins.test_polynomial_exactness_up_to_degree_9]),
    "Laplacian term subtracted": (
        "unext[p] = 2.0 * u[p] - u_prev[p] + c[p] * lap;",
        "unext[p] = 2.0 * u[p] - u_prev[p] - c[p] * lap;",
        [pins.test_dispersion_relation_exact]),
    "first-order time update": (
        "unext[p] = 2.0 * u[p] - u_prev[p] + c[p] * lap;",
        "unext[p] = u[p] + c[p] * lap;",
        [pins.test_dispersion_relation_exact]),
    "source one step late": (
        "double t = (double)(step0 + s) * dt;", "double t = (double)(step0 + s + 1) * dt;",
        [pins.test_source_first_two_steps_closed_form]),
    "receivers sampled before the update": (
        "traces[(size_t)s * nrec + r] = unext[pr];\n    }\n    /* rotate",
        "traces[(size_t)s * nrec + r] = u[pr];\n    }\n    /* rotate",
        [pins.test_source_first_two_steps_closed_form]),
    "periodic wrap uses the wrong extent": (
        "i = ((i % nx) + nx) % nx;", "i = ((i % nx) + nx) % ny;",
        [pins.test_dispersion_relation_exact]),
    "stability sum without the factor 2": (
        "s += 2.0 * fabs(ORACLE_W[m]);", "s += fabs(ORACLE_W[m]);",
        [pins.test_stability_limit]),
    "Ricker main-lobe factor": (
        "return amp * (1.0 - 2.0 * a) * exp(-a);", "return amp * (1.0 - a) * exp(-a);",
        [pins.test_ricker_closed_form]),
    "gradient without the second time difference": (
        "grad[p] += q2[p] * (a[p] - 2.0 * b[p] + d[p]);", "grad[p] += q2[p] * (a[p] - b[p]);",
        [pins.test_adjoint_gradient_matches_finite_differences]),
    "CPML damping profile linear": (
        "const double d = d0 * xi * xi;", "const double d = d0 * xi;",
        [cpml_pins.test_profile_integral_meets_the_reflection_target]),
    "CPML d0 without the cell size": (
        "const double L = npml * h;", "const double L = npml;",
        [cpml_pins.test_profile_integral_meets_the_reflection_target]),
    "CPML d0 without the profile's factor 3/2": (
        "3.0 * vmax * log(1.0 / R) / (2.0 * L)", "vmax * log(1.0 / R) / L",
        [cpml_pins.test_profile_integral_meets_the_reflection_target]),
    "CPML frequency shift largest at the wall": (
        "const double al = pi * fcps * (1.0 - xi);", "const double al = pi * fcps * xi;",
        [cpml_pins.test_frequency_shift_vanishes_at_the_wall]),
    "CPML convolution weight with the wrong sign": (
        "a[i] = (d + al > 0.0) ? d / (d + al) * (b[i] - 1.0) : 0.0;",
        "a[i] = (d + al > 0.0) ? d / (d + al) * (1.0 - b[i]) : 0.0;",
        [cpml_pins.test_recursive_convolution_is_exact_for_a_step]),
    "CPML decay without the frequency shift": (
        "b[i] = exp(-(d + al) * dt);", "b[i] = exp(-d * dt);",
        [cpml_pins.test_recursive_convolution_is_exact_for_a_step]),
    "CPML psi term with the wrong sign": (
        "sum += d2 + d1p + zeta[ax * n + p];", "sum += d2 - d1p + zeta[ax * n + p];",
        [cpml_pins.test_dense_state_space_brute_force]),
    "CPML adjoint with D1 in place of its transpose": (
        "mu[ax * n + p] = -oracle_d1(g + ax * n,", "mu[ax * n + p] = oracle_d1(g + ax * n,",
        [cpml_pins.test_cpml_adjoint_gradient_matches_finite_differences]),
    "CPML adjoint zeta multiplier without its decay": (
        "if (!last) nu[ax * n + p] = cq + b[ax][idx[ax]] * nu[ax * n + p];",
        "if (!last) nu[ax * n + p] = cq;",
        [cpml_pins.test_cpml_adjoint_gradient_matches_finite_differences]),
    "CPML adjoint psi multiplier term with the wrong sign": (
        "oracle_d1(am + ax * n, nx, ny, nz, i, j, k, ax, hs[ax]);\n            q2[p]",
        "-oracle_d1(am + ax * n, nx, ny, nz, i, j, k, ax, hs[ax]);\n            q2[p]",
        [cpml_pins.test_cpml_adjoint_gradient_matches_finite_differences]),
    "CPML psi from the previous field": (
        "oracle_d1(u, nx, ny, nz, i, j, k, ax, hs[ax]);",
        "oracle_d1(u_prev, nx, ny, nz, i, j, k, ax, hs[ax]);",
        [cpml_pins.test_dense_state_space_brute_force]),
}


def _build_mutant(text, old, new, out_dir):
    assert text.count(old) >= 1, "mutation site not found: %r" % old[:60]
    src = os.path.join(out_dir, "mutant.c")
    lib = os.path.join(out_dir, "libmutant.so")
    with open(src, "w") as f:
        f.write(text.replace(old, new))
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                    "-ffp-contract=off", src, "-o", lib, "-lm"], check=True)
    return lib


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistake(name, tmp_path):
    old, new, targets = MUTANTS[name]
    with open(SRC) as f:
        text = f.read()
    lib = _build_mutant(text, old, new, str(tmp_path))
    oracle._use_library(lib)
    try:
        caught = []
        for pin in targets:
            try:
                pin(oracle)
            except (AssertionError, ValueError):
                caught.append(pin.__name__)
        assert caught, "no pin rejected the mutant %r" % name
    finally:
        oracle._use_library(None)
