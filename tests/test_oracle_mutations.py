"""Planted mistakes: each mutation below is a plausible slip in oracle.c (a
dropped term, a flipped sign, a conjugate on the wrong index, a wrong mass
splitting, quadrature or chi^2 formula).  A copy of the oracle with that one
mistake is compiled on the CPU and the pin tests are run against it: at least
one pin must fail for every mutant."""
import inspect
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")

MUTATIONS = {
    "drop_im_term": ("P += -4.0 * creal(X) * sx * sx + 2.0 * cimag(X) * sin(2.0 * x);",
                     "P += -4.0 * creal(X) * sx * sx;"),
    "re_term_sign": ("P += -4.0 * creal(X) * sx * sx", "P += 4.0 * creal(X) * sx * sx"),
    "conj_wrong_index": ("conj(V[a][i]) * V[b][i] * V[a][j] * conj(V[b][j])",
                         "V[a][i] * conj(V[b][i]) * V[a][j] * conj(V[b][j])"),
    "antineutrino_not_conjugated": ("anti ? conj(U[r][c]) : U[r][c]", "U[r][c]"),
    "dm31_wrong": ("double m2[3] = {0.0, dm21, dm21 + dm32};\n    double P", "double m2[3] = {0.0, dm21, dm32};\n    double P"),
    "half_phase_factor": ("return dm2_eV2 * L_inv_eV / (4.0 * E_eV);", "return dm2_eV2 * L_inv_eV / (2.0 * E_eV);"),
    "pmns_r13_sign": ("{-s13 * ep, 0, c13}", "{s13 * ep, 0, c13}"),
    "legendre_recurrence_sign": ("((2.0 * j + 1.0) * x * p1 - j * p0)", "((2.0 * j + 1.0) * x * p1 + j * p0)"),
    "gl_weight_factor": ("w[n - k] = 2.0 /", "w[n - k] = 1.0 /"),
    "bin_half_width": ("double wt = half * w[k] * or_spectrum(E, e_scale);", "double wt = w[k] * or_spectrum(E, e_scale);"),
    "bin_midpoint": ("double half = 0.5 * (b - a), mid = 0.5 * (a + b);", "double half = 0.5 * (b - a), mid = a;"),
    "spectrum_coefficient": ("exp(0.87 - 0.16 * E - 0.091 * E * E)", "exp(0.87 - 0.16 * E + 0.091 * E * E)"),
    "pearson_denominator": ("term = (d - m) * (d - m) / m;", "term = (d - m) * (d - m) / d;"),
    "poisson_log_inverted": ("d * log(d / m)", "d * log(m / d)"),
    "nuisance_dropped": ("double m = N * (1.0 + e) * M;", "double m = N * M;"),
    "baseline_weight_index": ("M += omega[r] * mu_rb[(int64_t)r * nbins + i];", "M += omega[0] * mu_rb[(int64_t)r * nbins + i];"),
    "grad_product_rule_half": ("g12 -= 4.0 * (due_ds12[i] * ue[j] + ue[i] * due_ds12[j]) * s2;",
                               "g12 -= 4.0 * (due_ds12[i] * ue[j]) * s2;"),
    "grad_dm21_chain": ("double dm2_d21[3] = {0.0, 1.0, 1.0};", "double dm2_d21[3] = {0.0, 1.0, 0.0};"),
    "penalty_sigma": ("chi2 += eta[i] * eta[i] / (sigma * sigma);", "chi2 += eta[i] * eta[i] / sigma;"),
    "dU_delta_sign": ("double complex Dd[3][3] = {{0, 0, -I * s13 * em}", "double complex Dd[3][3] = {{0, 0, I * s13 * em}"),
    "dU_not_conjugated_for_antineutrinos": ("dV[q][r][c] = anti ? conj(dU[q][r][c]) : dU[q][r][c];",
                                            "dV[q][r][c] = dU[q][r][c];"),
    "dU_s23_cos_sign": ("double ds23 = 0.5 / s23, dc23 = -0.5 / c23;", "double ds23 = 0.5 / s23, dc23 = 0.5 / c23;"),
    "general_grad_product_rule_term": ("conj(V[a][i]) * V[b][i] * dV[q][a][j] * conj(V[b][j]) +\n", ""),
    "general_grad_im_term_dm": ("double dterm_dx = -4.0 * creal(X) * s2x + 4.0 * cimag(X) * c2x;",
                                "double dterm_dx = -4.0 * creal(X) * s2x + 2.0 * cimag(X) * c2x;"),
    "general_binned_baseline_index": ("prob_general_grad(alpha, beta, U, dU, osc6[4], osc6[5], L_km[r], E, anti, &P, dP);",
                                      "prob_general_grad(alpha, beta, U, dU, osc6[4], osc6[5], L_km[0], E, anti, &P, dP);"),
    "general_delta_ab_dropped": ("double p = (a == b) ? 1.0 : 0.0;", "double p = 0.0;"),
    "general_grad_dm32_chain": ("dP[5] += dterm_dx * dx * (dm2_d32[i] - dm2_d32[j]);",
                                "dP[5] += dterm_dx * dx * (dm2_d21[i] - dm2_d21[j]);"),
}


def pin_calls():
    """Every pin test with the parameters it is collected with (first values)."""
    calls = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        marks = getattr(fn, "pytestmark", [])
        params = {}
        for m in marks:
            if m.name == "parametrize":
                argnames = [a.strip() for a in m.args[0].split(",")]
                values = m.args[1]
                for v in values[:2]:
                    v = v if isinstance(v, tuple) else (v,)
                    calls.append((name, fn, dict(zip(argnames, v))))
                params = None
        if params is not None and not any(m.name == "parametrize" for m in marks):
            calls.append((name, fn, {}))
    return calls


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


@pytest.mark.slow
@pytest.mark.parametrize("mut", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(mut, source, tmp_path):
    old, new = MUTATIONS[mut]
    assert source.count(old) >= 1, "mutation anchor not found: %s" % mut
    src = tmp_path / "oracle_mut.c"
    src.write_text(source.replace(old, new, 1))
    lib = tmp_path / "liboracle_mut.so"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", str(src), "-o", str(lib), "-lm"]
    r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True)
    if r.returncode != 0:
        subprocess.run(cmd, check=True, capture_output=True)
    caught = []
    with oracle.use_library(str(lib)):
        for name, fn, kw in pin_calls():
            try:
                fn(**kw)
            except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError) as e:
                caught.append(name)
                break
    assert caught, "no pin failed for mutation %s" % mut
