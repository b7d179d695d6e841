"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them (the mistakes go into a temporary build of the oracle
source on the CPU; the real oracle is untouched)."""
import numpy as np
import pytest

import tests.test_oracle_pins as pins

MUTATIONS = {
    # wrong sign of the analysis exponent (e^{+i m lambda})
    "dft_sign": ("im -= g[k] * sn[t];", "im += g[k] * sn[t];"),
    # Condon-Shortley phase slipped into the sectoral seed
    "cs_phase": ("if (m > 0) pmm = sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm;",
                 "if (m > 0) pmm = -sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm;"),
    # weight without the square of the derivative
    "weight": ("double wj = 2.0 / ((1.0 - x * x) * dp * dp);",
               "double wj = 2.0 / ((1.0 - x * x) * dp * fabs(dp) * 1.0000001);"),
    # dropped factor 2 for the m > 0 conjugate pair in the synthesis
    "synth_factor": ("v += 2.0 * (F[2 * m] * cs[t] - F[2 * m + 1] * sn[t]);",
                     "v += (F[2 * m] * cs[t] - F[2 * m + 1] * sn[t]);"),
    # transposed re/im product in the synthesis
    "synth_sign": ("v += 2.0 * (F[2 * m] * cs[t] - F[2 * m + 1] * sn[t]);",
                   "v += 2.0 * (F[2 * m] * cs[t] + F[2 * m + 1] * sn[t]);"),
    # wrong index in the second recurrence coefficient
    "recur_b": ("double b = sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) /",
                "double b = sqrt(((double)n * n - (double)m * m) /"),
    # Nyquist mode kept on a row
    "row_trunc": ("int mj = (nj - 1) / 2;", "int mj = nj / 2;"),
    # quadrature weight dropped in the analysis
    "no_weight": ("double fr = w[j] * F[2 * m], fi = w[j] * F[2 * m + 1];",
                  "double fr = F[2 * m], fi = F[2 * m + 1];"),
    # derivative relation: wrong sign of the Pbar_{n+1} term
    "deriv_sign": ("H[spec_index(T, m, n)] = (n + 1.0) * eps_nm(n, m) * pm1 - (double)n * eps_nm(n + 1, m) * pp1;",
                   "H[spec_index(T, m, n)] = (n + 1.0) * eps_nm(n, m) * pm1 + (double)n * eps_nm(n + 1, m) * pp1;"),
    # derivative relation: eps index off by one
    "deriv_eps": ("H[spec_index(T, m, n)] = (n + 1.0) * eps_nm(n, m) * pm1 - (double)n * eps_nm(n + 1, m) * pp1;",
                  "H[spec_index(T, m, n)] = (n + 1.0) * eps_nm(n + 1, m) * pm1 - (double)n * eps_nm(n, m) * pp1;"),
    # d/dlambda as -i m instead of i m
    "dlam_sign": ("g[2 * m] = -(double)m * pi;", "g[2 * m] = (double)m * pi;"),
    # wind: V built with the wrong sign of the chi term
    "wind_sign": ("V[i] += a[i];", "V[i] -= a[i];"),
    # vorticity analysis without the 1 / (1 - mu^2) factor
    "vordiv_cos": ("double c = w[j] / ((1.0 - mu[j]) * (1.0 + mu[j]));", "double c = w[j];"),
    # spectral index with m and n swapped in the triangle offset
    "spec_index": ("return (long)m * (T + 1) - (long)m * (m - 1) / 2 + (n - m);",
                   "return (long)m * (T + 1) - (long)m * (m + 1) / 2 + (n - m);"),
}

PIN_CALLS = [
    lambda o: pins.test_weights_sum_to_two(o, 32),
    lambda o: pins.test_gauss_closed_forms(o),
    lambda o: pins.test_low_degree_closed_forms(o),
    lambda o: pins.test_discrete_orthonormality(o, 31, 32),
    lambda o: pins.test_dft_stage_matches_numpy_rfft(o),
    lambda o: pins.test_synthesis_stage_matches_numpy_irfft(o),
    lambda o: pins.test_single_mode(o, 3, 7, 1j),
    lambda o: pins.test_round_trip_regular(o, 15),
    lambda o: pins.test_parseval_regular(o),
    lambda o: pins.test_derivative_closed_forms(o, 0.41),
    lambda o: pins.test_derivative_values_match_finite_differences(o, 0.05),
    lambda o: pins.test_derivative_synthesis_matches_finite_differences(o),
    lambda o: pins.test_solid_body_rotation(o),
    lambda o: pins.test_wind_round_trip(o, 15, 16),
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(oracle_mod, tmp_path, name):
    old, new = MUTATIONS[name]
    src = oracle_mod.source_text()
    assert src.count(old) == 1, name
    lib = oracle_mod.build_variant(src.replace(old, new), str(tmp_path / f"lib_{name}.so"))
    caught = 0
    with oracle_mod.use_library(lib):
        for call in PIN_CALLS:
            try:
                call(oracle_mod)
            except (AssertionError, RuntimeError, IndexError, ValueError, FloatingPointError):
                caught += 1
    assert caught >= 1, f"no pin caught the planted mistake {name}"
    # and the real oracle passes every one of them
    for call in PIN_CALLS:
        call(oracle_mod)
