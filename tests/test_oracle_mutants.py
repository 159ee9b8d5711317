"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
the pins of ``test_oracle_pins.py`` reject every one of them."""
import numpy as np
import pytest

import oracle
import test_oracle_pins as P

MUTANTS = {
    # Eq. 1: the |m| term dropped from the exponent of the last factor
    "drop_m_in_power": [("2.0 * nstar - (double)am - 1.0);", "2.0 * nstar - 1.0);")],
    # Eq. 1: the cycle-averaging square root lost
    "drop_sqrt_factor": [(
        "model == 1 ? 1.0 : sqrt(3.0 * pow(nstar, 3.0) * E / (M_PI * pow(q, 3.0) * E_a));",
        "1.0;")],
    # static-field model: the cycle-averaging factor kept
    "static_keeps_sqrt": [("model == 1 ? 1.0 :", "model == 2 ? 1.0 :")],
    # Eq. 1: the n*-dependent prefactors, each with one power of n* lost
    "q2_over_2nstar": [("(q * q) / (2.0 * nstar * nstar)", "(q * q) / (2.0 * nstar)")],
    "flm_divisor_no_nstar": [("(2.0 * M_PI * nstar * pow(2.0, (double)am)",
                              "(2.0 * M_PI * pow(2.0, (double)am)")],
    "sqrt_nstar_squared": [("sqrt(3.0 * pow(nstar, 3.0) * E / (M_PI * pow(q, 3.0) * E_a))",
                            "sqrt(3.0 * pow(nstar, 2.0) * E / (M_PI * pow(q, 3.0) * E_a))")],
    # Eq. 1: (2e/n*)^(2n*) with the wrong exponent
    "power_2e_nstar": [("pow(2.0 * e / nstar, 2.0 * nstar)", "pow(2.0 * e / nstar, nstar)")],
    # Eq. 1: (l-|m|)! in the f(l,m) divisor replaced by l!
    "flm_l_minus_m": [("or_factorial(am) *\n           or_factorial(l - am))",
                       "or_factorial(am) *\n           or_factorial(l))")],
    # Eq. 1: sign of the tunnelling exponent
    "exponent_sign": [("      exp(-expo) *", "      exp(expo) *")],
    # Eq. 1: Q taken as the charge before ionization
    "charge_before": [("      const double Wk = or_adk_rate(E[c], U[k], l[k], m[k], k + 1, consts);",
                       "      const double Wk = or_adk_rate(E[c], U[k], l[k], m[k], k + 2, consts);")],
    # Eq. 3: the rate matrix transposed (gain written above the diagonal)
    "transposed_matrix": [("      A[(i + 1) * w + i] = Wk * dt;", "      A[i * w + (i + 1)] = Wk * dt;")],
    # exp: diagonal reset one squaring behind
    "stale_diagonal": [("X[i * n + i] = exp(ldexp(B[i * n + i], r));",
                        "X[i * n + i] = exp(ldexp(B[i * n + i], r - 1));")],
    # dn_e: electrons counted with the wrong sign (an index offset would not be
    # a mistake: sum_k (N'_k - N_k) = 0, so sum_k (k + c)(N'_k - N_k) is the same)
    "dne_sign": [("d += (double)(a + i) * (n1[i] - n0[i]);",
                  "d += (double)(a + i) * (n0[i] - n1[i]);")],
    # dn_e: the initial populations left out
    "dne_no_initial": [("d += (double)(a + i) * (n1[i] - n0[i]);",
                        "d += (double)(a + i) * n1[i];")],
    # window update: slides past the top state
    "slide_past_top": [("shifts < w - 1 && nb < Z &&", "shifts < w - 1 && nb <= Z &&")],
    # adaptive window: grows one state past w_max
    "grow_past_wmax": [("nb < Z && nb - na + 1 < wmax) ++nb;", "nb < Z && nb - na + 1 <= wmax) ++nb;")],
    # adaptive window: drops the bottom below w_min instead of sliding
    "shrink_below_wmin": [("if (nb - na + 1 > wmin) {", "if (nb - na + 1 >= wmin) {")],
}

PIN_TESTS = [
    (P.test_adk_hydrogen_closed_form, (510.0,)),
    (P.test_adk_hydrogenic_ion_closed_form, (1500.0,)),
    (P.test_adk_nstar_two_closed_form, (400.0, 0)),
    (P.test_adk_nstar_two_closed_form, (400.0, 1)),
    (P.test_adk_nstar_two_d_state_closed_form, (900.0, 1, 0)),
    (P.test_adk_f_state_m_two_closed_form, (2000.0,)),
    (P.test_adk_m_projection_ratio, (2, 300.0)),
    (P.test_adk_log_slope, (1, 800.0)),
    (P.test_adk_static_hydrogen_landau_lifshitz, (300.0,)),
    (P.test_expm_vs_arbitrary_precision, ([13.7, 49.7, 191.9, 142.6, 290.4],)),
    (P.test_expm_vs_arbitrary_precision, ([2500.0, 0.2, 1e-30, 7.0],)),
    (P.test_paper_four_level_solution, ((0.9, 2.7, 0.05),)),
    (P.test_step_four_level_matches_paper, ()),
    (P.test_step_single_level_closed_form, ()),
    (P.test_window_update_rules, ()),
    (P.test_adaptive_window_rules, ()),
]


def run_pins(lib):
    """Names of the pins that fail when the oracle is ``lib``."""
    failed = []
    saved = oracle._lib
    oracle._lib = lib
    try:
        for fn, args in PIN_TESTS:
            try:
                with np.errstate(all="ignore"):
                    fn(*args)
            except (AssertionError, ValueError, ZeroDivisionError, OverflowError):
                failed.append(fn.__name__)
            except pytest.skip.Exception:
                pass
    finally:
        oracle._lib = saved
    return failed


def test_unmodified_oracle_passes_the_pins():
    assert run_pins(oracle.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    lib = oracle.build_variant(MUTANTS[name], name)
    failed = run_pins(lib)
    assert failed, f"mutant {name} passed every pin"
