"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against what the paper or the mathematics fixes:
hand-reduced closed forms of Eq. 1, the paper's explicit reduced solutions
(Eqs. 6-9, with the sign typos of Eqs. 7 and 9 corrected), confluent
(equal-rate) closed forms, an arbitrary-precision matrix exponential
(mpmath), a brute-force RK4 integration, and invariants (conservation,
non-negativity, semigroup, identity at dt = 0).  ``test_oracle_mutants.py``
plants mistakes in a copy of the oracle and shows these pins catch them.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle

OMEGA_A, E_A, U_H = oracle.PAPER_CONSTANTS
# Nitrogen, Z = 7: U_k (eV) of the state k -> k+1 and its l (m = 0 for all).
N2_U = [14.53, 29.60, 47.45, 77.47, 97.89, 552.07, 667.05]
N2_L = [1, 1, 1, 0, 0, 0, 0]


# --------------------------------------------------------------------------
# Eq. 1
# --------------------------------------------------------------------------
@pytest.mark.parametrize("l,m,expect", [
    (0, 0, 1), (1, 0, 3), (1, 1, 3), (1, -1, 3), (2, 0, 5), (2, 1, 15),
    (2, 2, 15), (3, 1, 42), (3, 3, 105)])
def test_flm_small_integers(l, m, expect):
    # (2l+1)(l+|m|)! / (2^|m| |m|! (l-|m|)!) worked by hand
    assert oracle.flm(l, m) == expect


@pytest.mark.parametrize("E", [30.0, 120.0, 510.0, 2000.0, 9000.0])
def test_adk_hydrogen_closed_form(E):
    # Q = 1, U = U_H, l = m = 0  =>  n* = 1, and Eq. 1 reduces by hand to
    # W = w_a sqrt(3E/(pi E_a)) (2 e^2 / pi) (E_a/E) exp(-2 E_a / (3E)).
    want = (OMEGA_A * math.sqrt(3 * E / (math.pi * E_A)) * (2 * math.e ** 2 / math.pi)
            * (E_A / E) * math.exp(-2 * E_A / (3 * E))) * 1e-15
    got = oracle.adk_rate(E, U_H, 0, 0, 1)
    assert got == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("E", [200.0, 1500.0, 7000.0])
def test_adk_hydrogenic_ion_closed_form(E):
    # Q = 2, U = 4 U_H  =>  n* = 1 again; Eq. 1 reduces to
    # W = w_a sqrt(3E/(8 pi E_a)) (64 e^2 / pi) (E_a/E) exp(-16 E_a / (3E)).
    want = (OMEGA_A * math.sqrt(3 * E / (8 * math.pi * E_A)) * (64 * math.e ** 2 / math.pi)
            * (E_A / E) * math.exp(-16 * E_A / (3 * E))) * 1e-15
    got = oracle.adk_rate(E, 4 * U_H, 0, 0, 2)
    assert got == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("E", [60.0, 400.0, 3000.0])
def test_adk_nstar_two_closed_form(E, model):
    # Q = 1, U = U_H/4, l = m = 0  =>  n* = 2, where every power of n* in
    # Eq. 1 counts.  Term by term:
    #   sqrt(3 n*^3 E/(pi Q^3 E_a)) = sqrt(24 E/(pi E_a))
    #   Q^2/(2 n*^2)                = 1/8
    #   (2e/n*)^(2n*)               = e^4
    #   f(0,0)/(2 pi n*)            = 1/(4 pi)
    #   (2 E_a Q^3/(E n*^3))^(2n*-1) = (E_a/(4E))^3
    #   exp(-(2/3)(Q/n*)^3 E_a/E)    = exp(-E_a/(12 E))
    # so W = w_a sqrt(24E/(pi E_a)) e^4/(2048 pi) (E_a/E)^3 exp(-E_a/(12E));
    # the static-field model (model 1) drops the square root.
    cyc = 1.0 if model == 1 else math.sqrt(24 * E / (math.pi * E_A))
    want = (OMEGA_A * cyc * math.e ** 4 / (2048 * math.pi) * (E_A / E) ** 3
            * math.exp(-E_A / (12 * E))) * 1e-15
    got = oracle.adk_rate(E, U_H / 4, 0, 0, 1, model=model)
    assert got == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("m", [1, -1])
@pytest.mark.parametrize("E", [150.0, 900.0, 5000.0])
def test_adk_nstar_two_d_state_closed_form(E, m, model):
    # Q = 2, U = U_H, l = 2, |m| = 1  =>  n* = 2 and f(2,1) = 15.  Term by
    # term:
    #   sqrt(3 n*^3 E/(pi Q^3 E_a)) = sqrt(3 E/(pi E_a))
    #   Q^2/(2 n*^2)                = 1/2
    #   (2e/n*)^(2n*)               = e^4
    #   f(2,1)/(2 pi n*)            = 15/(4 pi)
    #   (2 E_a Q^3/(E n*^3))^(2n*-|m|-1) = (2 E_a/E)^2
    #   exp(-(2/3)(Q/n*)^3 E_a/E)    = exp(-2 E_a/(3 E))
    # so W = w_a sqrt(3E/(pi E_a)) (15 e^4/(2 pi)) (E_a/E)^2 exp(-2E_a/(3E)).
    cyc = 1.0 if model == 1 else math.sqrt(3 * E / (math.pi * E_A))
    want = (OMEGA_A * cyc * 15 * math.e ** 4 / (2 * math.pi) * (E_A / E) ** 2
            * math.exp(-2 * E_A / (3 * E))) * 1e-15
    got = oracle.adk_rate(E, U_H, 2, m, 2, model=model)
    assert got == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("E", [300.0, 2000.0])
def test_adk_f_state_m_two_closed_form(E):
    # Q = 3, U = 9 U_H/4, l = 3, |m| = 2  =>  n* = 3/(3/2) = 2, f(3,2) =
    # 7 * 5! / (4 * 2! * 1!) = 105.  Term by term:
    #   sqrt(3 n*^3 E/(pi Q^3 E_a)) = sqrt(24 E/(27 pi E_a)) = sqrt(8E/(9 pi E_a))
    #   Q^2/(2 n*^2)                = 9/8
    #   (2e/n*)^(2n*)               = e^4
    #   f/(2 pi n*)                 = 105/(4 pi)
    #   (2 E_a Q^3/(E n*^3))^(2n*-|m|-1) = (27 E_a/(4 E))^1
    #   exp(-(2/3)(Q/n*)^3 E_a/E)    = exp(-(2/3)(27/8) E_a/E) = exp(-9 E_a/(4E))
    want = (OMEGA_A * math.sqrt(8 * E / (9 * math.pi * E_A)) * (9 / 8) * math.e ** 4
            * 105 / (4 * math.pi) * (27 * E_A / (4 * E)) * math.exp(-9 * E_A / (4 * E))) * 1e-15
    for m in (2, -2):
        got = oracle.adk_rate(E, 9 * U_H / 4, 3, m, 3)
        assert got == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("k", range(7))
@pytest.mark.parametrize("E", [300.0, 2500.0])
def test_adk_m_projection_ratio(k, E):
    # For l = 1: f(1,1) = f(1,0), so W(m=1)/W(m=0) is the extra power of the
    # last factor of Eq. 1: (2 E_a Q^3 / (E n*^3))^(-1).
    Q = k + 1
    ns = Q * math.sqrt(U_H / N2_U[k])
    want = (E * ns ** 3) / (2 * E_A * Q ** 3)
    r = oracle.adk_rate(E, N2_U[k], 1, 1, Q) / oracle.adk_rate(E, N2_U[k], 1, 0, Q)
    assert r == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("k", range(7))
@pytest.mark.parametrize("E", [150.0, 800.0, 4000.0])
def test_adk_log_slope(k, E):
    # d ln W / d ln E = -(2n* - |m| - 3/2) + (2/3)(Q/n*)^3 E_a/E  (by hand from
    # Eq. 1), checked by a central difference of the oracle.
    Q = k + 1
    ns = Q * math.sqrt(U_H / N2_U[k])
    want = -(2 * ns - 1.5) + (2.0 / 3.0) * (Q / ns) ** 3 * E_A / E
    h = 1e-5
    w1 = oracle.adk_rate(E * math.exp(h), N2_U[k], N2_L[k], 0, Q)
    w0 = oracle.adk_rate(E * math.exp(-h), N2_U[k], N2_L[k], 0, Q)
    if w1 <= 0 or w0 <= 0:
        pytest.skip("rate underflows at this field")
    got = (math.log(w1) - math.log(w0)) / (2 * h)
    assert got == pytest.approx(want, rel=1e-6, abs=1e-6)


@pytest.mark.parametrize("E", [300.0, 1000.0, 4000.0])
def test_adk_static_hydrogen_landau_lifshitz(E):
    # Static-field model (Eq. 1 without its cycle-averaging factor), Q = 1,
    # U = U_H, l = m = 0: by hand W = w_a (2e^2/pi)(E_a/E) exp(-2E_a/(3E)).
    # The textbook static-field rate of the hydrogen ground state (Landau &
    # Lifshitz, Quantum Mechanics, Sec. 77) is 4 w_a (E_a/E) exp(-2E_a/(3E))
    # in atomic units.  Eq. 1's coefficient (2e/n*)^(2n*)/(2 pi n*) ... gives
    # 2e^2/pi in place of the exact 4, so the two differ by e^2/(2 pi).
    ll = 4 * OMEGA_A * (E_A / E) * math.exp(-2 * E_A / (3 * E)) * 1e-15
    got = oracle.adk_rate(E, U_H, 0, 0, 1, model=oracle.ADK_STATIC)
    assert got / ll == pytest.approx(math.e ** 2 / (2 * math.pi), rel=1e-13)


@pytest.mark.parametrize("k", [0, 3, 6])
@pytest.mark.parametrize("E", [800.0, 3000.0])
def test_adk_static_log_slope(k, E):
    # Without the factor sqrt(3 n*^3 E/(pi Q^3 E_a)) the slope loses 1/2:
    # d ln W / d ln E = -(2n* - |m| - 1) + (2/3)(Q/n*)^3 E_a/E.
    Q = k + 1
    ns = Q * math.sqrt(U_H / N2_U[k])
    want = -(2 * ns - 1.0) + (2.0 / 3.0) * (Q / ns) ** 3 * E_A / E
    h = 1e-5
    st = oracle.ADK_STATIC
    w1 = oracle.adk_rate(E * math.exp(h), N2_U[k], N2_L[k], 0, Q, model=st)
    w0 = oracle.adk_rate(E * math.exp(-h), N2_U[k], N2_L[k], 0, Q, model=st)
    if w1 <= 0 or w0 <= 0:
        pytest.skip("rate underflows at this field")
    got = (math.log(w1) - math.log(w0)) / (2 * h)
    assert got == pytest.approx(want, rel=1e-6, abs=1e-6)


def test_adk_cutoffs_and_units():
    # Zero field and fields whose exponent exceeds 700 give W = 0.
    assert oracle.adk_rate(0.0, 14.53, 1, 0, 1) == 0.0
    assert oracle.adk_rate(1e-7, 14.53, 1, 0, 1) == 0.0
    assert oracle.adk_rate(0.5, 552.07, 0, 0, 6) == 0.0
    # |E| is used: the sign of a field component does not matter.
    assert oracle.adk_rate(-700.0, 14.53, 1, 0, 1) == oracle.adk_rate(700.0, 14.53, 1, 0, 1)
    # units: omega_a = 4.13e16 1/s = 41.3 1/fs.  For n* = 1 at E = E_a the
    # hand value is 41.3 sqrt(3/pi) (2e^2/pi) e^(-2/3) 1/fs.
    want = 41.3 * math.sqrt(3 / math.pi) * 2 * math.e ** 2 / math.pi * math.exp(-2 / 3)
    assert oracle.adk_rate(E_A, U_H, 0, 0, 1) == pytest.approx(want, rel=1e-13)


# --------------------------------------------------------------------------
# exp of the window matrix (Eqs. 3-5)
# --------------------------------------------------------------------------
def window_matrix(lam):
    """dt*A for a window with rates lam (len w-1); the top state absorbs."""
    w = len(lam) + 1
    A = np.zeros((w, w))
    for i, x in enumerate(lam):
        A[i, i] = -x
        A[i + 1, i] = x
    return A


def mp_expm(A, dps=50):
    with mpmath.workdps(dps):
        M = mpmath.matrix(A.tolist())
        X = mpmath.expm(M)
        return np.array([[float(X[i, j]) for j in range(A.shape[1])]
                         for i in range(A.shape[0])])


LAM_CASES = [
    [0.7],
    [3.0, 2.0, 1.0],
    [13.7, 49.7, 191.9, 142.6, 290.4],
    [1.0, 1.0, 1.0],                      # equal rates (defective matrix)
    [0.5, 0.5 * (1 + 1e-9), 2.0],         # nearly equal
    [5.0, 1e-12, 5.0 + 1e-7, 0.3],        # non-adjacent near-equal pair
    [2500.0, 0.2, 1e-30, 7.0],            # stiff
    [0.0, 0.0, 1.0],                      # zero rates
    [1e-9, 3e-9, 2e-9, 5e-9, 4e-9],
]


@pytest.mark.parametrize("lam", LAM_CASES)
def test_expm_vs_arbitrary_precision(lam):
    A = window_matrix(lam)
    got = oracle.expm(A)
    want = mp_expm(A)
    assert np.max(np.abs(got - want)) <= 1e-14
    nz = want > 1e-280
    assert np.max(np.abs(got[nz] - want[nz]) / want[nz]) <= 1e-12


def uniformized_expm(A):
    """exp(A) for a generator A (off-diagonal >= 0, columns summing to 0) by
    uniformization (Jensen): with q >= max |A_ii| and P = I + A/q, exp(A) =
    e^{-q} sum_n q^n/n! P^n.  P is column-stochastic, so every term is
    non-negative and nothing cancels.  Large q is split into m substeps,
    each done this way, and the results multiplied."""
    w = A.shape[0]
    q = max(1e-300, float(np.max(-np.diag(A))))
    m = max(1, int(math.ceil(q / 20.0)))
    qs = q / m
    P = np.eye(w) + A / q
    term = np.eye(w) * math.exp(-qs)
    X = term.copy()
    n = 0
    while True:
        n += 1
        term = term @ P * (qs / n)
        X += term
        if n > qs and term.max() < 1e-20:
            break
    return np.linalg.matrix_power(X, m)


@pytest.mark.parametrize("lam", LAM_CASES)
def test_expm_vs_uniformization(lam):
    A = window_matrix(lam)
    got = oracle.expm(A)
    want = uniformized_expm(A)
    # the m substep products of the uniformization round about m times
    m = max(1, int(math.ceil(float(np.max(-np.diag(A))) / 20.0)))
    assert np.max(np.abs(got - want)) <= 2e-15 * (m + 10)


def test_expm_equal_rate_closed_forms():
    # Equal rates lam, unit population at the bottom: N_j = lam^j e^-lam / j!
    # below the absorbing top (Poisson), the top gets the rest.
    for lam in [0.3, 1.0, 4.0, 20.0]:
        P = oracle.expm(window_matrix([lam] * 4))
        for j in range(4):
            assert P[j, 0] == pytest.approx(lam ** j * math.exp(-lam) / math.factorial(j),
                                            rel=1e-13, abs=1e-300)
        tail = 1 - sum(lam ** j * math.exp(-lam) / math.factorial(j) for j in range(4))
        assert P[4, 0] == pytest.approx(tail, rel=1e-12, abs=1e-15)


def test_expm_two_level_closed_form():
    for lam in [1e-8, 0.01, 1.0, 37.0]:
        P = oracle.expm(window_matrix([lam]))
        assert P[0, 0] == pytest.approx(math.exp(-lam), rel=1e-15)
        assert P[1, 0] == pytest.approx(-math.expm1(-lam), rel=1e-13)
        assert P[1, 1] == 1.0 and P[0, 1] == 0.0


def paper_eqs_6_to_9(a, b, c, n):
    """The paper's explicit 4-level solution, Eqs. 6-9, with the typos fixed:
    Eq. 7's e^{+W_{p+1}dt} is e^{-W_{p+1}dt}; in Eq. 9 the three e^{-W_{p+2}dt}
    terms change sign, which is what makes Eq. 9 equal 1 - (Eqs. 6-8)."""
    ea, eb, ec = math.exp(-a), math.exp(-b), math.exp(-c)
    n0, n1, n2, n3 = n
    p0 = n0 * ea                                                       # Eq. 6
    p1 = n0 * a / (a - b) * (eb - ea) + n1 * eb                        # Eq. 7
    p2 = (n0 * (a * b * ec / ((a - c) * (b - c)) - a * b * eb / ((a - b) * (b - c))
                + a * b * ea / ((a - b) * (a - c)))
          + n1 * ((a * b - b * c) * ec / ((a - c) * (b - c))
                  - (a * b - b * b) * eb / ((a - b) * (b - c)))
          + n2 * ((c * c + a * b - a * c - b * c) * ec / ((a - c) * (b - c))))  # Eq. 8
    p3 = (n0 * (1 - a * b * ec / ((a - c) * (b - c)) + a * c * eb / ((a - b) * (b - c))
                - b * c * ea / ((a - b) * (a - c)))
          + n1 * (1 - (a * b - b * c) * ec / ((a - c) * (b - c))
                  + (a * c - b * c) * eb / ((a - b) * (b - c)))
          + n2 * (1 - (c * c + a * b - a * c - b * c) * ec / ((a - c) * (b - c)))
          + n3)                                                         # Eq. 9
    return np.array([p0, p1, p2, p3])


@pytest.mark.parametrize("abc", [(3.0, 2.0, 1.0), (0.9, 2.7, 0.05), (13.7, 49.7, 191.9),
                                 (0.02, 0.011, 0.3)])
def test_paper_four_level_solution(abc):
    a, b, c = abc
    rng = np.random.default_rng(1)
    n = rng.dirichlet(np.ones(4))
    got = oracle.expm(window_matrix([a, b, c])) @ n
    want = paper_eqs_6_to_9(a, b, c, n)
    assert np.max(np.abs(got - want)) <= 1e-13


def test_corrected_eq9_numbers():
    # Column of the bottom state for (a,b,c) = (3,2,1), dt = 0.7: the top
    # state's coefficients from Eq. 9 (corrected) -- the printed signs give
    # values above 1, the corrected ones are probabilities.
    a, b, c = 3 * 0.7, 2 * 0.7, 1 * 0.7
    P = oracle.expm(window_matrix([a, b, c]))
    for j, e in enumerate(np.eye(4)[:3]):
        assert P[3, j] == pytest.approx(paper_eqs_6_to_9(a, b, c, e)[3], abs=1e-14)
        assert 0.0 <= P[3, j] <= 1.0


def rk4(A, n0, steps):
    h = 1.0 / steps
    n = np.array(n0, dtype=np.float64)
    for _ in range(steps):
        k1 = A @ n
        k2 = A @ (n + 0.5 * h * k1)
        k3 = A @ (n + 0.5 * h * k2)
        k4 = A @ (n + h * k3)
        n = n + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return n


@pytest.mark.parametrize("lam", [[0.4, 2.2, 1.3], [5.0, 5.0, 0.7, 3.1], [9.0, 0.1]])
def test_expm_vs_rk4_brute_force(lam):
    A = window_matrix(lam)
    n0 = np.random.default_rng(2).dirichlet(np.ones(A.shape[0]))
    want = rk4(A, n0, 20000)
    got = oracle.expm(A) @ n0
    assert np.max(np.abs(got - want)) <= 1e-12


@pytest.mark.parametrize("lam", LAM_CASES)
def test_expm_invariants(lam):
    A = window_matrix(lam)
    P = oracle.expm(A)
    assert np.all(P >= 0.0)
    assert np.all(np.triu(P, 1) == 0.0)
    assert np.max(np.abs(P.sum(axis=0) - 1.0)) <= 1e-14      # conservation
    P2 = oracle.expm(2 * A)
    assert np.max(np.abs(P @ P - P2)) <= 1e-13                # semigroup
    assert np.array_equal(oracle.expm(0 * A), np.eye(A.shape[0]))


# --------------------------------------------------------------------------
# The full step: windows, dn_e, window update
# --------------------------------------------------------------------------
def nitrogen():
    return oracle.Species(N2_U, N2_L, [0] * 7)


def test_step_single_level_closed_form():
    sp = nitrogen()
    E = np.array([800.0, 1500.0, 3000.0])
    dt = 0.05
    N = np.zeros((8, 3))
    N[3] = 1.0
    lo = np.full(3, 3, np.uint8)
    hi = np.full(3, 4, np.uint8)
    N1, lo1, hi1, dne = oracle.step(sp, E, N, dt, lo, hi, window_update=False)
    lam = np.array([oracle.adk_rate(e, N2_U[3], 0, 0, 4) * dt for e in E])
    assert np.allclose(N1[3], np.exp(-lam), rtol=1e-14, atol=0)
    assert np.allclose(N1[4], -np.expm1(-lam), rtol=1e-13, atol=0)
    # dn_e = 3 (N3' - 1) + 4 N4' = 1 - e^-lam   (one electron per ionization)
    assert np.allclose(dne, -np.expm1(-lam), rtol=1e-12, atol=1e-16)
    ng = np.array([2.0, 3.0, 0.5])
    _, _, _, dne_g = oracle.step(sp, E, N, dt, lo, hi, n_gas=ng, window_update=False)
    assert np.allclose(dne_g, ng * dne, rtol=1e-15)


def test_step_four_level_matches_paper():
    sp = nitrogen()
    rng = np.random.default_rng(3)
    E = rng.uniform(200, 3000, 64)
    dt = 0.05
    N = np.zeros((8, 64))
    lo = rng.integers(0, 4, 64).astype(np.uint8)
    hi = (lo + 3).astype(np.uint8)
    for c in range(64):
        N[lo[c]:lo[c] + 4, c] = rng.dirichlet(np.ones(4))
    N1, _, _, dne = oracle.step(sp, E, N, dt, lo, hi, window_update=False)
    for c in range(64):
        p = lo[c]
        lam = [oracle.adk_rate(E[c], N2_U[p + i], N2_L[p + i], 0, p + i + 1) * dt
               for i in range(3)]
        want = paper_eqs_6_to_9(*lam, N[p:p + 4, c])
        assert np.max(np.abs(N1[p:p + 4, c] - want)) <= 1e-12
        # states outside the window are untouched
        mask = np.ones(8, bool)
        mask[p:p + 4] = False
        assert np.array_equal(N1[mask, c], N[mask, c])
        # one electron per unit of population crossing each boundary
        assert dne[c] == pytest.approx(float(np.dot(np.arange(p, p + 4),
                                                    want - N[p:p + 4, c])), abs=1e-13)


def test_full_window_equals_full_system():
    # A window [0, Z] is the whole Eq. 3 system, whose top (Z+) state has no
    # outflow; the reduced step then equals exp(dt A_full) N.
    sp = nitrogen()
    E = np.array([2300.0])
    N = np.zeros((8, 1))
    N[0] = 1.0
    N1, _, _, _ = oracle.step(sp, E, N, 0.05, [0], [7], window_update=False)
    lam = [oracle.adk_rate(2300.0, N2_U[k], N2_L[k], 0, k + 1) * 0.05 for k in range(7)]
    want = mp_expm(window_matrix(lam)) @ N[:, 0]
    assert np.max(np.abs(N1[:, 0] - want)) <= 1e-14
    assert abs(N1[:, 0].sum() - 1.0) <= 1e-14


def test_window_update_rules():
    sp = nitrogen()
    dt = 0.2
    # cell 0: strong field empties the bottom level -> slides
    # cell 1: zero field, bottom level populated -> stays
    # cell 2: window already at the top (hi = Z) -> stays
    # cell 3: everything in the top level of the window -> slides w-1 times
    # cell 4: bottom level holds exactly nothing and the field is zero -> slides
    E = np.array([3000.0, 0.0, 3000.0, 0.0, 0.0])
    N = np.zeros((8, 5))
    N[0, 0] = 1.0
    N[1, 1] = 1.0
    N[4:8, 2] = 0.25
    N[5, 3] = 1.0
    N[3, 4] = 0.5
    N[4, 4] = 0.5
    lo = np.array([0, 1, 4, 2, 2], np.uint8)
    hi = np.array([3, 4, 7, 5, 5], np.uint8)
    N1, lo1, hi1, _ = oracle.step(sp, E, N, dt, lo, hi, eps_shift=1e-6)
    assert N1[0, 0] < 1e-6 and N1[1, 0] < 1e-6  # W_0 dt, W_1 dt >> 14 here
    shifts0 = 0
    while shifts0 < 3 and N1[shifts0, 0] < 1e-6:
        shifts0 += 1
    assert (lo1[0], hi1[0]) == (shifts0, 3 + shifts0) and shifts0 >= 2
    assert (lo1[1], hi1[1]) == (1, 4)
    assert (lo1[2], hi1[2]) == (4, 7)
    assert (lo1[3], hi1[3]) == (4, 7)  # slide stops at hi = Z
    assert (lo1[4], hi1[4]) == (3, 6)
    # fixed windows when the update is off
    _, lo2, hi2, _ = oracle.step(sp, E, N, dt, lo, hi, window_update=False)
    assert np.array_equal(lo2, lo) and np.array_equal(hi2, hi)


def test_adaptive_window_rules():
    """The adaptive policy on hand-made cells at zero field (populations
    unchanged), each expected window worked out by hand from the rule."""
    sp = nitrogen()
    N = np.zeros((8, 5))
    N[1:3, 0] = 0.5            # [0,3]: empty bottom dropped -> [1,3]
    N[3, 1] = 1.0              # [2,3] at w_min: slides, full top grows -> [3,5]
    N[7, 2] = 1.0              # [4,7]: shrinks to w_min at the top -> [6,7]
    N[1:6, 3] = 0.18           # [1,6] at w_max with a populated top -> [1,6]
    N[6, 3] = 0.1
    N[0, 4] = 0.6              # [0,2], populated top -> grows to [0,3]
    N[2, 4] = 0.4
    lo = np.array([0, 2, 4, 1, 0], np.uint8)
    hi = np.array([3, 3, 7, 6, 2], np.uint8)
    E = np.zeros(5)
    N1, lo1, hi1, dne = oracle.step(sp, E, N, 0.05, lo, hi, policy=oracle.WINDOW_ADAPTIVE,
                                    w_min=2, w_max=6, eps_grow=1e-6)
    assert np.array_equal(N1, N) and np.all(dne == 0)
    assert list(zip(lo1, hi1)) == [(1, 3), (3, 5), (6, 7), (1, 6), (0, 3)]
    # w_min = 3: the bottom is dropped once, then the window slides
    M = np.zeros((8, 1))
    M[2:4, 0] = 0.5
    _, lo2, hi2, _ = oracle.step(sp, np.zeros(1), M, 0.05, [0], [3],
                                 policy=oracle.WINDOW_ADAPTIVE, w_min=3, w_max=6)
    assert (lo2[0], hi2[0]) == (2, 5)
    # with w_min = w_max = w and no growth it is the paper's rule
    E2 = np.array([3000.0, 0.0])
    P = np.zeros((8, 2))
    P[0] = [1.0, 0.0]
    P[1] = [0.0, 1.0]
    a = oracle.step(sp, E2, P, 0.2, [0, 1], [3, 4])
    b = oracle.step(sp, E2, P, 0.2, [0, 1], [3, 4], policy=oracle.WINDOW_ADAPTIVE,
                    w_min=4, w_max=4, eps_grow=np.inf)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_window_width_one_and_dt_zero():
    sp = nitrogen()
    N = np.zeros((8, 2))
    N[2] = [0.3, 1.0]
    N[3] = [0.7, 0.0]
    N1, lo1, hi1, dne = oracle.step(sp, np.array([5000.0, 5000.0]), N, 0.05,
                                    [2, 2], [2, 2], window_update=True)
    assert np.array_equal(N1, N) and np.all(dne == 0.0)
    N2, _, _, dne2 = oracle.step(sp, np.array([5000.0, 5000.0]), N, 0.0, [2, 2],
                                 [5, 5], window_update=False)
    assert np.array_equal(N2, N) and np.all(dne2 == 0.0)
