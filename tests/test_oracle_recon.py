"""Pins of the oracle's reconstruction against what the paper prints and what mathematics fixes.

The oracle derives every weight by solving the stencil conditions; these tests compare
the results with the coefficients the paper prints (Sec. 3.1, Sec. 3.3, Appendix), with
exact polynomial reproduction, and with the modified-wavenumber closed forms (Sec. 3.2).
"""
from fractions import Fraction

import math

import numpy as np
import pytest

import oracle
from conftest import golden_coeffs

G = golden_coeffs()


def printed(name):
    den, nums = G[name]
    return np.array(nums, dtype=float) / den


# --------------------------------------------------------------------------- linear
@pytest.mark.parametrize("order,names", [
    (6, ("lin6_value", "lin6_deriv", "lin6_deriv2")),
    (8, ("lin8_value", "lin8_deriv", "lin8_deriv2")),
])
def test_linear_weights_match_printed(order, names):
    w = oracle.linear_weights(order)
    for q, name in enumerate(names):
        np.testing.assert_allclose(w[q], printed(name), rtol=0, atol=1e-13, err_msg=name)


def _exact_stencil_inputs(k):
    """Exact cell averages and dx*averaged slopes of s^k on cells -1..2 (unit cells centred
    at the offsets), as Fractions."""
    ins = []
    for o in (-1, 0, 1, 2):
        a, b = Fraction(2 * o - 1, 2), Fraction(2 * o + 1, 2)
        ins.append((b ** (k + 1) - a ** (k + 1)) / (k + 1))
    for o in (-1, 0, 1, 2):
        a, b = Fraction(2 * o - 1, 2), Fraction(2 * o + 1, 2)
        ins.append(b ** k - a ** k)
    return ins


@pytest.mark.parametrize("order,maxdeg", [(6, 5), (8, 7)])
def test_linear_reconstruction_polynomial_exactness(order, maxdeg):
    """P^5 / P^7 reproduce interface value and first two derivatives of any polynomial of
    degree <= 5 / <= 7 (Sec. 3.1: truncation error O(dx^{n+1}))."""
    w = oracle.linear_weights(order)
    half = Fraction(1, 2)
    for k in range(maxdeg + 1):
        ins = np.array([float(x) for x in _exact_stencil_inputs(k)])
        exact = [half ** k, k * half ** (k - 1) if k >= 1 else 0, k * (k - 1) * half ** (k - 2) if k >= 2 else 0]
        for q in range(3):
            assert abs(w[q] @ ins - float(exact[q])) < 1e-14 * np.abs(ins).sum() * 8, (order, k, q)
    # and it is genuinely of that order: degree maxdeg+1 is not reproduced by the value
    ins = np.array([float(x) for x in _exact_stencil_inputs(maxdeg + 1)])
    if order == 8:
        assert abs(w[0] @ ins - 0.5 ** (maxdeg + 1)) > 1e-6


@pytest.mark.parametrize("order,name", [(6, "disc6"), (8, "disc8")])
def test_semidiscrete_derivative_matches_printed(order, name):
    """(P(x_{i+1/2}) - P(x_{i-1/2}))/dx expressed on W_{i-2..i+2}, W'_{i-2..i+2}
    equals Eqs. (discrete-6th)/(discrete-8th)."""
    v = oracle.linear_weights(order)[0]
    coef = np.zeros(10)
    # interface i+1/2 uses cells i-1..i+2 -> indices 1..4 of W_{i-2..i+2}
    for m in range(4):
        coef[1 + m] += v[m]
        coef[5 + 1 + m] += v[4 + m]
        coef[m] -= v[m]          # interface i-1/2 uses cells i-2..i+1
        coef[5 + m] -= v[4 + m]
    np.testing.assert_allclose(coef, printed(name), atol=1e-13)


@pytest.mark.parametrize("order,name", [(6, "wave6"), (8, "wave8")])
def test_modified_wavenumber_closed_form(order, name):
    """Fourier symbol of the scheme's derivative with exact slopes (Sec. 3.2) equals the
    printed closed forms of Eqs. (wavenumber-6th)/(wavenumber-8th)."""
    v = oracle.linear_weights(order)[0]
    den, c = G[name]
    for om in np.linspace(0.05, np.pi, 40):
        # W_j = e^{i om j}, dx W'_j = i om e^{i om j}; interface i+1/2 minus i-1/2
        j = np.arange(-1, 3)
        plus = np.sum(v[:4] * np.exp(1j * om * j)) + np.sum(v[4:] * 1j * om * np.exp(1j * om * j))
        deriv = plus * (1 - np.exp(-1j * om))
        omega_p = deriv.imag
        closed = (c[0] * np.sin(om) + c[1] * np.sin(2 * om) + c[2] * om * np.cos(om)
                  + c[3] * om * np.cos(2 * om) + c[4] * om) / den
        assert abs(omega_p - closed) < 1e-12
        assert abs(deriv.real) < 1e-12      # symmetric stencil: no dissipation
    # values at pi/2 and pi from the closed form
    if order == 6:
        assert abs(0.76 * np.pi - (c[2] * np.pi * -1 + c[3] * np.pi + c[4] * np.pi) / den) < 1e-12


# --------------------------------------------------------------------------- WENO
@pytest.mark.parametrize("k", range(7))
def test_candidate_point_values_match_printed(k):
    """Candidates solved from their sub-stencil conditions give the printed w_{k,i+1/2}."""
    C, deg = oracle.candidate(k)
    val = np.array([sum(C[p, m] * 0.5 ** p for p in range(deg + 1)) for m in range(8)])
    np.testing.assert_allclose(val, printed(f"cand{k}_value"), atol=1e-13)
    assert deg == {0: 2, 1: 2, 2: 3, 3: 2, 4: 2, 5: 4, 6: 4}[k]


@pytest.mark.parametrize("k", [0, 2, 3, 4, 5, 6, 7])
def test_candidate_taylor_coefficients_match_appendix(k):
    """Appendix: w(x) = sum a_k x^k/k!; the oracle's solved polynomial has a_p = p! c_p."""
    C, deg = oracle.candidate(k)
    fact = [1, 1, 2, 6, 24]
    for p in range(deg + 1):
        np.testing.assert_allclose(fact[p] * C[p], printed(f"app{k}_a{p}"), atol=1e-11,
                                   err_msg=f"candidate {k}, a_{p}")


def test_appendix_w6_operator_reading():
    """The garbled operator before a_4 of w_6: only '+' satisfies the cell-average
    condition on I_i (average of w over [-1/2, 1/2] is a_0 + a_2/24 + a_4/1920)."""
    a0, a2, a4 = printed("app6_a0"), printed("app6_a2"), printed("app6_a4")
    e_i = np.array([0, 1, 0, 0, 0, 0, 0, 0], dtype=float)
    np.testing.assert_allclose(a0 + a2 / 24 + a4 / 1920, e_i, atol=1e-14)
    assert np.abs(a0 + a2 / 24 - a4 / 1920 - e_i).max() > 1e-3


@pytest.mark.parametrize("order,name", [(6, "d6"), (8, "d8")])
def test_linear_weights_recover_linear_reconstruction(order, name):
    """Sec. 3.3: sum_k d_k w_{k,i+1/2} = P^n(x_{i+1/2}) identically, and sum_k d_k = 1."""
    d = printed(name)
    assert abs(d.sum() - 1.0) < 1e-15
    comb = np.zeros(8)
    for k in range(7):
        comb += d[k] * printed(f"cand{k}_value")
    np.testing.assert_allclose(comb, oracle.linear_weights(order)[0], atol=1e-13)


def test_smoothness_indicator_constants():
    """Appendix beta constants from the definition (Eq. smooth-indicator): the oracle's
    integration reproduces 1, 13/12, 1043/960, 1/12, 7/80; the (a4 h^4)^2 constant is
    87617/80640 (the printed 35045/32256 differs by 5e-5 relative)."""
    fact = [1, 1, 2, 6, 24]

    def beta_of(a):   # a = Taylor coefficients a_k h^k
        c = np.array([a[p] / fact[p] for p in range(5)])
        return oracle.smoothness(c, 4)
    num = G["beta_const_num"][1]
    den = G["beta_const_den"][1]
    printed_c = [n / d for n, d in zip(num, den)]
    basis = np.eye(5)
    b1 = beta_of(basis[1]); b2 = beta_of(basis[2]); b3 = beta_of(basis[3]); b4 = beta_of(basis[4])
    assert abs(b1 - printed_c[0]) < 1e-15
    assert abs(b2 - printed_c[1]) < 1e-15
    assert abs(b3 - printed_c[2]) < 1e-15
    assert abs(b4 - 87617 / 80640) < 1e-15
    assert abs(b4 - printed_c[3]) > 1e-5
    cross13 = beta_of(basis[1] + basis[3]) - b1 - b3
    cross24 = beta_of(basis[2] + basis[4]) - b2 - b4
    assert abs(cross13 - printed_c[4]) < 1e-14
    assert abs(cross24 - printed_c[5]) < 1e-14


def test_smoothness_indicator_vs_quadrature():
    """beta = sum_q dx^{2q-1} int_{I_i} (d^q w/dx^q)^2 dx by adaptive quadrature."""
    from scipy.integrate import quad
    rng = np.random.default_rng(3)
    for deg in (2, 3, 4):
        c = rng.standard_normal(deg + 1)
        tot = 0.0
        for q in range(1, deg + 1):
            dq = np.polynomial.polynomial.polyder(c, q)
            tot += quad(lambda s: np.polynomial.polynomial.polyval(s, dq) ** 2, -0.5, 0.5,
                        epsabs=1e-14, epsrel=1e-13)[0]
        assert abs(oracle.smoothness(c, deg) - tot) < 1e-12 * max(1, tot)


def _sine_stencil(h, x_i=0.3, slope=True):
    xs = x_i + h * np.arange(-1, 3)
    avg = (np.cos(xs - h / 2) - np.cos(xs + h / 2)) / h          # average of sin
    sl = (np.sin(xs + h / 2) - np.sin(xs - h / 2)) / h * h        # dx * averaged slope
    return np.concatenate([avg, sl])


@pytest.mark.parametrize("order", [6, 8])
def test_wenoz_weights_collapse_on_smooth_data(order):
    """Sec. 3.4: delta_k - d_k = O(dx^5) on smooth data (observed rate >= 4)."""
    d = printed("d6" if order == 6 else "d8")
    errs = []
    hs = [0.1, 0.05, 0.025, 0.0125]
    for h in hs:
        _, _, delta, _ = oracle.weno_left(order, _sine_stencil(h), eps=1e-40)
        errs.append(np.abs(delta - d).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > 4.0, rates


@pytest.mark.parametrize("order", [6, 8])
def test_wenoz_special_cases(order):
    d = printed("d6" if order == 6 else "d8")
    # constant data: all beta = 0 -> weights are the linear ones, value exact
    val, der, delta, beta = oracle.weno_left(order, [2.0] * 4 + [0.0] * 4)
    np.testing.assert_allclose(delta, d, atol=1e-15)
    assert abs(val - 2.0) < 1e-14 and abs(der) < 1e-13
    # linear data: value and derivative are exact (every candidate reproduces lines)
    val, der, _, _ = oracle.weno_left(order, [-1.0, 0.0, 1.0, 2.0] + [1.0] * 4)
    assert abs(val - 0.5) < 1e-13 and abs(der - 1.0) < 1e-12
    # a jump between cells i+1 and i+2: stencils containing I_{i+2} get small weight,
    # and the left value stays within the data range of I_{i-1}..I_{i+1}
    val, der, delta, _ = oracle.weno_left(order, [1.0, 1.0, 1.0, 0.0] + [0.0] * 4)
    assert delta[2] + delta[4] + delta[6] < 1e-6
    assert 1.0 - 1e-6 < val < 1.0 + 1e-6


@pytest.mark.parametrize("order", [6, 8])
def test_weno_right_is_mirror_of_left(order):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(8)
    mirrored = [x[3], x[2], x[1], x[0], -x[7], -x[6], -x[5], -x[4]]
    vl, dl, _, _ = oracle.weno_left(order, mirrored)
    vr, dr = oracle.weno_right(order, x)
    assert vr == vl and dr == -dl


# --------------------------------------------------------------------------- tangential
def test_tangential_quartic_exactness_and_gauss_rule():
    """Quartic through five segment averages: exact for polynomials of degree <= 4 at the
    three Gauss points (value and first two derivatives); 3-point Gauss-Legendre rule is
    exact for degree <= 5."""
    w, gs, gw = oracle.tangential_weights()
    for k in range(5):
        avgs = np.array([((o + 0.5) ** (k + 1) - (o - 0.5) ** (k + 1)) / (k + 1) for o in range(-2, 3)])
        for g in range(3):
            s = gs[g]
            exact = [s ** k, k * s ** (k - 1) if k else 0.0, k * (k - 1) * s ** (k - 2) if k > 1 else 0.0]
            for q in range(3):
                assert abs(w[g, q] @ avgs - exact[q]) < 1e-12
    for k in range(6):
        exact = ((0.5) ** (k + 1) - (-0.5) ** (k + 1)) / (k + 1)
        assert abs(np.sum(gw * gs ** k) - exact) < 1e-15


# --------------------------------------------------------------------------- tangential WENO-Z
def _avg_poly(offsets, deg, q):
    """Polynomial (coefficients of s^p) whose averages over the unit segments centred at
    `offsets` are q (numpy, independent of the oracle)."""
    A = np.array([[((o + 0.5) ** (p + 1) - (o - 0.5) ** (p + 1)) / (p + 1) for p in range(deg + 1)]
                  for o in offsets])
    return np.linalg.solve(A, np.asarray(q, dtype=float))


def _eval(c, s, der=0):
    return np.polyval(np.polyder(c[::-1], der) if der else c[::-1], s)


GAUSS = [-0.5 * math.sqrt(0.6), 0.0, 0.5 * math.sqrt(0.6)]


@pytest.mark.parametrize("g", [0, 1, 2])
@pytest.mark.parametrize("der", [0, 1])
def test_tangential_weno_linear_weights_recombine_the_quartic(g, der):
    """Variant of reading R9: the linear weights of the three quadratic candidates at a Gauss
    point give the quartic through the five line averages, for any data (random data, the
    candidates and the quartic built here with numpy); the value weights at the outer points
    are positive (126/655 +- 71 sqrt(15)/5240, 403/655), at the centre negative at both ends
    (-9/80, 49/40, -9/80); the derivative weights are positive."""
    rng = np.random.default_rng(g + 3 * der)
    _, d = oracle.tan_weno([0.0] * 5, g, der)
    for _ in range(5):
        q = rng.standard_normal(5)
        P4 = _avg_poly([-2, -1, 0, 1, 2], 4, q)
        cands = [_avg_poly(offs, 2, q[k:k + 3]) for k, offs in enumerate(([-2, -1, 0], [-1, 0, 1], [0, 1, 2]))]
        lhs = sum(d[k] * _eval(cands[k], GAUSS[g], der) for k in range(3))
        assert abs(lhs - _eval(P4, GAUSS[g], der)) < 1e-13 * (1 + np.abs(q).max())
    if der == 0 and g != 1:
        r = 71 * math.sqrt(15) / 5240
        want = [126 / 655 + r, 403 / 655, 126 / 655 - r]
        np.testing.assert_allclose(d, want if g == 0 else want[::-1], rtol=1e-12)
    elif der == 0:
        np.testing.assert_allclose(d, [-9 / 80, 49 / 40, -9 / 80], rtol=1e-12)
    else:
        assert (d > 0).all()


@pytest.mark.parametrize("g", [0, 1, 2])
def test_tangential_weno_on_smooth_and_step_data(g):
    """Smooth data: the WENO-Z value and derivative approach the quartic's (the candidates'
    weights tend to the linear ones) faster than the quartic's own error shrinks; step data:
    the outer-point values stay within the data range (no overshoot), where the quartic
    overshoots."""
    errs = []
    for h in (0.8, 0.4, 0.2):
        # averages of 2 + sin(h s + 0.7) (no symmetry about the centre, so the weights move)
        q = [(math.cos(h * (o - 0.5) + 0.7) - math.cos(h * (o + 0.5) + 0.7)) / h + 2.0 for o in range(-2, 3)]
        P4 = _avg_poly([-2, -1, 0, 1, 2], 4, q)
        v, _ = oracle.tan_weno(q, g, 0)
        dv, _ = oracle.tan_weno(q, g, 1)
        errs.append(max(abs(v - _eval(P4, GAUSS[g])), abs(dv - _eval(P4, GAUSS[g], 1)) / h))
    assert errs[0] > 4 * errs[1] > 16 * errs[2] and errs[2] < 1e-5, errs
    step = [1.0, 1.0, 1.0, 0.0, 0.0]
    P4 = _avg_poly([-2, -1, 0, 1, 2], 4, step)
    v, _ = oracle.tan_weno(step, g, 0)
    if g != 1:
        assert -1e-6 <= v <= 1.0 + 1e-6
    assert _eval(P4, GAUSS[2]) > 1.0 + 1e-3 or _eval(P4, GAUSS[0]) > 1.0 + 1e-3
