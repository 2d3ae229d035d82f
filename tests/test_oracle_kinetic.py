"""Pins of the oracle's gas-kinetic part (Sec. 2.1, Eq. 3rd-simplify-flux, Sec. 4 collision
times) against closed forms of the Maxwellian and of the Euler / Navier-Stokes equations."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import gamma as Gamma

import oracle

GAM = 1.4
K1 = (3 - GAM) / (GAM - 1)          # 1D internal degrees of freedom (reading R11)
K2 = (4 - 2 * GAM) / (GAM - 1)      # 2D, Sec. 2.1


def prim(W, dim):
    rho = W[0]
    U = W[1] / rho
    V = W[2] / rho if dim == 2 else 0.0
    p = (GAM - 1) * (W[-1] - 0.5 * rho * (U * U + V * V))
    return rho, U, V, p


def euler_flux(W, dim, direction=0):
    rho, U, V, p = prim(W, dim)
    un = U if direction == 0 else V
    F = np.array(W, dtype=complex) * un
    F[1 + direction] += p
    F[-1] += p * un
    return F


def jacobian(W, dim, direction=0):
    """Euler flux Jacobian by complex-step differentiation (exact to rounding)."""
    n = dim + 2
    A = np.zeros((n, n))
    for k in range(n):
        Wc = np.array(W, dtype=complex)
        Wc[k] += 1e-30j
        A[:, k] = euler_flux(Wc, dim, direction).imag / 1e-30
    return A


def W_from_prim(rho, U, V, p, dim):
    if dim == 1:
        return np.array([rho, rho * U, p / (GAM - 1) + 0.5 * rho * U * U])
    return np.array([rho, rho * U, rho * V, p / (GAM - 1) + 0.5 * rho * (U * U + V * V)])


# --------------------------------------------------------------------------- moments
@pytest.mark.parametrize("U,lam", [(0.3, 0.7), (-1.2, 2.5), (2.0, 0.3)])
def test_maxwellian_moments_vs_quadrature(U, lam):
    m = oracle.maxwell_moments(2, K2, U, -0.4, lam)
    g = lambda u: math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
    for n in range(8):
        full = quad(lambda u: u ** n * g(u), -np.inf, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
        pos = quad(lambda u: u ** n * g(u), 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
        neg = quad(lambda u: u ** n * g(u), -np.inf, 0, epsabs=1e-14, epsrel=1e-13)[0]
        scale = max(1.0, abs(full))
        assert abs(m["mu"][n] - full) < 1e-11 * scale
        assert abs(m["mup"][n] - pos) < 1e-11 * scale
        assert abs(m["mun"][n] - neg) < 1e-11 * scale
        assert abs(m["mup"][n] + m["mun"][n] - m["mu"][n]) < 1e-13 * scale
    # internal degrees of freedom: E|xi|^{2k} = lam^{-k} Gamma(K/2 + k) / Gamma(K/2)
    for k in range(4):
        ref = lam ** (-k) * Gamma(K2 / 2 + k) / Gamma(K2 / 2)
        assert abs(m["mx"][k] - ref) < 1e-13 * max(1, ref)


def _maxwellian_log_derivative(dim, K, rho, U, V, lam, drho, dU, dV, dlam):
    """Coefficients (on psi) of d/dx ln g for g = rho (lam/pi)^{(K+dim)/2} e^{-lam c^2}."""
    n = dim + 2
    a = np.zeros(n)
    a[0] = drho / rho + 0.5 * (K + dim) * dlam / lam - dlam * (U * U + V * V) - 2 * lam * (U * dU + V * dV)
    a[1] = 2 * (dlam * U + lam * dU)
    if dim == 2:
        a[2] = 2 * (dlam * V + lam * dV)
    a[-1] = -2 * dlam
    return a


@pytest.mark.parametrize("dim", [1, 2])
def test_solve_coef_is_maxwellian_log_derivative(dim):
    """Sec. 2.1: the solved coefficients a (int psi (a.psi) g = dW/dx) equal the exact
    logarithmic derivative of the Maxwellian along a smooth primitive field."""
    K = K1 if dim == 1 else K2
    rng = np.random.default_rng(11)
    for _ in range(5):
        rho, U, V, p = 0.5 + rng.random(), rng.standard_normal(), rng.standard_normal(), 0.5 + rng.random()
        if dim == 1:
            V = 0.0
        drho, dU, dV, dp = rng.standard_normal(4)
        if dim == 1:
            dV = 0.0
        lam = rho / (2 * p)
        dlam = drho / (2 * p) - rho * dp / (2 * p * p)
        # dW/dx by complex step on W(prim(x))
        h = 1e-30
        Wc = W_from_prim(rho + 1j * h * drho, U + 1j * h * dU, V + 1j * h * dV, p + 1j * h * dp, dim)
        b = Wc.imag / h
        a = oracle.solve_coef(dim, K, rho, U, V, lam, b)
        ref = _maxwellian_log_derivative(dim, K, rho, U, V, lam, drho, dU, dV, dlam)
        np.testing.assert_allclose(a, ref, rtol=1e-12, atol=1e-12)


def test_time_integrals_vs_quadrature():
    """E0 = int_0^d e^{-t/tau} dt and E1 = int_0^d t e^{-t/tau} dt: against adaptive quadrature
    of the definition, and against 50-digit evaluation over d/tau in [1e-8, 1e8] (the
    range where naive double formulas cancel)."""
    import mpmath
    mpmath.mp.dps = 50
    for tau in (1e-3, 1.0):
        for r in np.logspace(-8, 8, 33):
            d = r * tau
            E0, E1 = oracle.time_integrals(d, tau)
            if 1e-3 < r < 40:
                q0 = quad(lambda t: math.exp(-t / tau), 0, d, epsabs=0, epsrel=1e-12)[0]
                q1 = quad(lambda t: t * math.exp(-t / tau), 0, d, epsabs=0, epsrel=1e-12)[0]
                assert abs(E0 - q0) <= 1e-11 * q0 and abs(E1 - q1) <= 1e-11 * q1
            T, D = mpmath.mpf(tau), mpmath.mpf(d)
            e0 = mpmath.quad(lambda t: mpmath.exp(-t / T), [0, D])
            e1 = mpmath.quad(lambda t: t * mpmath.exp(-t / T), [0, D])
            assert abs(E0 - float(e0)) <= 1e-14 * float(e0)
            assert abs(E1 - float(e1)) <= 1e-13 * float(e1)
    # limits: d << tau -> (d, d^2/2); d >> tau -> (tau, tau^2)
    E0, E1 = oracle.time_integrals(1e-9, 1.0)
    assert abs(E0 / 1e-9 - 1) < 1e-8 and abs(E1 / 0.5e-18 - 1) < 1e-8
    E0, E1 = oracle.time_integrals(1e3, 1.0)
    assert E0 == 1.0 and E1 == 1.0


@pytest.mark.parametrize("dim", [1, 2])
def test_characteristic_eigenvectors(dim):
    """Right eigenvectors of the normal Euler Jacobian (reading R8): A r = lambda r with
    eigenvalues U - c, U, (U), U + c."""
    W = W_from_prim(1.3, 0.7, -0.2, 2.1, dim)
    R = oracle.eigvecs(dim, GAM, W)
    A = jacobian(W, dim)
    rho, U, V, p = prim(W, dim)
    c = math.sqrt(GAM * p / rho)
    lams = [U - c, U, U + c] if dim == 1 else [U - c, U, U, U + c]
    for k in range(dim + 2):
        np.testing.assert_allclose(A @ R[:, k], lams[k] * R[:, k], atol=1e-12)
    assert abs(np.linalg.det(R)) > 1e-6


# --------------------------------------------------------------------------- point
def _fields(dim, W0, W0x, W0xx=None, W0y=None, W0xy=None, W0yy=None, Wl=None, Wr=None,
            Wlx=None, Wrx=None):
    z = np.zeros(dim + 2)
    f = dict(W0=W0, W0x=W0x, W0xx=z if W0xx is None else W0xx,
             Wl=W0 if Wl is None else Wl, Wr=W0 if Wr is None else Wr,
             Wlx=W0x if Wlx is None else Wlx, Wrx=W0x if Wrx is None else Wrx)
    if dim == 2:
        f.update(W0y=z if W0y is None else W0y, W0xy=z if W0xy is None else W0xy,
                 W0yy=z if W0yy is None else W0yy, Wly=z if W0y is None else W0y,
                 Wry=z if W0y is None else W0y)
    return f


@pytest.mark.parametrize("dim", [1, 2])
def test_uniform_state_gives_euler_flux(dim):
    W0 = W_from_prim(0.8, 0.4, 0.25, 1.1, dim)
    z = np.zeros(dim + 2)
    out = oracle.point(dim, GAM, 0.0, 1.0, _fields(dim, W0, z), 1e-3)
    np.testing.assert_allclose(out["F"], euler_flux(W0, dim).real, atol=1e-14)
    assert np.abs(out["Ft"]).max() < 1e-14
    assert np.abs(out["Wt"]).max() < 1e-14 and np.abs(out["Wtt"]).max() < 1e-14
    np.testing.assert_allclose(out["W0"], W0, atol=1e-14)


@pytest.mark.parametrize("dim", [1, 2])
def test_equilibrium_branch_matches_euler_derivatives(dim):
    """Linear case (g_l = g_r = g0): F = F_Euler(W0); W_t = -A W_x - B W_y (Euler);
    F_t = A W_t; and the simplified chain gives W_tt = -(A W_xt + B W_yt) with
    W_xt = -(A W_xx + B W_xy), W_yt = -(A W_xy + B W_yy) (the Jacobians frozen at W0)."""
    rng = np.random.default_rng(5)
    W0 = W_from_prim(1.1, 0.3, -0.5, 0.9, dim)
    n = dim + 2
    Wx, Wxx = rng.standard_normal(n) * 0.3, rng.standard_normal(n) * 0.3
    Wy = rng.standard_normal(n) * 0.3 if dim == 2 else np.zeros(n)
    Wxy = rng.standard_normal(n) * 0.3 if dim == 2 else np.zeros(n)
    Wyy = rng.standard_normal(n) * 0.3 if dim == 2 else np.zeros(n)
    f = _fields(dim, W0, Wx, Wxx, Wy if dim == 2 else None, Wxy if dim == 2 else None,
                Wyy if dim == 2 else None)
    out = oracle.point(dim, GAM, 0.0, 1.0, f, 1e-3)
    A = jacobian(W0, dim, 0)
    B = jacobian(W0, dim, 1) if dim == 2 else np.zeros((n, n))
    Wt = -(A @ Wx + B @ Wy)
    Wxt = -(A @ Wxx + B @ Wxy)
    Wyt = -(A @ Wxy + B @ Wyy)
    Wtt = -(A @ Wxt + B @ Wyt)
    np.testing.assert_allclose(out["F"], euler_flux(W0, dim).real, atol=1e-13)
    np.testing.assert_allclose(out["Wt"], Wt, atol=1e-12)
    np.testing.assert_allclose(out["Ft"], A @ Wt, atol=1e-12)
    np.testing.assert_allclose(out["Wtt"], Wtt, atol=1e-11)


def _hess(W, dim, direction, u, v, eps=1e-5):
    """(dA/dW . u) v, the flux Hessian contracted with u and v (central difference of the
    complex-step Jacobian; error ~1e-10)."""
    return (jacobian(W + eps * u, dim, direction) @ v - jacobian(W - eps * u, dim, direction) @ v) / (2 * eps)


@pytest.mark.parametrize("dim", [1, 2])
def test_full_product_coefficients_give_the_cauchy_kowalewski_derivatives(dim):
    """Reading R6, variant coef_mode = 1 (the second-order Taylor polynomial of the local
    Maxwellian, products of first-order coefficients included): the interface values' time
    derivatives are those of the Euler equations themselves, W_t = -(A W_x + B W_y) and
    W_tt = -d/dt (A W_x + B W_y) = -(A W_xt + B W_yt + A'[W_t] W_x + B'[W_t] W_y) with
    W_xt = -(A W_xx + B W_xy + A'[W_x] W_x + B'[W_x] W_y) and W_yt likewise (A'[u] the
    Jacobian's derivative along u), while the simplified chain of the default reading lacks
    the Jacobian-derivative terms; F and F_t are the same in both."""
    rng = np.random.default_rng(11)
    W0 = W_from_prim(1.1, 0.3, -0.5, 0.9, dim)
    n = dim + 2
    Wx, Wxx = rng.standard_normal(n) * 0.3, rng.standard_normal(n) * 0.3
    Wy = rng.standard_normal(n) * 0.3 if dim == 2 else np.zeros(n)
    Wxy = rng.standard_normal(n) * 0.3 if dim == 2 else np.zeros(n)
    Wyy = rng.standard_normal(n) * 0.3 if dim == 2 else np.zeros(n)
    f = _fields(dim, W0, Wx, Wxx, Wy if dim == 2 else None, Wxy if dim == 2 else None,
                Wyy if dim == 2 else None)
    full = oracle.point(dim, GAM, 0.0, 1.0, f, 1e-3, coef_mode=1)
    simp = oracle.point(dim, GAM, 0.0, 1.0, f, 1e-3)
    A = jacobian(W0, dim, 0)
    B = jacobian(W0, dim, 1) if dim == 2 else np.zeros((n, n))
    HA = lambda u, v: _hess(W0, dim, 0, u, v)   # noqa: E731
    HB = (lambda u, v: _hess(W0, dim, 1, u, v)) if dim == 2 else (lambda u, v: np.zeros(n))  # noqa: E731
    Wt = -(A @ Wx + B @ Wy)
    Wxt = -(A @ Wxx + B @ Wxy + HA(Wx, Wx) + HB(Wx, Wy))
    Wyt = -(A @ Wxy + B @ Wyy + HA(Wx, Wy) + HB(Wy, Wy))
    Wtt = -(A @ Wxt + B @ Wyt + HA(Wt, Wx) + HB(Wt, Wy))
    np.testing.assert_allclose(full["Wt"], Wt, atol=1e-12)
    np.testing.assert_allclose(full["Wtt"], Wtt, atol=1e-8)
    np.testing.assert_allclose(full["F"], simp["F"], atol=1e-14)
    np.testing.assert_allclose(full["Ft"], simp["Ft"], atol=1e-13)
    assert np.abs(simp["Wtt"] - Wtt).max() > 1e-3 * np.abs(Wtt).max()


def _d4(fun, x, h):
    """Fourth-order central first derivative."""
    return (-fun(x + 2 * h) + 8 * fun(x + h) - 8 * fun(x - h) + fun(x - 2 * h)) / (12 * h)


def test_full_product_interface_values_of_the_translating_vortex():
    """The isentropic vortex translating at (1, 1) is an exact Euler solution, W(x, y, t) =
    W(x - t, y - t, 0), so W_t = -(W_x + W_y) and W_tt = (d/dx + d/dy)^2 W exactly.  With the
    point values and derivatives of the vortex (fourth-order differences), the full-product
    variant gives both; the simplified chain misses W_tt by more than its size."""
    from paper_1901_00261_gb300 import inputs
    Wf = lambda x, y: inputs.vortex_point(np.array(x), np.array(y), 0.0, GAM)   # noqa: E731
    x0, y0, h = 5.7, 4.6, 1e-3
    dx = lambda F: (lambda x, y: _d4(lambda s: F(s, y), x, h))   # noqa: E731
    dy = lambda F: (lambda x, y: _d4(lambda s: F(x, s), y, h))   # noqa: E731
    Wx, Wy = dx(Wf), dy(Wf)
    W, Wxv, Wyv = Wf(x0, y0), Wx(x0, y0), Wy(x0, y0)
    Wxx, Wxy, Wyy = dx(Wx)(x0, y0), dy(Wx)(x0, y0), dy(Wy)(x0, y0)
    f = dict(W0=W, W0x=Wxv, W0y=Wyv, W0xx=Wxx, W0xy=Wxy, W0yy=Wyy, Wl=W, Wr=W, Wlx=Wxv,
             Wrx=Wxv, Wly=Wyv, Wry=Wyv)
    exact_tt = Wxx + 2 * Wxy + Wyy
    full = oracle.point(2, GAM, 0.0, 1.0, f, 1e-3, coef_mode=1)
    simp = oracle.point(2, GAM, 0.0, 1.0, f, 1e-3)
    np.testing.assert_allclose(full["Wt"], -(Wxv + Wyv), atol=1e-9)
    np.testing.assert_allclose(full["Wtt"], exact_tt, atol=1e-7 * np.abs(exact_tt).max())
    assert np.abs(simp["Wtt"] - exact_tt).max() > np.abs(exact_tt).max()


def test_full_product_variant_needs_the_euler_bracket_free_setting():
    with pytest.raises(ValueError):
        oracle.Solver(10, 1, mu=0.01, coef_mode=1)
    with pytest.raises(ValueError):
        oracle.Solver(10, 1, tau_mode=1, coef_mode=1)
    oracle.Solver(10, 1, coef_mode=1)


@pytest.mark.parametrize("dim,Pr", [(1, 1.0), (1, 0.72), (2, 1.0), (2, 0.72)])
def test_chapman_enskog_bracket_is_navier_stokes(dim, Pr):
    """With tau = mu/p (reading R1) the bracket of Eq. (3rd-simplify-flux) yields the
    Navier-Stokes viscous flux of a gas with N = K + dim translational+internal degrees of
    freedom: sigma_xx = mu (2 U_x - 2/N (U_x + V_y)), sigma_xy = mu (U_y + V_x),
    q_x = -mu (N+2)/2 d/dx(p/rho); and the Prandtl fix (R10) divides q by Pr."""
    mu = 0.03
    rho, U, V, p = 1.2, 0.4, -0.3, 0.8
    d = dict(rho=(0.3, -0.2), U=(0.5, 0.1), V=(-0.25, 0.35), p=(0.2, 0.15))
    if dim == 1:
        V = 0.0
        d["V"] = (0.0, 0.0)
        for k in d:
            d[k] = (d[k][0], 0.0)
    K = K1 if dim == 1 else K2
    N = K + dim
    h = 1e-30

    def grad(ax):
        Wc = W_from_prim(rho + 1j * h * d["rho"][ax], U + 1j * h * d["U"][ax],
                         V + 1j * h * d["V"][ax], p + 1j * h * d["p"][ax], dim)
        return Wc.imag / h

    W0 = W_from_prim(rho, U, V, p, dim)
    Wx = grad(0)
    Wy = grad(1) if dim == 2 else None
    f = _fields(dim, W0, Wx, None, Wy)
    inv = oracle.point(dim, GAM, 0.0, 1.0, f, 1e-3)["F"]
    vis = oracle.point(dim, GAM, mu, Pr, f, 1e-3)["F"]
    Ux, Vx = d["U"][0], d["V"][0]
    Uy, Vy = d["U"][1], d["V"][1]
    sxx = mu * (2 * Ux - 2.0 / N * (Ux + Vy))
    sxy = mu * (Uy + Vx)
    dT = (d["p"][0] * rho - p * d["rho"][0]) / rho ** 2
    qx = -mu * (N + 2) / 2 * dT
    expect = np.zeros(dim + 2)
    expect[1] = -sxx
    if dim == 2:
        expect[2] = -sxy
    expect[-1] = -(sxx * U + sxy * V) + qx / Pr
    np.testing.assert_allclose(vis - inv, expect, atol=1e-13)


def test_collision_value_is_half_space_sum():
    """Reading R23: W0 = int_{u>0} psi g_l + int_{u<0} psi g_r, checked by quadrature (1D)."""
    Wl = W_from_prim(1.0, 0.2, 0.0, 1.0, 1)
    Wr = W_from_prim(0.6, -0.1, 0.0, 0.5, 1)
    z = np.zeros(3)
    out = oracle.point(1, GAM, 0.0, 1.0, dict(W0=(Wl + Wr) / 2, Wl=Wl, Wr=Wr, W0x=z, Wlx=z, Wrx=z, W0xx=z), 1e-3)

    def half(W, lo, hi):
        rho, U, _, p = prim(W, 1)
        lam = rho / (2 * p)
        g = lambda u: rho * math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
        m0 = quad(g, lo, hi, epsabs=1e-15, epsrel=1e-14)[0]
        m1 = quad(lambda u: u * g(u), lo, hi, epsabs=1e-15, epsrel=1e-14)[0]
        m2 = quad(lambda u: u * u * g(u), lo, hi, epsabs=1e-15, epsrel=1e-14)[0]
        return np.array([m0, m1, 0.5 * (m2 + K1 / (2 * lam) * m0)])
    ref = half(Wl, 0, np.inf) + half(Wr, -np.inf, 0)
    np.testing.assert_allclose(out["W0"], ref, atol=1e-12)


def test_noneq_terms_vanish_for_identical_states():
    """With g_l = g_r = g0 and equal slopes the three e^{-t/tau} terms of Eq.
    (3rd-simplify-flux) cancel: the flux is independent of the collision time."""
    W0 = W_from_prim(1.0, 0.3, 0.0, 1.0, 1)
    Wx = np.array([0.2, 0.1, 0.3])
    f = _fields(1, W0, Wx)
    a = oracle.point(1, GAM, 0.0, 1.0, f, 1e-3)
    b = oracle.point(1, GAM, 0.0, 1.0, f, 1e-1)
    np.testing.assert_allclose(a["F"], b["F"], atol=1e-13)
    np.testing.assert_allclose(a["Ft"], b["Ft"], atol=1e-12)


def test_free_transport_limit():
    """tau_n -> infinity (mu huge, no jump): the non-equilibrium branch dominates and the
    flux tends to the collisionless (kinetic flux-vector split) flux of g_l, g_r."""
    Wl = W_from_prim(1.0, 0.2, 0.0, 1.0, 1)
    Wr = W_from_prim(0.8, -0.1, 0.0, 0.9, 1)
    z = np.zeros(3)
    dt = 1e-6
    # mu large but bracket off via literal tau_mode? use mu large, Pr = 1; bracket terms
    # are proportional to zero gradients here, so only the exponential branch matters
    out = oracle.point(1, GAM, 1e3, 1.0, dict(W0=Wl, Wl=Wl, Wr=Wr, W0x=z, Wlx=z, Wrx=z, W0xx=z), dt)

    def half_flux(W, lo, hi):
        rho, U, _, p = prim(W, 1)
        lam = rho / (2 * p)
        g = lambda u: rho * math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
        m1 = quad(lambda u: u * g(u), lo, hi, epsabs=1e-15, epsrel=1e-14)[0]
        m2 = quad(lambda u: u * u * g(u), lo, hi, epsabs=1e-15, epsrel=1e-14)[0]
        m3 = quad(lambda u: u ** 3 * g(u), lo, hi, epsabs=1e-15, epsrel=1e-14)[0]
        return np.array([m1, m2, 0.5 * (m3 + K1 / (2 * lam) * m1)])
    ref = half_flux(Wl, 0, np.inf) + half_flux(Wr, -np.inf, 0)
    np.testing.assert_allclose(out["F"], ref, rtol=1e-6, atol=1e-9)
