"""Pins of oracle/cheb.py against textbook facts about Chebyshev series and
Clenshaw-Curtis quadrature (Sec. 3.1.3-3.1.4)."""
import numpy as np
import pytest

from oracle import cheb


def test_nodes_are_extrema_with_endpoints():
    x = cheb.nodes(9)
    assert x[0] == 1.0 and abs(x[-1] + 1.0) < 1e-15
    # T_8 has its 9 extrema (+-1) exactly at these points
    assert np.allclose(np.abs(np.cos(8 * np.arccos(np.clip(x, -1, 1)))), 1.0, atol=1e-14)


@pytest.mark.parametrize("M", [4, 7, 30])
def test_first_kind_points_are_roots(M):
    y = cheb.first_kind(M)
    assert np.allclose(np.cos(M * np.arccos(y)), 0.0, atol=1e-13)


def test_coeffs_of_cubic_textbook():
    # x^3 = (3 T_1 + T_3) / 4
    x = cheb.nodes(6)
    c = cheb.values_to_coeffs(np.stack([x ** 3] * 3, axis=1))[:, 0]
    assert np.allclose(c, [0, 0.75, 0, 0.25, 0, 0], atol=1e-14)


def test_cc_weights_textbook_values():
    # Simpson's rule for N = 3; Trefethen's clencurt(4) for N = 5
    assert np.allclose(cheb.cc_weights(3), [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    assert np.allclose(cheb.cc_weights(5), [1 / 15, 8 / 15, 12 / 15, 8 / 15, 1 / 15], atol=1e-15)


@pytest.mark.parametrize("N", [8, 17, 32, 64])
def test_cc_exact_on_polynomials(N):
    w = cheb.cc_weights(N)
    x = cheb.nodes(N)
    assert abs(w.sum() - 2.0) < 1e-13
    for k in range(0, N, 3):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(w @ x ** k - exact) < 1e-12


def test_cc_spectral_on_smooth():
    # int_{-1}^{1} exp(x) dx = e - 1/e
    w = cheb.cc_weights(20)
    assert abs(w @ np.exp(cheb.nodes(20)) - (np.e - 1 / np.e)) < 1e-14


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
def test_nodal_derivatives_exact_on_polynomials(m):
    N = 12
    pts = np.linspace(-0.95, 0.97, 7)
    D = cheb.nodal_deriv_matrix(N, pts, m)
    f = cheb.nodes(N) ** 7
    expect = {0: pts ** 7, 1: 7 * pts ** 6, 2: 42 * pts ** 5, 3: 210 * pts ** 4, 4: 840 * pts ** 3}[m]
    assert np.allclose(D @ f, expect, rtol=1e-11, atol=1e-10)


@pytest.mark.parametrize("N", [16, 32, 64])
def test_fourth_derivative_of_cubic_is_zero(N):
    # zero bending force for a straight rod / any cubic centreline; the bound
    # is the rounding of the data amplified by the 4th-derivative norm ~ N^8
    x = cheb.nodes(N)
    X = np.stack([1 + 2 * x, x ** 2 - x ** 3, 0.5 * x ** 3], axis=1)
    d4 = cheb.series_at(cheb.values_to_coeffs(X), x, 4)
    assert np.abs(d4).max() < 1e-16 * float(N) ** 8
    d3 = cheb.series_at(cheb.values_to_coeffs(X), [0.3], 3)
    assert np.allclose(d3[0], [0.0, -6.0, 3.0], atol=1e-16 * float(N) ** 6)


def test_integrated_basis_properties():
    N = 16
    BV = cheb.basis_V(N)
    pts = np.linspace(-1, 1, 11)
    # 4th derivative of I^4 T_j is T_j, and I^4 T_j and its first 3 derivatives vanish at -1
    d4 = cheb.basis_matrix(BV, pts, 4)
    for j in range(N - 4):
        assert np.allclose(d4[:, j], np.cos(j * np.arccos(pts)), atol=1e-11)
        for m in range(4):
            assert abs(cheb.basis_matrix(BV, [-1.0], m)[0, j]) < 1e-13
    # the last four columns are T_0..T_3 and have zero 4th derivative
    assert np.abs(d4[:, N - 4:]).max() == 0.0
    BT = cheb.basis_T(N)
    d2 = cheb.basis_matrix(BT, pts, 2)
    for j in range(N - 2):
        assert np.allclose(d2[:, j], np.cos(j * np.arccos(pts)), atol=1e-11)


@pytest.mark.parametrize("N", [16, 32, 64])
def test_extended_precision_derivatives_on_polynomials(N):
    """Derivatives of the interpolant in extended precision are exact on
    polynomials up to the rounding of the double data amplified by N^(2m)."""
    ld_eps = 2.0 * float(np.finfo(np.float64).eps)
    x = cheb.nodes(N)
    X = np.stack([2.0 + 3.0 * x, 1.0 - x ** 3, 0.25 * x ** 5], axis=1)
    pts = np.array([1.0, 0.3, -0.77, -1.0])
    d1 = cheb.interp_derivs_ext(X, pts, 1)
    exact1 = np.stack([3.0 + 0 * pts, -3 * pts ** 2, 1.25 * pts ** 4], 1)
    assert np.abs(d1 - exact1).max() <= max(100 * ld_eps * N ** 2 * 3.0, 1e-15)
    d3 = cheb.interp_derivs_ext(X, pts, 3)
    exact3 = np.stack([0 * pts, -6.0 + 0 * pts, 15 * pts ** 2], 1)
    assert np.abs(d3 - exact3).max() <= max(100 * ld_eps * float(N) ** 6 * 3.0, 1e-14)


@pytest.mark.parametrize("N", [12, 24])
def test_extended_precision_matches_high_precision(N):
    """Against a 40-digit evaluation (mpmath) of the same interpolant on the
    same double data: the extended-precision route adds only its own rounding."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(N)
    x = cheb.nodes(N)
    X = 30.0 + np.stack([np.sin(1.3 * x + 0.2), np.cos(0.7 * x), x ** 2], 1) + 1e-3 * rng.normal(size=(N, 3))
    pts = [1.0, 0.41, -1.0]
    ld_eps = float(np.finfo(np.longdouble).eps)
    xs = [mpmath.cos(mpmath.pi * k / (N - 1)) for k in range(N)]
    V = mpmath.matrix([[mpmath.chebyt(j, xk) for j in range(N)] for xk in xs])
    for m in (1, 2, 3):
        got = cheb.interp_derivs_ext(X, pts, m)
        for a in range(3):
            coef = mpmath.lu_solve(V, mpmath.matrix([mpmath.mpf(float(v)) for v in X[:, a]]))
            # m-th derivative of sum c_j T_j via the polynomial in monomials
            poly = [mpmath.mpf(0)] * N
            for j in range(N):
                tj = mpmath.taylor(lambda t: mpmath.chebyt(j, t), 0, N - 1)
                for i in range(N):
                    poly[i] += coef[j] * tj[i]
            for ip, p in enumerate(pts):
                val = sum(poly[i] * mpmath.ff(i, m) * mpmath.mpf(p) ** (i - m) for i in range(m, N))
                assert abs(got[ip, a] - float(val)) <= 1e-13 + 100 * ld_eps * float(N) ** (2 * m) * 30.0
