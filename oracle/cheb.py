"""Chebyshev machinery of the fiber discretisation (oracle; test infrastructure).

Sec. 3.1.3 (Eq. cheb-basis): a centreline is X(alpha) = sum_k Xhat_k T_k(alpha)
on alpha in [-1, 1] with collocation points alpha_k = cos(k pi / p),
k = 0..p (N = p + 1 points, endpoints included).  Derivatives are exact
operations on the coefficient series (Sec. 3.1.3) and smooth integrals use
Clenshaw-Curtis weights (Sec. 3.1.4).

Everything here is built from numpy.polynomial.chebyshev (evaluation,
differentiation, integration) and dense linear solves: slow and plain.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import chebyshev as C


def nodes(N: int) -> np.ndarray:
    """alpha_k = cos(k pi/(N-1)), k = 0..N-1 (Sec. 3.1.3)."""
    return np.cos(np.pi * np.arange(N) / (N - 1))


def first_kind(M: int) -> np.ndarray:
    """M Chebyshev points of the first kind, cos((2j+1) pi / (2M)); the
    rectangular-collocation row points (velocity rows: M = N-4, tension rows:
    M = N-2) (Sec. 3.1.3)."""
    return np.cos(np.pi * (2.0 * np.arange(M) + 1.0) / (2.0 * M))


def vander(x: np.ndarray, n: int) -> np.ndarray:
    """V[i, j] = T_j(x_i), j < n (Sec. 3.1.3, Eq. cheb-basis)."""
    return C.chebvander(np.asarray(x, float), n - 1)


def values_to_coeffs(values: np.ndarray) -> np.ndarray:
    """Chebyshev coefficients of the degree N-1 interpolant of nodal values
    (rows = nodes), by solving the Chebyshev-Vandermonde system exactly (Sec. 3.1.3)."""
    N = values.shape[0]
    return np.linalg.solve(vander(nodes(N), N), values)


def cc_weights(N: int) -> np.ndarray:
    """Clenshaw-Curtis weights on the N nodes (Sec. 3.1.4): w = integral over
    [-1,1] of each Lagrange cardinal function, i.e. V^T w = moments with
    moment_j = int T_j = 2/(1-j^2) for even j, 0 for odd j."""
    mom = np.zeros(N)
    j = np.arange(0, N, 2).astype(float)
    mom[0::2] = 2.0 / (1.0 - j * j)
    return np.linalg.solve(vander(nodes(N), N).T, mom)


def series_at(coef: np.ndarray, x, m: int = 0) -> np.ndarray:
    """m-th alpha-derivative of the series `coef` [n, 3] at the points x -> [len(x), 3] (Sec. 3.1.3)."""
    x = np.atleast_1d(np.asarray(x, float))
    c = C.chebder(coef, m, axis=0) if m > 0 else coef
    if c.shape[0] == 0:
        return np.zeros((x.shape[0], coef.shape[1]))
    return C.chebval(x, c, tensor=True).T


def nodal_deriv_matrix(N: int, x: np.ndarray, m: int) -> np.ndarray:
    """Matrix mapping nodal values at the N nodes to the m-th derivative of
    their interpolant at the points x (Sec. 3.1.3; D_s = (2/L) D_alpha, Sec. 3.2)."""
    cols = []
    Vinv = np.linalg.inv(vander(nodes(N), N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        cj = C.chebder(e, m) if m > 0 else e
        cols.append(C.chebval(np.asarray(x, float), cj) if cj.size else np.zeros(len(x)))
    Tm = np.stack(cols, axis=1)          # [len(x), N]: T_j^{(m)}(x)
    return Tm @ Vinv


def integrated_T(j: int, m: int) -> np.ndarray:
    """Coefficients of I^m T_j: m-fold integral of T_j from alpha = -1 (each
    antiderivative vanishes at -1) (Sec. 3.1.3, Eq. cheb-basis)."""
    e = np.zeros(j + 1)
    e[j] = 1.0
    return C.chebint(e, m, lbnd=-1.0)


# ---------------------------------------------------------- extended precision
LD = np.longdouble
PI_LD = LD("3.141592653589793238462643383279502884197")


def nodes_ld(N: int) -> np.ndarray:
    """The N collocation nodes cos(k pi/(N-1)) in numpy.longdouble (Sec. 3.1.3)."""
    return np.cos(PI_LD * np.arange(N, dtype=LD) / LD(N - 1))


def first_kind_ld(M: int) -> np.ndarray:
    """The M first-kind points in numpy.longdouble (Sec. 3.1.3)."""
    return np.cos(PI_LD * (LD(2) * np.arange(M, dtype=LD) + LD(1)) / LD(2 * M))


def solve_ld(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Gaussian elimination with partial pivoting in numpy.longdouble, for the
    extended-precision geometry of Sec. 3.1.3."""
    A = np.array(A, dtype=LD)
    B = np.array(B, dtype=LD)
    n = A.shape[0]
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if p != k:
            A[[k, p]] = A[[p, k]]
            B[[k, p]] = B[[p, k]]
        f = A[k + 1:, k] / A[k, k]
        A[k + 1:, k:] -= f[:, None] * A[k, k:][None, :]
        B[k + 1:] -= f[:, None] * B[k][None, :]
    X = np.zeros_like(B)
    for k in range(n - 1, -1, -1):
        X[k] = (B[k] - A[k, k + 1:] @ X[k + 1:]) / A[k, k]
    return X


def interp_derivs_ext(values: np.ndarray, pts: np.ndarray, m: int) -> np.ndarray:
    """m-th derivative at pts of the degree N-1 interpolant of nodal values
    [N, 3], computed in extended precision (numpy.longdouble): values are taken
    relative to the first node, the Chebyshev-Vandermonde system is solved by
    Gaussian elimination, then differentiated and evaluated with
    numpy.polynomial.chebyshev.  Returns float64 [len(pts), 3] (Sec. 3.1.3, in extended precision)."""
    N = values.shape[0]
    v = np.asarray(values, dtype=LD)
    v = v - v[0][None, :]
    V = C.chebvander(nodes_ld(N), N - 1)
    coef = solve_ld(V, v)
    c = C.chebder(coef, m, axis=0) if m > 0 else coef
    pts = np.atleast_1d(np.asarray(pts, dtype=LD))
    out = C.chebval(pts, c, tensor=True).T
    if m == 0:
        out = out + np.asarray(values, dtype=LD)[0][None, :]
    return out.astype(np.float64)


def basis_V(N: int):
    """Unknown basis for one velocity component (Sec. 3.1.3 representation,
    integrated form): columns are I^4 T_0 .. I^4 T_{N-5}, then T_0..T_3, so
    V = I^4 sigma + cubic lies in P_{N-1}."""
    return [integrated_T(j, 4) for j in range(N - 4)] + [integrated_T(k, 0) for k in range(4)]


def basis_T(N: int):
    """Unknown basis for the tension: I^2 T_0 .. I^2 T_{N-3}, then T_0, T_1 (Sec. 3.1.3, Eq. cheb-basis)."""
    return [integrated_T(j, 2) for j in range(N - 2)] + [integrated_T(k, 0) for k in range(2)]


def basis_matrix(basis, x: np.ndarray, m: int = 0) -> np.ndarray:
    """[len(x), len(basis)]: m-th derivative of each basis function at x (Sec. 3.1.3, Eq. cheb-basis)."""
    x = np.atleast_1d(np.asarray(x, float))
    out = np.zeros((x.shape[0], len(basis)))
    for j, c in enumerate(basis):
        cm = C.chebder(c, m) if m > 0 else c
        out[:, j] = C.chebval(x, cm) if cm.size else 0.0
    return out
