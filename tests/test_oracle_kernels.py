"""Pins of the oracle's direct sums (oracle/pairsum.c) against textbook
properties of the Stokes fundamental solutions (Sec. 2, Eqs. oseen,
stresslet, double-layer) and of the sphere quadrature inputs (Sec. 3.1.1)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import kernels


def point_u(x, y, F, mu=1.0):
    return kernels.stokeslet(np.atleast_2d(x), np.atleast_2d(y), np.atleast_2d(F), mu)


def test_stokeslet_textbook_axial_and_transverse():
    # a point force F drives velocity F/(4 pi mu r) along its line of action
    # and F/(8 pi mu r) perpendicular to it
    mu, r = 2.5, 3.0
    F = np.array([0.0, 0.0, 1.7])
    ua = point_u([0, 0, r], [0, 0, 0], F, mu)[0]
    ut = point_u([r, 0, 0], [0, 0, 0], F, mu)[0]
    assert np.allclose(ua, F / (4 * math.pi * mu * r), rtol=1e-14)
    assert np.allclose(ut, F / (8 * math.pi * mu * r), rtol=1e-14)


def _fd_grad(fun, x, h=1e-4):
    """Central-difference Jacobian d fun_i / d x_j (4th order)."""
    J = np.zeros((3, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        J[:, j] = (-fun(x + 2 * e) + 8 * fun(x + e) - 8 * fun(x - e) + fun(x - 2 * e)) / (12 * h)
    return J


def test_stokeslet_divergence_free_and_momentum_balance():
    """u = G(x - y) F satisfies div u = 0 and mu lap u = grad p with the
    textbook Stokeslet pressure p = F.r / (4 pi r^3); the traction of
    sigma = -p I + mu (grad u + grad u^T) through any sphere around y is F in
    magnitude (unit point force normalisation)."""
    rng = np.random.default_rng(0)
    mu = 1.3
    y = rng.normal(size=3)
    F = rng.normal(size=3)
    u = lambda x: point_u(x, y, F, mu)[0]
    p = lambda x: F @ (x - y) / (4 * math.pi * np.linalg.norm(x - y) ** 3)
    for _ in range(4):
        x = y + rng.normal(size=3) * 2
        J = _fd_grad(u, x)
        assert abs(np.trace(J)) < 1e-9 * np.abs(J).max()
        h = 1e-3
        lap = np.zeros(3)
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            lap += (u(x + e) - 2 * u(x) + u(x - e)) / h ** 2
        gp = _fd_grad(lambda z: np.array([p(z)] * 3), x)[0]
        assert np.allclose(mu * lap, gp, rtol=1e-4, atol=1e-6 * np.abs(gp).max())
    # traction through a sphere of radius 0.7 around y (Gauss-Legendre x trapezoid)
    R = 0.7
    xt, wt = np.polynomial.legendre.leggauss(24)
    nph = 48
    total = np.zeros(3)
    for ct, w in zip(xt, wt):
        st = math.sqrt(1 - ct * ct)
        for k in range(nph):
            ph = 2 * math.pi * k / nph
            n = np.array([st * math.cos(ph), st * math.sin(ph), ct])
            x = y + R * n
            J = _fd_grad(u, x, h=1e-5)
            sig = -p(x) * np.eye(3) + mu * (J + J.T)
            total += w * (2 * math.pi / nph) * R * R * sig @ n
    assert abs(np.linalg.norm(total) - np.linalg.norm(F)) < 1e-6 * np.linalg.norm(F)


def test_stokeslet_fiber_skip_and_symmetry():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(40, 3)) * 3
    fid = np.repeat(np.arange(8), 5).astype(np.int32)
    a, b = rng.normal(size=(40, 3)), rng.normal(size=(40, 3))
    # <a, G b> = <G a, b> (G is symmetric and even in r)
    lhs = np.sum(a * kernels.stokeslet(X, X, b, 1.0, fid, fid))
    rhs = np.sum(kernels.stokeslet(X, X, a, 1.0, fid, fid) * b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # skipping same-fiber pairs equals summing fiber by fiber over the others
    full = kernels.stokeslet(X, X, b, 1.0, fid, fid)
    for m in range(8):
        t = fid == m
        s = fid != m
        assert np.allclose(full[t], kernels.stokeslet(X[t], X[s], b[s], 1.0), rtol=1e-13)


def test_stokeslet_translation_rotation_invariance():
    rng = np.random.default_rng(2)
    X, F = rng.normal(size=(30, 3)), rng.normal(size=(30, 3))
    fid = np.repeat(np.arange(6), 5).astype(np.int32)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    u = kernels.stokeslet(X, X, F, 1.0, fid, fid)
    u2 = kernels.stokeslet(X @ Q.T + 5.0, X @ Q.T + 5.0, F @ Q.T, 1.0, fid, fid)
    assert np.allclose(u2, u @ Q.T, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("nt,nph", [(8, 16), (16, 48)])
def test_sphere_quadrature_moments(nt, nph):
    R = 2.0
    b = wl.sphere_quadrature(R, nt, nph)
    assert b.nodes.shape[0] == nt * nph * 16
    assert abs(b.weights.sum() - 4 * math.pi * R * R) < 1e-12 * 4 * math.pi * R * R
    nn = np.einsum("i,ia,ib->ab", b.weights, b.normals, b.normals)
    assert np.allclose(nn, 4 * math.pi * R * R / 3 * np.eye(3), atol=1e-11)
    assert np.allclose(np.linalg.norm(b.nodes, axis=1), R)


def test_double_layer_gauss_identity():
    """Double layer of a constant density c: c inside, 0 outside (Sec. 3.1.2
    identity); its fluid-side (interior) limit on the surface is c, and
    N[c] = 0 because the normals integrate to zero."""
    b = wl.sphere_quadrature(1.0, 16, 32)
    c = np.array([0.3, -1.2, 0.7])
    q = np.tile(c, (b.nodes.shape[0], 1))
    inside = np.array([[0, 0, 0], [0.3, -0.2, 0.1], [0.0, 0.5, 0.0]])
    outside = np.array([[0, 0, 3.0], [2.0, -1.0, 0.5]])
    ui = kernels.stresslet(inside, b.nodes, b.normals, b.weights, q)
    uo = kernels.stresslet(outside, b.nodes, b.normals, b.weights, q)
    assert np.allclose(ui[0], c, atol=1e-12)          # exact at the centre
    assert np.allclose(ui, c, atol=2e-6)
    assert np.allclose(uo, 0.0, atol=1e-6)
    us = kernels.surface_self(b.nodes, b.normals, b.weights, q)
    assert np.allclose(us, c, atol=1e-10)


def test_surface_diag_matches_operator():
    b = wl.sphere_quadrature(1.0, 2, 4)
    n = b.nodes.shape[0]
    d = kernels.surface_diag(b.nodes, b.normals, b.weights)
    for i in [0, 7, n - 1]:
        for a in range(3):
            e = np.zeros((n, 3))
            e[i, a] = 1.0
            col = kernels.surface_self(b.nodes, b.normals, b.weights, e)
            assert abs(col[i, a] - d[i, a]) < 1e-13


@pytest.mark.parametrize("mu", [1.0, 2.5])
def test_confined_point_force_at_centre(mu):
    """A point force F at the centre of a no-slip sphere of radius R: the
    periphery equation (Eq. main-cortex-density) must give the interior image
    flow u^c = (1/8 pi mu)[-(3/R) I + (2 r^2 I - x x)/R^3] F (the Stokes flow
    that cancels G F on |x| = R), to quadrature accuracy, converging with
    refinement.  At mu != 1 this also fixes the stresslet's scaling: the
    equation's identity term q/2 does not scale with 1/mu, so a stresslet
    carrying 1/mu would miss the closed form."""
    import scipy.sparse.linalg as sla
    R = 2.0
    F = np.array([0.4, -0.3, 1.0])
    pts = np.array([[0.0, 0.0, 0.0], [0.5, 0.2, -0.3], [-0.8, 0.4, 0.6]])

    def exact(x):
        r2 = x @ x
        return (-(3 / R) * F + (2 * r2 * F - x * (x @ F)) / R ** 3) / (8 * math.pi * mu)

    errs = []
    for nt, nph in [(4, 8), (8, 16)]:
        b = wl.sphere_quadrature(R, nt, nph)
        n = b.nodes.shape[0]
        rhs = -point_u(b.nodes, np.zeros(3), F, mu).reshape(-1)
        op = sla.LinearOperator((3 * n, 3 * n), dtype=float,
                                matvec=lambda v: kernels.surface_self(b.nodes, b.normals, b.weights,
                                                                     v.reshape(-1, 3)).reshape(-1))
        q, info = sla.gmres(op, rhs, rtol=1e-12, atol=0.0, restart=100, maxiter=200)
        assert info == 0
        uc = kernels.stresslet(pts, b.nodes, b.normals, b.weights, q.reshape(-1, 3))
        ex = np.array([exact(x) for x in pts])
        errs.append(np.abs(uc - ex).max() / np.abs(ex).max())
    assert errs[1] < 2e-3 and errs[1] < errs[0] / 2
