"""Pins of the oracle's fiber discretisation and implicit step (oracle/fiber.py,
oracle/system.py) against closed forms derived from the paper's equations
(Eqs. main-sb-local, sb-stokes-reg, main-elastic-force, main-inextensibility,
bc-free; Sec. 3.2), invariants and brute force."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import cheb, system


def c_log(eps):
    return -math.log(eps * eps * math.e)


def straight(N, L, d, centre=(0.0, 0.0, 0.0)):
    a = cheb.nodes(N)
    d = np.asarray(d, float) / np.linalg.norm(d)
    return np.asarray(centre)[None, :] + (a[:, None] * L / 2.0) * d[None, :], d


def arclength(N, L):
    return (cheb.nodes(N) + 1.0) * L / 2.0


@pytest.mark.parametrize("lsb", [False, True])
@pytest.mark.parametrize("N", [12, 32])
def test_straight_rod_uniform_force_closed_form(N, lsb):
    """Straight rod, uniform f^E, no bending: V = M f^E exactly and T = 0;
    perpendicular mobility (c+2)/(8 pi mu), parallel 2c/(8 pi mu) (K_delta
    vanishes identically here); drag ratio 2c/(c+2) -> 2 as eps -> 0."""
    mu, eps, L = 1.7, 1e-3, 2.3
    X, d = straight(N, L, [1.0, 2.0, -0.5], [3.0, 1.0, 2.0])
    rng = np.random.default_rng(0)
    fe = rng.normal(size=3)
    S = system.System(X, [L], [N], np.tile(fe, (N, 1)), mu=mu, eps=eps, lsb=lsb)
    r = S.step(tol=1e-13)
    c = c_log(eps)
    fpar = (fe @ d) * d
    expect = (2 * c * fpar + (c + 2) * (fe - fpar)) / (8 * math.pi * mu)
    assert np.allclose(r.V, expect[None, :], rtol=1e-10, atol=1e-12)
    assert np.abs(r.T).max() < 1e-9
    assert abs((c + 2) / (8 * math.pi) - 0.589490) < 5e-7
    assert abs(2 * c / (8 * math.pi) - 1.019826) < 5e-7
    assert abs(2 * c / (c + 2) - 1.730013) < 5e-7


@pytest.mark.parametrize("lsb", [False, True])
def test_straight_rod_axial_stretch_tension(lsb):
    """Axial external force f0 (s - L/2)/L t on a straight rod: inextensibility
    forces V = 0 and the tension balances it, T_s = -f^E.t with T(0)=T(L)=0, so
    T(s) = f0 s (L - s) / (2 L) (Eqs. force-balance, main-elastic-force, bc-free)."""
    N, L, f0 = 24, 2.0, 3.0
    X, d = straight(N, L, [0.3, -0.4, 0.8])
    s = arclength(N, L)
    fe = (f0 * (s - L / 2) / L)[:, None] * d[None, :]
    r = system.System(X, [L], [N], fe, lsb=lsb).step(tol=1e-13)
    assert np.abs(r.V).max() < 1e-9
    assert np.allclose(r.T, f0 * s * (L - s) / (2 * L), atol=1e-9)


def test_straight_rod_rigid_rotation():
    """Transverse force linear in s on a straight rod (local theory): V = M f^E,
    a rigid rotation about the midpoint; no bending, T = 0."""
    N, L, eps = 20, 2.0, 1e-2
    X, d = straight(N, L, [0.0, 0.0, 1.0])
    s = arclength(N, L)
    fe = np.zeros((N, 3))
    fe[:, 0] = 2.0 * (s - L / 2)
    r = system.System(X, [L], [N], fe, eps=eps, lsb=True).step(tol=1e-13)
    assert np.allclose(r.V[:, 0], (c_log(eps) + 2) / (8 * math.pi) * fe[:, 0], rtol=1e-10, atol=1e-12)
    assert np.abs(r.T).max() < 1e-9


def beam_mode(s, L):
    kL = 4.730040744862704
    k = kL / L
    beta = (math.cosh(kL) - math.cos(kL)) / (math.sinh(kL) - math.sin(kL))
    return np.cosh(k * s) + np.cos(k * s) - beta * (np.sinh(k * s) + np.sin(k * s)), k


@pytest.mark.parametrize("N", [16, 32])
def test_free_free_beam_mode_relaxation(N):
    """Small-amplitude first free-free mode (kL = 4.7300407...) of a straight
    rod relaxes in one backward-Euler step by 1/(1 + dt (c+2) E k^4/(8 pi mu))
    (local theory; Eqs. main-sb-local, EB-force, bc-free; implicit bending)."""
    L, E, dt, eps, A = 2.0, 1.0, 1e-3, 1e-3, 1e-7
    X, d = straight(N, L, [0.0, 0.0, 1.0])
    s = arclength(N, L)
    phi, k = beam_mode(s, L)
    X = X.copy()
    X[:, 0] += A * phi
    r = system.System(X, [L], [N], np.zeros((N, 3)), E=E, dt=dt, eps=eps, lsb=True).step(tol=1e-14)
    factor = 1.0 / (1.0 + dt * (c_log(eps) + 2) * E * k ** 4 / (8 * math.pi))
    amp_new = X[:, 0] + dt * r.V[:, 0]
    assert np.allclose(amp_new, factor * A * phi, rtol=0, atol=1e-6 * A)


def test_regularised_self_term_large_delta_closed_form():
    """K_delta (Eq. sb-stokes-reg) on a straight rod with transverse force
    f(s) = (s - L/2) e: K[f](s).e = (1/8 pi mu)[sqrt((L-s)^2+d^2) - sqrt(s^2+d^2)];
    with delta = L the integrand is smooth and Clenshaw-Curtis is exact to
    rounding at N = 40."""
    N, L, mu = 40, 2.0, 1.0
    X, d = straight(N, L, [0.0, 1.0, 0.0])
    s = arclength(N, L)
    S_on = system.System(X, [L], [N], np.zeros((N, 3)), delta_over_L=1.0).fibers[0]
    S_off = system.System(X, [L], [N], np.zeros((N, 3)), lsb=True).fibers[0]
    f = np.zeros((N, 3))
    f[:, 0] = s - L / 2
    K = S_on.from_cm((S_on.S - S_off.S) @ S_on.to_cm(f))
    delta = L
    exact = (np.sqrt((L - s) ** 2 + delta ** 2) - np.sqrt(s ** 2 + delta ** 2)) / (8 * math.pi * mu)
    assert np.allclose(K[:, 0], exact, atol=1e-12)
    assert np.abs(K[:, 1:]).max() < 1e-13


def test_single_fiber_one_gmres_iteration():
    """An isolated fiber has P^-1 A = I (Eq. prec uses the exact self block),
    so GMRES stops after one iteration, up to the block's conditioning."""
    s = wl.free_space(1, 32, 1.0, seed=4, curved_amp=0.05)
    r = system.from_suspension(s).step(tol=1e-8)
    assert r.iters == 1 and r.resid < 1e-8


def test_affine_in_external_force():
    """V(f1 + f2) = V(f1) + V(f2) - V(0): the step is affine in f^E."""
    s = wl.free_space(4, 16, 3.0, seed=5, curved_amp=0.05)
    f1, f2 = s.f_ext, np.random.default_rng(9).normal(size=s.f_ext.shape)

    def V(fe):
        s.f_ext = fe
        return system.from_suspension(s).step(tol=1e-13).V

    assert np.allclose(V(f1 + f2), V(f1) + V(f2) - V(0 * f1), rtol=1e-9, atol=1e-9)


def test_rotation_translation_invariance():
    """Rotating and translating all inputs rotates the velocities."""
    s = wl.free_space(5, 16, 4.0, seed=6, curved_amp=0.05)
    r0 = system.from_suspension(s).step(tol=1e-13)
    Q, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))
    s.X = s.X @ Q.T + np.array([7.0, -3.0, 11.0])
    s.f_ext = s.f_ext @ Q.T
    r1 = system.from_suspension(s).step(tol=1e-13)
    assert np.allclose(r1.V, r0.V @ Q.T, rtol=1e-8, atol=1e-8 * np.abs(r0.V).max())
    assert np.allclose(r1.T, r0.T, rtol=1e-8, atol=1e-8 * np.abs(r0.T).max())


def test_gmres_matches_dense_solve_brute_force():
    """Assemble A column by column (2-3 fibers + a small periphery), solve with
    LAPACK, compare with preconditioned GMRES."""
    s = wl.confined(3, 10, R=3.0, R_centres=1.5, n_theta=2, n_phi=3, seed=7)
    S = system.from_suspension(s)
    n = S.n_unknowns
    A = np.stack([S.matvec(e) for e in np.eye(n)], axis=1)
    b = S.rhs()
    u_dense = np.linalg.solve(A, b)
    u_gm, its, res = S.gmres(b, 1e-14)
    assert np.linalg.norm(u_gm - u_dense) <= 1e-11 * np.linalg.norm(u_dense)


def test_far_apart_fibers_point_force_coupling():
    """Two fibers far apart: fiber 1's velocity change due to fiber 2 is the
    Stokeslet of fiber 2's total force, G(D) F_2, to O(L/D)."""
    N, L, D = 16, 2.0, 400.0
    X1, _ = straight(N, L, [1, 0, 0])
    X2, _ = straight(N, L, [0, 1, 1], [D, 0.0, 0.0])
    f2 = np.tile([0.0, 0.0, 1.0], (N, 1))
    X = np.concatenate([X1, X2])
    fe = np.concatenate([np.zeros((N, 3)), f2])
    r = system.System(X, [L, L], [N, N], fe).step(tol=1e-13)
    F2 = np.array([0.0, 0.0, L])                    # total force of fiber 2
    uG = F2 / (8 * math.pi * D)                      # transverse Stokeslet at distance D
    assert np.allclose(r.V[:N].mean(0), uG, rtol=2 * L / D, atol=1e-9)


def test_confined_no_slip_on_wall():
    """Fibers inside a sphere: the total flow (fiber Stokeslets + periphery
    double layer) nearly vanishes just inside the wall, compared with the
    fibers' own flow there."""
    s = wl.confined(4, 12, R=4.0, R_centres=1.0, n_theta=8, n_phi=16, seed=8)
    S = system.from_suspension(s)
    r = S.step(tol=1e-12)
    from oracle import kernels
    b = s.boundary
    probe = 0.9 * b.nodes[::97]
    f = np.concatenate([fb.f_lin(S._split(r.u)[0][m]) + fb.f_known for m, fb in enumerate(S.fibers)])
    uf = kernels.stokeslet(probe, s.X, f * S.Wall[:, None], 1.0)
    uc = kernels.stresslet(probe, b.nodes, b.normals, b.weights, r.q)
    uf_w = kernels.stokeslet(b.nodes[::97] * 1.0, s.X, f * S.Wall[:, None], 1.0)
    assert np.linalg.norm(uf + uc) < 0.25 * np.linalg.norm(uf)
    # at the quadrature nodes themselves the discrete equation holds exactly
    us = kernels.surface_self(b.nodes, b.normals, b.weights, r.q)[::97]
    assert np.allclose(us + uf_w, 0.0, atol=1e-7 * np.abs(uf_w).max())


def _compatible_curve(alpha, L, k0, frame, centre):
    """Planar centreline with curvature k0 sin^4(pi s / L): zero, with its
    first derivatives, at both ends, so it meets the free-end conditions
    X_ss = X_sss = 0 (Eq. bc-free).  Arclength-parametrised by integrating the
    tangent angle with Gauss-Legendre quadrature."""
    gx, gw = np.polynomial.legendre.leggauss(80)
    kappa = lambda u: k0 * np.sin(np.pi * u / L) ** 4

    def theta(u):
        return 0.5 * u * np.sum(gw * kappa(0.5 * u * (gx + 1.0)))

    pts = []
    for s in (alpha + 1.0) * L / 2.0:
        th = np.array([theta(x) for x in 0.5 * s * (gx + 1.0)])
        pts.append([0.5 * s * np.sum(gw * np.cos(th)), 0.5 * s * np.sum(gw * np.sin(th)), 0.0])
    return np.asarray(centre) + np.array(pts) @ frame


def test_spectral_convergence_in_N():
    """Two interacting curved fibers whose initial shape meets the free-end
    conditions, under a uniform load, local slender-body theory: the step's
    velocity and tension, interpolated to common points, converge
    geometrically in N (measured against N = 48: V 4e-4, 6e-7, 1e-9 and T
    2e-2, 1e-4, 6e-7 at N = 16, 24, 32).  A curve with curvature at a free
    end breaks those conditions: its tension then carries a mode that grows
    like N^2 and V converges only algebraically, so the input must be
    compatible.  With K_delta the node quadrature resolves the kernel's
    width delta = 0.01 L only near N ~ 160, and V converges algebraically
    (1e-3, 4e-4, 1.5e-4)."""
    from numpy.polynomial import chebyshev as C
    L = 2.0
    frames = [np.eye(3), np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], float)]
    centres = [np.zeros(3), np.array([0.5, 1.2, -0.6])]
    probe = np.linspace(-1.0, 1.0, 11)

    def run(N):
        a = cheb.nodes(N)
        X = np.concatenate([_compatible_curve(a, L, 0.8, fr, c) for fr, c in zip(frames, centres)])
        f = np.tile([0.3, -0.2, -1.0], (X.shape[0], 1))
        r = system.System(X, np.full(2, L), np.full(2, N, np.int32), f, 1.0, 1e-3, 1.0, 1e-2, 0.01,
                          True).step(tol=1e-14)
        V, T = r.V.reshape(2, N, 3), r.T.reshape(2, N)
        Vi = np.concatenate([np.stack([C.chebval(probe, C.chebfit(a, V[m, :, k], N - 1)) for k in range(3)], -1)
                             for m in range(2)])
        Ti = np.concatenate([C.chebval(probe, C.chebfit(a, T[m], N - 1)) for m in range(2)])
        return Vi, Ti

    Vr, Tr = run(48)
    eV, eT = [], []
    for N in (16, 24, 32):
        V, T = run(N)
        eV.append(np.linalg.norm(V - Vr) / np.linalg.norm(Vr))
        eT.append(np.linalg.norm(T - Tr) / np.linalg.norm(Tr))
    assert eV[1] < eV[0] / 100 and eV[2] < eV[1] / 100 and eV[2] < 1e-8, eV
    assert eT[1] < eT[0] / 30 and eT[2] < eT[1] / 30 and eT[2] < 1e-5, eT


def test_multistep_growth_of_a_curved_end_fiber_at_64_points():
    """The divergence of multi-step runs belongs to the discrete method, not
    to an implementation: one free curved fiber (the workloads' recipe, whose
    ends carry curvature against Eq. bc-free), a uniform load, dt = 1e-3,
    stepped by the oracle alone.  At N = 64 its tension grows about 600-fold
    in seven steps (17 -> 1e4); the same fiber at N = 32 keeps it within 10 % (it relaxes, 2.8 -> 2.7)."""
    def run(N):
        s = wl.free_space(1, N, 5.0, seed=0, curved_amp=0.05, L_range=(2.5, 3.0))
        s.f_ext = np.tile(np.random.default_rng(0).normal(size=3), (N, 1))
        X, T = s.X.copy(), []
        for _ in range(7):
            sub = wl.Suspension(s.n_per_fiber, X, s.L, s.f_ext, s.mu, s.eps, s.E, s.dt)
            r = system.from_suspension(sub).step(tol=1e-12)
            X = r.X_new
            T.append(np.abs(r.T).max())
        return T
    T64, T32 = run(64), run(32)
    assert T64[-1] > 100.0 * T64[0]
    assert max(T32) < 1.1 * min(T32)


def test_block_sensitivity_by_points_per_fiber():
    """The conditioning gate of the discretisation (rectangular collocation in
    the integrated basis): the relative change of a single fiber's velocities
    when every entry of its block is perturbed by a relative 1e-16 (four
    random sign patterns, the largest change).  Recorded: 3.1e-13, 3.7e-12,
    7.4e-10, 2.1e-6 at N = 16, 32, 64, 128 (block condition numbers 7e6,
    1e9, 6e11, 9e14); a discretisation change that worsens them by 5x fails."""
    rng = np.random.default_rng(0)
    recorded = {16: 3.1e-13, 32: 3.7e-12, 64: 7.4e-10, 128: 2.1e-6}
    for N, rec in recorded.items():
        s = wl.free_space(1, N, 5.0, seed=3, curved_amp=0.05, L_range=(2.0, 2.0))
        s.f_ext = np.tile([0.3, -0.2, -1.0], (N, 1))
        S = system.from_suspension(s)
        fb = S.fibers[0]
        b = S.rhs()
        V0 = fb.velocity_nodes(np.linalg.solve(fb.B, b))
        worst = 0.0
        for _ in range(4):
            Bp = fb.B * (1.0 + 1e-16 * rng.choice([-1.0, 1.0], size=fb.B.shape))
            V = fb.velocity_nodes(np.linalg.solve(Bp, b))
            worst = max(worst, np.linalg.norm(V - V0) / np.linalg.norm(V0))
        assert worst <= 5.0 * rec, (N, worst)
