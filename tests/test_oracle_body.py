"""Oracle pins for the rigid body and attached fibers (Sec. 2.2-2.3): the
exterior double layer completed by a Stokeslet and a rotlet at the centre
(Eq. main-nsb-second-kind) with the rigid-motion constraints (Eqs.
main-nsb-rgbt, main-nsb-rgbr), fibers clamped or hinged at their minus ends
(Eqs. BC2-1, BC2-2, BC2-T), and the force and torque they exert on the body
(Eqs. f-ext, t-ext).

Pins (none of them re-derives the oracle's own formulas):
* an isolated sphere: Stokes drag U = F / (6 pi mu a) and rotational drag
  Omega = L / (8 pi mu a^3), converging with the surface quadrature;
* a sphere at the centre of a no-slip sphere six times larger: the
  concentric-sphere drag the paper quotes (Eq. concentric-sphere, Happel and
  Brenner), a 57 % correction to Stokes drag;
* six straight fibers along +-x, +-y, +-z clamped (or hinged) to the sphere:
  the reflection symmetries of the configuration give U || F and Omega = 0,
  cubic symmetry an isotropic mobility, and the fibers add drag;
* momentum balance: the force the fibers and the body exert on the fluid
  equals the applied force, and the torque likewise (straight fibers), which
  fixes the sign and size of the end force and torque;
* attached ends move with the body (and clamped ends turn with it);
* reciprocity: the 6 x 6 mobility of a stiff aster is symmetric positive
  definite (Lorentz reciprocal theorem);
* GMRES equals a dense LAPACK solve of the assembled operator.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import kernels as ok
from oracle import system
from oracle.fiber import CLAMPED, HINGED

MU = 1.0


@pytest.fixture(scope="module", autouse=True)
def _build():
    ok.build()


def bare_sphere(grid, force=(0.0, 0.0, 0.0), torque=(0.0, 0.0, 0.0), periphery=None, centre=(0.0, 0.0, 0.0),
                mu=MU):
    b = wl.sphere_body(centre, 1.0, *grid, force=force, torque=torque)
    return wl.Suspension(n_per_fiber=np.zeros(0, np.int32), X=np.zeros((0, 3)), L=np.zeros(0),
                         f_ext=np.zeros((0, 3)), mu=mu, body=b, attach=np.zeros(0, np.int32),
                         boundary=periphery)


def cross_aster(attach, force, N=16, E=1.0, grid=(6, 12)):
    dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    a = wl.collocation_alpha(N)
    X = np.concatenate([d[None, :] * (1.0 + (a[:, None] + 1.0)) for d in dirs])   # L = 2
    b = wl.sphere_body((0.0, 0.0, 0.0), 1.0, *grid, force=force)
    return wl.Suspension(n_per_fiber=np.full(6, N, np.int32), X=X, L=np.full(6, 2.0), f_ext=np.zeros_like(X),
                         E=E, dt=1e-2, body=b, attach=np.full(6, attach, np.int32))


@pytest.mark.parametrize("mu", [MU, 2.5])
def test_isolated_sphere_stokes_drag_converges(mu):
    F = np.array([0.2, -0.5, 1.0])
    errs = []
    for grid in ((4, 8), (6, 12)):
        r = system.from_suspension(bare_sphere(grid, force=F, centre=(0.3, -0.2, 0.1), mu=mu)).step(tol=1e-12)
        errs.append(np.linalg.norm(r.U - F / (6 * np.pi * mu)) / np.linalg.norm(F / (6 * np.pi * mu)))
        assert np.linalg.norm(r.Omega) <= 1e-12 * np.linalg.norm(r.U)
    assert errs[1] < errs[0] / 10 and errs[1] <= 5e-9, errs


@pytest.mark.parametrize("mu", [MU, 2.5])
def test_isolated_sphere_rotational_drag(mu):
    Lt = np.array([0.3, 0.1, -0.7])
    r = system.from_suspension(bare_sphere((4, 8), torque=Lt, mu=mu)).step(tol=1e-12)
    assert np.linalg.norm(r.Omega - Lt / (8 * np.pi * mu)) <= 1e-10 * np.linalg.norm(Lt / (8 * np.pi * mu))
    assert np.linalg.norm(r.U) <= 1e-12


def test_concentric_sphere_drag():
    lam = 1.0 / 6.0
    gamma = 6 * np.pi * MU * 4 * (1 - lam ** 5) / (4 - 9 * lam + 10 * lam ** 3 - 9 * lam ** 5 + 4 * lam ** 6)
    F = np.array([0.2, -0.5, 1.0])
    s = bare_sphere((6, 12), force=F, periphery=wl.sphere_quadrature(6.0, 8, 16))
    r = system.from_suspension(s).step(tol=1e-12)
    err = np.linalg.norm(r.U - F / gamma) / np.linalg.norm(F / gamma)
    assert err <= 5e-5
    # the confinement correction is large, so the pin is not the free-space drag
    assert np.linalg.norm(r.U - F / (6 * np.pi * MU)) >= 0.5 * np.linalg.norm(F / gamma)


@pytest.mark.parametrize("attach", [CLAMPED, HINGED])
def test_cross_aster_symmetry(attach):
    rz = system.from_suspension(cross_aster(attach, (0.0, 0.0, 1.0))).step(tol=1e-12)
    rx = system.from_suspension(cross_aster(attach, (1.0, 0.0, 0.0))).step(tol=1e-12)
    for r, k in ((rz, 2), (rx, 0)):
        off = np.delete(r.U, k)
        assert np.linalg.norm(off) <= 1e-10 * abs(r.U[k])
        assert np.linalg.norm(r.Omega) <= 1e-10 * abs(r.U[k])
    # cubic symmetry (broken only by the (theta, phi) patch grid)
    assert abs(rx.U[0] / rz.U[2] - 1.0) <= 1e-3
    # the fibers add drag
    assert 0.9 / (6 * np.pi) < rz.U[2] < 1.0 / (6 * np.pi)


@pytest.fixture(scope="module")
def generic_aster():
    s = wl.aster(5, N=16, body_grid=(6, 12), R_periphery=None, fiber_force_std=1.0, tilt=0.5,
                 torque=(0.3, -0.2, 0.5), force=(0.1, 0.4, -0.2), seed=3)
    s.attach[1] = HINGED
    sy = system.from_suspension(s)
    return s, sy, sy.step(tol=1e-12)


def test_aster_force_and_torque_balance(generic_aster):
    s, sy, r = generic_aster
    us, _ = sy._split(r.u)
    Fk, Lk = sy._body_load(us, True)
    Fl, Ll = sy._body_load(us, False)
    F, Lt = Fk + Fl, Lk + Ll
    f_fl = np.zeros(3)
    t_fl = np.zeros(3)
    f_ap = np.array(s.body.force, float)
    t_ap = np.array(s.body.torque, float)
    for m, fb in enumerate(sy.fibers):
        a, c = sy.ptr[m], sy.ptr[m + 1]
        f = fb.f_known + fb.f_lin(us[m])
        arm = s.X[a:c] - sy.Xp
        f_fl += (fb.W[:, None] * f).sum(0)
        t_fl += (fb.W[:, None] * np.cross(arm, f)).sum(0)
        f_ap += (fb.W[:, None] * s.f_ext[a:c]).sum(0)
        t_ap += (fb.W[:, None] * np.cross(arm, s.f_ext[a:c])).sum(0)
    assert np.linalg.norm(f_fl + F - f_ap) <= 1e-9 * np.linalg.norm(f_ap)
    assert np.linalg.norm(t_fl + Lt - t_ap) <= 1e-9 * np.linalg.norm(t_ap)


def test_attached_ends_move_with_the_body(generic_aster):
    s, sy, r = generic_aster
    us, _ = sy._split(r.u)
    assert np.linalg.norm(r.Omega) > 1e-3
    root_curv = {}
    for m, fb in enumerate(sy.fibers):
        N, g = fb.N, 2.0 / fb.L
        c = [us[m][a * N:(a + 1) * N] for a in range(3)]
        v_end = np.array([fb.op.V0_pm[1] @ ca for ca in c])
        rigid = r.U + np.cross(r.Omega, fb.X_end - sy.Xp)
        assert np.linalg.norm(v_end - rigid) <= 1e-6 * np.linalg.norm(rigid)
        turn = g * np.array([fb.op.V1_pm[1] @ ca for ca in c])
        spin = np.cross(r.Omega, fb.t[N - 1])
        root_curv[m] = np.linalg.norm(fb.X2m + fb.dt * np.array([fb.op.V2_pm[1] @ ca for ca in c]))
        if fb.attach == CLAMPED:
            assert np.linalg.norm(turn - spin) <= 1e-6 * np.linalg.norm(spin)
        else:
            # hinged: free to turn
            assert np.linalg.norm(turn - spin) > 0.1 * np.linalg.norm(spin)
    # no couple at a hinge (X+_ss = 0 there); clamped roots bend
    clamped = max(v for m, v in root_curv.items() if sy.fibers[m].attach == CLAMPED)
    hinged = max(v for m, v in root_curv.items() if sy.fibers[m].attach == HINGED)
    assert clamped > 0.0 and hinged <= 1e-6 * clamped


def test_stiff_aster_mobility_is_symmetric_positive_definite():
    mob = np.zeros((6, 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = 1.0
        s = wl.aster(5, N=16, body_grid=(6, 12), R_periphery=None, tilt=0.6, force=e[:3], torque=e[3:],
                     seed=3, E=1e3, dt=1e-2)
        r = system.from_suspension(s).step(tol=1e-13)
        mob[:3, k], mob[3:, k] = r.U, r.Omega
    off = np.abs(mob - np.diag(np.diag(mob))).max()
    assert off > 1e-3                     # translation-rotation coupling present
    assert np.linalg.norm(mob - mob.T) <= 1e-3 * np.linalg.norm(mob)
    assert np.linalg.eigvalsh(0.5 * (mob + mob.T)).min() > 0.0


def test_aster_gmres_equals_dense_solve():
    s = wl.aster(2, N=10, body_grid=(2, 4), R_periphery=3.0, periphery_grid=(2, 4), fiber_force_std=1.0,
                 tilt=0.4, torque=(0.1, 0.2, -0.3), seed=5)
    s.attach[1] = HINGED
    sy = system.from_suspension(s)
    n = sy.n_unknowns
    A = np.stack([sy.matvec(e) for e in np.eye(n)], axis=1)
    b = sy.rhs()
    u = np.linalg.solve(A, b)
    r = sy.step(tol=1e-13)
    assert np.linalg.norm(r.u - u) <= 1e-9 * np.linalg.norm(u)


def test_table2_aster_inputs():
    """The Table 2 configuration: fibers attached at distinct points on the
    sphere, pointing outwards, inside the periphery, with the paper's load."""
    s = wl.table2_aster(64, grid=(8, 16))
    N = 31
    ends = s.X[N - 1::N]                       # minus ends (alpha = -1, last node)
    assert np.allclose(np.linalg.norm(ends, axis=1), 1.0)
    d = np.linalg.norm(ends[:, None, :] - ends[None, :, :], axis=-1) + np.eye(64) * 10
    assert d.min() > 0.05                       # distinct attachment points
    plus = s.X[0::N]
    assert np.allclose(np.linalg.norm(plus, axis=1), 3.0)          # length 2, radial
    assert np.all(np.linalg.norm(s.boundary.nodes, axis=1) <= 6.0 + 1e-12)
    assert np.allclose(s.body.force, (0.0, 0.0, 1.0 / (32 * 4.0)))
    # no attachment point sits on a surface quadrature node
    dn = np.linalg.norm(ends[:, None, :] - s.body.nodes[None, :, :], axis=-1)
    assert dn.min() > 1e-3
