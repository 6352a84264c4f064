"""Full-size checks of the confined and batched workloads in the launch
configurations bench.py times (mixed precision): the GPU's unknowns must be a
fixed point of the ORACLE's discrete system, built independently in FP64 (as
test_gpu_fullsize.py does for the cloud).

* Confined (2,000 fibers x 32 points in a radius-20 sphere, 12,288 surface
  nodes): for every fiber the oracle forms the coupling rows from the GPU's
  unknowns (other fibers' Stokeslets and the periphery's double layer of the
  GPU's density) and solves its own self block; the nodal velocities must
  agree.  The surface rows of the oracle's operator applied to the GPU's
  unknowns must vanish relative to the surface right-hand side, scaled by the
  Jacobi diagonal as the solver's residual is.
* Batched (256 systems, 8..512 fibers, 16/32/64 points): the same fiber
  fixed-point test on 12 sampled systems, each built by the oracle alone.

Tolerance.  The stopping test bounds the residual of the coefficients, not of
the velocities: with the workloads' per-node N(0,1) forcing the oracle's own
GMRES at 1e-8 sits up to 1.5e-4 (in V) from its fixed point (printed per
system).  The check therefore solves to 1e-12, where the measured residuals
are 1.9e-8 (confined fibers), 5.5e-8 (confined surface rows) and at most
5.5e-8 (batched systems): gates 1e-6."""
import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import kernels as ok
from oracle import system
from tests.gpu_helpers import dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402

TOL = 1e-12


def fiber_fixed_point(sy, b, u):
    us, q = sy._split(u)
    bs, _ = sy._split(b)
    f = np.concatenate([fb.f_lin(um) for fb, um in zip(sy.fibers, us)])
    ub, _ = sy._couplings(f, q)
    num = den = 0.0
    for m, fb in enumerate(sy.fibers):
        a, c = sy.ptr[m], sy.ptr[m + 1]
        um = scipy.linalg.lu_solve(sy.lu[m], bs[m] - fb.rows_from_ubar(ub[a:c]))
        V = fb.velocity_nodes(us[m])
        num += float(np.sum((fb.velocity_nodes(um) - V) ** 2))
        den += float(np.sum(V ** 2))
    return np.sqrt(num / den)


def test_confined_full_size_is_a_fixed_point():
    ok.build()
    s = wl.cfg_confined(0)
    opt = fs.fs_options_default()
    opt.prec, opt.tol = fs.FS_MIXED, TOL
    h = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, boundary=s.boundary, options=opt)
    fs.fs_set_state(h, dev(s.X, torch), dev(s.L, torch), dev(s.f_ext, torch))
    inf = fs.fs_step(h)
    u = fs.fs_get_unknowns(h)
    fs.fs_destroy(h)
    assert inf.resid <= TOL
    sy = system.from_suspension(s)
    b = sy.rhs()
    res_f = fiber_fixed_point(sy, b, u)
    r = sy.matvec(u) - b
    n0, d = sy.uptr[-1], sy.sdiag          # the surface rows and their Jacobi diagonal
    rs = r[n0:n0 + d.shape[0]] / d
    bsurf = b[n0:n0 + d.shape[0]] / d
    res_s = np.linalg.norm(rs) / np.linalg.norm(bsurf)
    print("confined: fiber fixed point %.2e, surface rows %.2e (%d iterations)" % (res_f, res_s, inf.iters))
    assert res_f <= 1e-6
    assert res_s <= 1e-6


def test_batched_full_size_sampled_systems():
    ok.build()
    systems = wl.batched(256, seed=0)
    opt = fs.fs_options_default()
    opt.prec, opt.tol = fs.FS_MIXED, TOL
    fps = [x.n_fibers for x in systems]
    h = fs.fs_create_batch(fps, np.concatenate([x.n_per_fiber for x in systems]), 1.0, 1e-3, 1.0, 1e-3,
                           options=opt)
    X = dev(np.concatenate([x.X for x in systems]), torch)
    L = dev(np.concatenate([x.L for x in systems]), torch)
    F = dev(np.concatenate([x.f_ext for x in systems]), torch)
    fs.fs_set_state(h, X, L, F)
    fs.fs_step(h)
    info = fs.fs_batch_info(h)
    u = fs.fs_get_unknowns(h)
    fs.fs_destroy(h)
    assert all(info["converged"])
    offs = np.concatenate([[0], np.cumsum([4 * int(x.n_per_fiber.sum()) for x in systems])])
    rng = np.random.default_rng(1)
    worst = 0.0
    for k in sorted(rng.choice(len(systems), 12, replace=False)):
        x = systems[k]
        sy = system.from_suspension(x)
        b = sy.rhs()
        res = fiber_fixed_point(sy, b, u[offs[k]:offs[k + 1]])
        own = fiber_fixed_point(sy, b, sy.gmres(b, 1e-8)[0])
        worst = max(worst, res)
        print("batched system %d (%d x %d): fiber fixed point %.2e (oracle GMRES at 1e-8: %.2e)"
              % (k, x.n_fibers, x.n_per_fiber[0], res, own))
    assert worst <= 1e-6
