"""Full-size check of the bench workload (1,024 curved fibers x 64 points,
65,536 points, N(0,1) force per node; the launch configuration bench.py times):
the GPU's solution must be a fixed point of the ORACLE's discrete system -- its
own right-hand side, coupling operator and fiber blocks, built independently in
FP64 (Sec. 3.2-3.3).

For every fiber m the oracle takes the GPU's unknowns of all bodies, forms the
coupling rows C_m u from them (Stokeslets of the other fibers' forces, Eq.
complementary-uf) and solves its own self block, u'_m = B_m^-1 (b_m - C_m u);
the check compares the nodal velocities V(u'_m) with V(u_m).

Why velocities and not coefficients: at N = 64 the self blocks have
||B^-1|| ~ 5e10..1e11 and the rough per-node forcing gives coefficient vectors
of norm 1e7..5e8 that cancel in V.  Two FP64 builds of the same block then
differ by rounding that no solve tolerance can remove: the coefficient-space
residual is 5e-5 for FP64 and mixed alike, and the unpreconditioned per-fiber
residual changes a hundredfold between the same oracle built on x86 and on
Arm.  In velocity space the floor is measured: perturbing the geometry by one
ulp moves the oracle's own velocities by 2.0e-6 (relative, all fibers), and
the GPU solution sits at 1.1e-6 (Arm build of the oracle) and 5.3e-6 (x86).
The gate is 2e-5.  The coupling carries 25% of the velocity in this
workload, so the gate still resolves a 1e-4 relative error in the coupling
(a dropped term, a sign, a wrong weight)."""
import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import kernels as ok
from oracle import system
from tests.gpu_helpers import dev, make_ctx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402

GATE = 2e-5


@pytest.fixture(scope="module")
def cloud():
    ok.build()
    s = wl.cfg_cloud_mixed(0)
    sy = system.from_suspension(s)
    return s, sy, sy.rhs()


def fixed_point_velocity_residual(sy, b, u):
    """||V(u') - V(u)|| / ||V(u)|| over all nodes, u'_m = B_m^-1 (b_m - C_m u)."""
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


@pytest.mark.parametrize("prec,tol", [(fs.FS_MIXED, 1e-8), (fs.FS_FP64, 1e-10)])
def test_cloud_solution_is_a_fixed_point_of_the_oracle_system(cloud, prec, tol):
    s, sy, b = cloud
    h = make_ctx(s, prec=prec, tol=tol)
    fs.fs_set_state(h, dev(s.X, torch), dev(s.L, torch), dev(s.f_ext, torch))
    inf = fs.fs_step(h)
    u = fs.fs_get_unknowns(h)
    V = torch.empty(s.X.shape, dtype=torch.float64, device="cuda:0")
    fs.fs_get_state(h, V=V)
    fs.fs_destroy(h)
    assert inf.resid <= tol
    assert u.shape[0] == sy.n_unknowns
    # the unknowns returned are the ones the step's velocities come from (V is
    # formed from coefficients that cancel by ~1e5: agreement to ~1e-9)
    us, _ = sy._split(u)
    Vu = np.concatenate([fb.velocity_nodes(um) for fb, um in zip(sy.fibers, us)])
    assert np.linalg.norm(Vu - V.cpu().numpy()) <= 1e-8 * np.linalg.norm(Vu)
    res = fixed_point_velocity_residual(sy, b, u)
    print("fixed-point velocity residual %.3e (gate %.0e)" % (res, GATE))
    assert res <= GATE
