"""Oracle and input recipes against values the paper prints (fixtures in
tests/golden/, each citing its source).

sedimenting_cloud.txt and table2_aster.txt (Sec. 4.3, Table 2): the
synthetic workloads that stand in for the paper's cloud and confined aster
have the sizes, parameters and layout the paper prints.

microtubule_parameters.txt (Sec. 4, table of simulation parameters): the
dynamic-instability rates, bending modulus and viscosity of the kinetics
workload.

kdelta_regularisation.txt (Sec. 3.5, regularisation of K_delta): a sphere
with 32 hinged fibers of length 5r in free space, pulled by a force.  The
paper reports three things:
* keeping the nonlocal self term changes the sphere's velocity by at most
  1.4 % against local slender-body theory;
* between the two smallest factors, delta = 5e-3 and 1e-2, the velocity
  changes by O(1e-5);
* that change shrinks with delta.
The oracle takes delta as a fraction of the fiber length (δ = 0.01 L by
default).  At the first step it gives 1.07 % and 2.7e-5 at N = 16, and
1.05 % and 1.8e-5 at N = 32.  Taking the printed delta as an absolute length
with L = 5 would give 2.4e-6, a decade below the printed order.

Mistakes planted in the oracle's K_delta and caught here:
* subtraction term dropped: 9.8 %;
* subtraction with the wrong sign: 18 %;
* subtraction without its t t part: 4.8 %;
* 8 pi missing from the subtraction: 99 %;
* regularisation factor |r| / sqrt(|r|^2 + delta^2) dropped: the change
  between the two delta values becomes 6.6e-4.
"""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import kernels as ok
from oracle import system
from oracle.fiber import HINGED

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (x.strip() for x in line.split("=", 1))
                vals[k] = float(v)
    return vals


@pytest.fixture(scope="module", autouse=True)
def _build():
    ok.build()


def test_kdelta_regularisation_matches_the_printed_values():
    g = read_golden("kdelta_regularisation.txt")
    # the sphere (radius 1) carries the default force of the aster workload
    s = wl.aster(32, N=16, radius=1.0, L=5.0, R_periphery=None, body_grid=(6, 12), attach=HINGED, seed=0)

    def U(**kw):
        return system.from_suspension(s, **kw).step(tol=1e-12).U

    u_lsb = U(lsb=True)
    d_hi, d_lo = g["delta_large"], g["delta_small"]
    us = [U(delta_over_L=d) for d in (d_hi, d_lo, d_lo / 2)]
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    nl = rel(us[0], u_lsb)
    step1, step2 = rel(us[0], us[1]), rel(us[1], us[2])
    print("|U_NLSB/U_LSB - 1| = %.3e; delta %.0e -> %.0e: %.2e; -> %.1e: %.2e"
          % (nl, d_hi, d_lo, step1, d_lo / 2, step2))
    # nonlocal self term: a small, nonzero correction within the printed bound
    assert 1e-3 < nl <= g["max_rel_diff_nlsb_lsb"]
    # the two smallest factors agree to the printed order (within a decade)
    order = g["rel_diff_delta_order"]
    assert order / 10 <= step1 <= order * 10
    # and the change shrinks as delta decreases
    assert step2 < step1


def test_sedimenting_cloud_follows_the_printed_setup():
    """The synthetic cloud (workloads.sedimenting_cloud) has the sizes,
    parameters and layout Sec. 4.3 prints, and its four lengths give the
    quoted effective volume fractions (to their rounding, 5 %)."""
    g = read_golden("sedimenting_cloud.txt")
    R0 = g["R0"]
    for i in range(1, 5):
        L = g["L_%d" % i]
        s = wl.sedimenting_cloud(L, R0=R0)
        assert s.n_fibers == int(g["n_fibers"])
        assert s.eps == g["eps"] and s.E == pytest.approx(g["E_over_f0_R0_cubed"] * R0 ** 3)
        assert np.all(s.L == L * R0)
        phi = s.n_fibers * (L * R0 / 2) ** 3 / (4.0 / 3.0 * np.pi * R0 ** 3)
        assert phi == pytest.approx(g["phi_%d" % i], rel=0.05)
        X = s.X.reshape(s.n_fibers, -1, 3)
        assert np.linalg.norm(X.mean(axis=1), axis=1).max() <= R0      # centres in the ball
        assert np.all(s.f_ext[:, :2] == 0.0) and np.all(s.f_ext[:, 2] < 0.0)   # downward load


def test_table2_aster_follows_the_printed_setup():
    """workloads.table2_aster is the Table 2 configuration, and its time step
    is below the paper's largest stable step for every fiber count."""
    g = read_golden("table2_aster.txt")
    from oracle.fiber import CLAMPED
    r = g["r"]
    for i in range(1, 5):
        n = int(g["n_fibers_%d" % i])
        s = wl.table2_aster(n, grid=(4, 8))
        L = g["L_over_r"] * r
        assert s.n_fibers == n and np.all(s.n_per_fiber == int(g["points_per_fiber"]))
        assert np.all(s.L == L) and np.all(s.attach == CLAMPED)
        assert s.body.radius == r and s.boundary.R == pytest.approx(g["R_outer_over_r"] * r)
        assert np.linalg.norm(s.body.force) == pytest.approx(g["force_over_E_per_L2"] * s.E / L ** 2)
        assert not np.any(s.f_ext)                                      # load on the sphere only
        # minus ends on the sphere, fibers pointing outwards to radius r + L
        X = s.X.reshape(n, -1, 3)
        assert np.allclose(np.linalg.norm(X[:, -1], axis=1), r)
        assert np.allclose(np.linalg.norm(X[:, 0], axis=1), r + L)
        tau_e = 8.0 * np.pi * s.mu * L ** 4 / (-np.log(s.eps ** 2 * np.e))
        assert s.dt <= 1e-3 * g["dt_max_%d" % i] * tau_e


def test_microtubule_parameters_are_the_printed_table():
    g = read_golden("microtubule_parameters.txt")
    assert wl.MICROTUBULE == g
