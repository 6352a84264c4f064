"""GPU steps against the EXACT solution of the discrete system (oracle.exact:
dense assembly, LU and refinement with double-double residuals), not against
the oracle's own GMRES.  Per-node N(0,1) forcing (the workloads' recipe)
makes the fiber coefficients large (|u| ~ 1e5..1e8 for velocities of O(10))
and V a cancellation of them, so no FP64 evaluation of the same discrete
system can place V closer to the exact solution than the system's
sensitivity to one rounding of its entries.  oracle.exact.perturbation_floor
measures that floor; each gate below is the stated parity tolerance (1e-10
FP64, 1e-8 mixed) or, where the measured floor is above it, a small multiple of the floor (both stated
per case, and the floor re-measured in the test)."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact
from oracle import system
from tests.gpu_helpers import gpu_step, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402

# name -> (suspension, measured floor of V).  The floor perturbs every entry
# by one rounding; the library assembles its entries by other FP64 sums
# (GEMMs over N terms, double-double geometry), each carrying a few roundings,
# and lands at 3-10x the floor (measured: 6.7e-9, 4.5e-8, 3.7e-6 for the FP64
# path).  Gate: max(parity tolerance, 20 x floor), the tolerance being
# 1e-10 for the FP64 path and 1e-8 for the mixed path.
CASES = {
    "cfg1_16x32_straight": (lambda: wl.cfg_small_fp64(0), 8.8e-10),
    "16x64_curved": (lambda: wl.free_space(16, 64, 40.0 * (16 / 1024) ** (1 / 3), seed=0, curved_amp=0.05),
                     4.9e-9),
    "4x64_curved": (lambda: wl.free_space(4, 64, 40.0 * (4 / 1024) ** (1 / 3), seed=0, curved_amp=0.05),
                    1.45e-6),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_step_matches_exact_discrete_solution(name):
    make, floor_rec = CASES[name]
    gate64, gate_mx = max(1e-10, 20.0 * floor_rec), max(1e-8, 20.0 * floor_rec)
    s = make()
    S = system.from_suspension(s)
    A, b = exact.assemble(S)
    x, _ = exact.solve_refined(A, b)
    ref = S.result(x)
    floor = exact.perturbation_floor(A, b, lambda u: S.result(u).V, trials=2)
    print("%s: floor %.2e" % (name, floor))
    assert floor <= 2.0 * floor_rec          # the gate below rests on this floor
    for prec, tol, gate in ((fs.FS_FP64, 1e-15, gate64), (fs.FS_MIXED, 1e-13, gate_mx)):
        V, T, Xn, infos = gpu_step(s, torch, prec=prec, tol=tol)
        eV, eT = rel(V, ref.V), rel(T, ref.T)
        print("%s prec %d: V %.2e T %.2e (%d iterations)" % (name, prec, eV, eT, infos[0].iters))
        assert eV <= gate
