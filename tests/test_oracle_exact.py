"""Pins of the oracle's exact discrete solve (oracle/exact.py): the
double-double residual is exact to double-double rounding, the refined
solution of an ill-conditioned matrix equals a 40-digit mpmath solution of
the same FP64 entries to FP64 accuracy, and the refined solution of a small
fiber system equals the mpmath solution of its assembled operator and the
oracle's GMRES at a tight tolerance."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact
from oracle import kernels as ok
from oracle import system

mpmath = pytest.importorskip("mpmath")


def _mp_solve(A, b, dps=40):
    with mpmath.workdps(dps):
        Am = mpmath.matrix([[mpmath.mpf(float(v)) for v in row] for row in A])
        bm = mpmath.matrix([mpmath.mpf(float(v)) for v in b])
        return np.array([float(v) for v in mpmath.lu_solve(Am, bm)])


def test_residual_is_exact_to_double_double():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(7, 7)) * np.exp(rng.uniform(-20, 20, size=(7, 7)))
    x = rng.normal(size=7)
    b = rng.normal(size=7)
    r = exact.residual_dd(A, x, b)
    with mpmath.workdps(60):
        want = [mpmath.mpf(float(b[i])) - mpmath.fsum(mpmath.mpf(float(A[i, j])) * mpmath.mpf(float(x[j]))
                                                      for j in range(7)) for i in range(7)]
        err = max(abs(mpmath.mpf(float(r[i])) - want[i]) / max(abs(want[i]), mpmath.mpf(1e-300))
                  for i in range(7))
    assert float(err) <= 2.0 ** -52


def test_refined_solution_of_a_hilbert_matrix():
    """cond(H_10) ~ 1.6e13: plain LU loses ~13 digits, refinement recovers
    the exact solution of the FP64 matrix to FP64 accuracy."""
    n = 10
    H = 1.0 / (np.arange(n)[:, None] + np.arange(n)[None, :] + 1.0)
    b = np.ones(n)
    want = _mp_solve(H, b)
    x, steps = exact.solve_refined(H, b)
    assert np.linalg.norm(x - want) <= 4e-16 * np.linalg.norm(want)
    plain = np.linalg.solve(H, b)
    assert np.linalg.norm(plain - want) > 1e-8 * np.linalg.norm(want)   # the refinement is needed


def test_exact_step_of_a_small_fiber_system():
    ok.build()
    s = wl.free_space(2, 8, 2.0, seed=5, curved_amp=0.05)
    S = system.from_suspension(s)
    A, b = exact.assemble(S)
    x, _ = exact.solve_refined(A, b)
    want = _mp_solve(A, b)
    assert np.linalg.norm(x - want) <= 1e-15 * np.linalg.norm(want)
    ref = S.exact_step()
    gm = S.step(tol=1e-14)
    assert np.linalg.norm(gm.V - ref.V) <= 1e-11 * np.linalg.norm(ref.V)


def test_perturbation_floor_is_the_systems_sensitivity():
    """The floor of a well-conditioned system sits at rounding level, that of
    the Hilbert matrix near cond x 2^-53."""
    rng = np.random.default_rng(3)
    A = np.eye(20) + 0.1 * rng.normal(size=(20, 20))
    b = rng.normal(size=20)
    assert exact.perturbation_floor(A, b, lambda x: x) <= 1e-14
    n = 10
    H = 1.0 / (np.arange(n)[:, None] + np.arange(n)[None, :] + 1.0)
    fl = exact.perturbation_floor(H, np.ones(n), lambda x: x)
    assert 1e-6 <= fl <= 1e-1
