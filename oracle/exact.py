"""The exact solution of the discrete step's linear system (oracle; test
infrastructure).

GMRES stops at a tolerance, so the oracle's own step is only within that
tolerance of the solution of A u = b (Eq. sche-linear-eq).  This module solves
the assembled system to the accuracy its FP64 entries allow: an LU
factorisation in FP64 followed by iterative refinement (Wilkinson; Moler,
J. ACM 14, 1967) whose residuals b - A x are accumulated in double-double
arithmetic (Dekker's exact product by Veltkamp splitting and Knuth's
TwoSum), so that the refined x is the solution of the FP64 system up to
~cond(A) x 1e-30 -- far below the system's own sensitivity to 1-ulp changes
of its entries, which `perturbation_floor` measures.

No GPU code shares anything with this module.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

_SPLIT = 134217729.0   # 2^27 + 1: Veltkamp's splitting constant for FP64


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a, b):
    """p + e = a b exactly (Dekker)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _two_sum(a, b):
    """s + e = a + b exactly (Knuth)."""
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def residual_dd(A: np.ndarray, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """b - A x with every product and sum carried in double-double, rounded
    to FP64 at the end (row by row over the columns)."""
    n = A.shape[1]
    sh = b.astype(np.float64).copy()
    sl = np.zeros_like(sh)
    for j in range(n):
        p, e = _two_prod(A[:, j], -x[j])
        s, t = _two_sum(sh, p)
        sl = sl + (t + e)
        sh = s
    return sh + sl


def equilibration(A: np.ndarray, rounds: int = 4):
    """Power-of-two row and column scalings r, c (exact in FP64) that bring
    the largest entry of every row and column of diag(r) A diag(c) near 1
    (alternating max-norm scaling); they shrink the condition number the
    rows' mixed units (velocities, end conditions, tension rows) give A."""
    r = np.ones(A.shape[0])
    c = np.ones(A.shape[1])
    for _ in range(rounds):
        M = np.abs(A) * r[:, None] * c[None, :]
        rm = M.max(axis=1)
        r = r * np.where(rm > 0, 2.0 ** -np.round(np.log2(np.where(rm > 0, rm, 1.0))), 1.0)
        M = np.abs(A) * r[:, None] * c[None, :]
        cm = M.max(axis=0)
        c = c * np.where(cm > 0, 2.0 ** -np.round(np.log2(np.where(cm > 0, cm, 1.0))), 1.0)
    return r, c


def solve_refined(A: np.ndarray, b: np.ndarray, sweeps: int = 12):
    """x with A x = b to working accuracy of the FP64 system: FP64 LU of the
    equilibrated matrix, then refinement x += A^-1 r with r = b - A x in
    double-double.  Returns x and the FP64 norms of the successive
    corrections."""
    rs, cs = equilibration(A)
    lu = scipy.linalg.lu_factor(A * rs[:, None] * cs[None, :])

    def inv(v):
        return cs * scipy.linalg.lu_solve(lu, rs * v)

    x = inv(b)
    steps = []
    for _ in range(sweeps):
        d = inv(residual_dd(A, x, b))
        x = x + d
        steps.append(float(np.linalg.norm(d)))
        if steps[-1] <= 1e-30 * np.linalg.norm(x):
            break
    return x, steps


def assemble(system) -> tuple:
    """The dense operator A (column j = A e_j through the system's own
    matvec) and the right-hand side b of an oracle System."""
    n = system.n_unknowns
    A = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = system.matvec(e)
        e[j] = 0.0
    return A, system.rhs()


def perturbation_floor(A: np.ndarray, b: np.ndarray, observe, trials: int = 3, seed: int = 0) -> float:
    """Largest relative change of observe(x) when every entry of A and b is
    perturbed by an independent random relative 2^-53 (one rounding): the
    spread any FP64 evaluation of the same discrete system has, whatever
    solver it uses."""
    rng = np.random.default_rng(seed)
    x0, _ = solve_refined(A, b)
    y0 = observe(x0)
    worst = 0.0
    for _ in range(trials):
        Ap = A * (1.0 + 2.0 ** -53 * rng.choice([-1.0, 1.0], size=A.shape))
        bp = b * (1.0 + 2.0 ** -53 * rng.choice([-1.0, 1.0], size=b.shape))
        x, _ = solve_refined(Ap, bp)
        worst = max(worst, float(np.linalg.norm(observe(x) - y0) / np.linalg.norm(y0)))
    return worst
