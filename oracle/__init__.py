"""CPU oracle of the implicit fiber step -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU legs (its
``cpu_baseline`` and its ``--impl reference`` arm) may import this package.
The library (``paper_1602_05650_gb300``) never imports, links or runs it, and
the two share no code: the only shared module is ``workloads``, which
generates seeded inputs and holds none of the method's arithmetic.

Plain FP64 throughout: numpy / scipy for the Chebyshev algebra, dense
per-fiber matrices, LU and GMRES; plain C double loops (pairsum.c) for the
all-pairs Stokeslet / stresslet sums.

Modules and the passages they follow:
  cheb.py     Sec. 3.1.3 (Eq. cheb-basis), Sec. 3.1.4 (Clenshaw-Curtis)
  pairsum.c   Eqs. oseen, stresslet, single-layer, double-layer,
              main-cortex-density with Sec. 3.1.2 singularity subtraction
  fiber.py    Eqs. main-sb-local, sb-stokes-reg, force-balance,
              main-elastic-force, main-inextensibility, bc-free; Sec. 3.2;
              attached minus ends (Eqs. BC2-1, BC2-2, BC2-T) and growth
              (Sec. 2.4)
  system.py   Eqs. complementary-uc/uf, sche-linear-eq, prec; Sec. 3.3 GMRES;
              the rigid body (Eqs. main-nsb-second-kind, main-nsb-rgbt,
              main-nsb-rgbr, f-ext, t-ext)
  kinetics.py Sec. 2.4 / Sec. 5 two-state dynamic instability

Pinning (tests/test_oracle_*.py, all `-m "not gpu"`): every function above
is pinned against closed forms, invariants, brute force, convergence in N
or values the paper prints (tests/golden/); the test docstrings say which
pin covers which function.
"""
from . import cheb, kernels, fiber, system  # noqa: F401
