"""The opt-in far-field autotuner (fs_options.autotune): the first sum of
each precision class times the three launch shapes and keeps the fastest.

Checks: the classes a step uses come out tuned (shape ids 1..3); an
autotuned context gives the untuned context's velocities to the accuracy of
the sums (FP64 path: the same system solved with another summation order,
gated at 1e-10; mixed path: two refined solutions that each meet the 1e-8
residual tolerance with the inner FP32 sums in different orders, gated at
1e-7); and a tuned context repeats its own step bit for bit (the shape stays
fixed after tuning)."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import dev, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402


def run(s, prec, tol, autotune, steps=1):
    opt = fs.fs_options_default()
    opt.prec, opt.tol, opt.autotune = prec, tol, autotune
    h = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, options=opt)
    X = dev(s.X, torch)
    out = []
    for _ in range(steps):
        fs.fs_set_state(h, X, dev(s.L, torch), dev(s.f_ext, torch))
        fs.fs_step(h)
        V = torch.empty_like(X)
        fs.fs_get_state(h, V=V)
        out.append(V.cpu().numpy())
    tuned = fs.fs_get_tuned_shapes(h)
    fs.fs_destroy(h)
    return out, tuned


@pytest.mark.parametrize("prec,tol,gate", [(fs.FS_FP64, 1e-12, 1e-10), (fs.FS_MIXED, 1e-8, 1e-7)])
def test_autotuned_step_matches_default(prec, tol, gate):
    s = wl.free_space(96, 32, 10.0, seed=7, curved_amp=0.05)
    (v0,), t0 = run(s, prec, tol, 0)
    (v1a, v1b), t1 = run(s, prec, tol, 1, steps=2)
    print("precision %d: tuned shapes %s, relative difference %.2e" % (prec, t1, rel(v1a, v0)))
    assert t0 == {}
    assert t1 and all(1 <= v <= 3 for v in t1.values())
    assert rel(v1a, v0) <= gate
    assert np.array_equal(v1a, v1b)
