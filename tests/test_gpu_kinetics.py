"""Growing and shrinking fibers on the GPU (fs_set_growth): parity of the step
with the oracle for both growth schemes (the paper's explicit term of Eq.
discrete-rhs, the default, and the implicit variant), the exact extension of
a force-free straight fiber, lengths updated by dt Ldot, and steps driven by
the dynamic instability."""
import copy

import numpy as np
import pytest

import workloads as wl
from oracle import cheb
from oracle import kinetics as kin
from oracle import system
from tests.gpu_helpers import dev, make_ctx, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402


GROWTH = {"explicit": False, "implicit": True}


def step_with_growth(s, Ldot, prec=fs.FS_FP64, tol=1e-12, growth="explicit"):
    h = make_ctx(s, prec=prec, tol=tol, growth_implicit=GROWTH[growth])
    X = dev(s.X, torch)
    fs.fs_set_state(h, X, dev(s.L, torch), dev(s.f_ext, torch))
    fs.fs_set_growth(h, np.asarray(Ldot, float))
    fs.fs_step(h)
    V = torch.empty_like(X)
    Xn = torch.empty_like(X)
    fs.fs_get_state(h, X=Xn, V=V)
    L = fs.fs_get_lengths(h, s.n_fibers)
    fs.fs_destroy(h)
    return V.cpu().numpy(), Xn.cpu().numpy(), L


@pytest.mark.parametrize("growth", ["explicit", "implicit"])
@pytest.mark.parametrize("prec,tol,gate", [(fs.FS_FP64, 1e-12, 1e-10), (fs.FS_MIXED, 1e-10, 1e-8)])
def test_growth_step_matches_oracle(prec, tol, gate, growth):
    s = wl.free_space(12, 24, 6.0, seed=7, curved_amp=0.05)
    s.f_ext = np.tile([0.0, 0.0, -1.0], (s.n_points, 1))
    Ldot = np.random.default_rng(1).uniform(-2.0, 2.0, 12)
    ref = system.from_suspension(s, Ldot=Ldot, growth=growth).step(tol=1e-13)
    V, Xn, L = step_with_growth(s, Ldot, prec, tol, growth)
    assert rel(V, ref.V) <= gate
    assert rel(Xn, ref.X_new) <= gate
    assert np.allclose(L, s.L + s.dt * Ldot, rtol=1e-15, atol=0.0)


@pytest.mark.parametrize("growth", ["explicit", "implicit"])
def test_force_free_straight_fiber_extends_exactly(growth):
    s = wl.free_space(3, 16, 20.0, seed=1)
    s.f_ext[:] = 0.0
    Ldot = np.array([0.7, -0.4, 2.0])
    _, Xn, L = step_with_growth(s, Ldot, growth=growth)
    a = cheb.nodes(16)
    for m in range(3):
        X = s.X[m * 16:(m + 1) * 16]
        t = (X[0] - X[-1]) / np.linalg.norm(X[0] - X[-1])
        want = X[-1][None, :] + ((a + 1.0) * L[m] / 2.0)[:, None] * t[None, :]
        assert np.abs(Xn[m * 16:(m + 1) * 16] - want).max() <= 1e-12 * s.L[m]


def test_rejects_a_rate_that_would_empty_a_fiber():
    s = wl.free_space(2, 16, 5.0, seed=2)
    h = make_ctx(s)
    fs.fs_set_state(h, s.X, s.L, s.f_ext)
    with pytest.raises(fs.FsError):
        fs.fs_set_growth(h, np.array([0.0, -2.0 * s.L[1] / s.dt]))
    fs.fs_destroy(h)


@pytest.mark.parametrize("growth", ["explicit", "implicit"])
def test_dynamic_instability_steps_match_oracle(growth):
    """Three steps; each step the library's host state machine sets the rates
    (the oracle's gives the same, bit for bit) and both sides step from the
    GPU's current state."""
    s = wl.free_space(10, 16, 5.0, seed=9, curved_amp=0.05)
    s.f_ext = np.tile([0.1, 0.0, -1.0], (s.n_points, 1))
    h = make_ctx(s, tol=1e-12, growth_implicit=GROWTH[growth])
    X = dev(s.X, torch)
    fs.fs_set_state(h, X, dev(s.L, torch), dev(s.f_ext, torch))
    rng = np.random.default_rng(3)
    state = np.ones(10, dtype=np.int32)
    cur = copy.deepcopy(s)
    Xn = torch.empty_like(X)
    V = torch.empty_like(X)
    args = (s.dt, 5.0, 10.0, 200.0, 50.0, 0.5)
    for k in range(3):
        L = fs.fs_get_lengths(h, 10)
        u = rng.random(10)
        state_o, Ld_o = kin.dynamic_instability(state, L, u, *args)
        state, Ld = fs.fs_dynamic_instability(state, L, u, *args)
        assert np.array_equal(state, state_o) and np.array_equal(Ld, Ld_o)
        fs.fs_set_growth(h, Ld)
        cur.L = L
        ref = system.from_suspension(cur, Ldot=Ld, growth=growth).step(tol=1e-13)
        fs.fs_step(h)
        fs.fs_get_state(h, X=Xn, V=V)
        assert rel(V.cpu().numpy(), ref.V) <= 1e-10
        assert np.allclose(fs.fs_get_lengths(h, 10), ref.L_new, rtol=1e-15, atol=0.0)
        cur.X = Xn.cpu().numpy().copy()
    fs.fs_destroy(h)
