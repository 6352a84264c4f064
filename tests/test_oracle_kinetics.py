"""Pins of fiber (de)polymerization (Sec. 2.4 kinetics; the dynamic
instability of Sec. 5) in the oracle.  The default growth scheme is the
paper's: the reparametrisation term of Eq. chain-rule on the right-hand side
at the current time (Eq. discrete-rhs), with the sign that advances the plus
end.  The named variant growth="implicit" takes the same term at the new time.
* a force-free straight fiber with plus-end growth rate Ldot extends exactly:
  its minus end stays, its plus end advances by Ldot dt, tension zero (both
  schemes);
* a curved fiber gains dt Ldot of arclength from the growth term (the
  material is inextensible; only the plus end adds length), to a relative
  error that shrinks with dt (explicit), or within 5e-4 (implicit);
* the explicit step is exactly affine in Ldot (the term is a known
  right-hand side); the implicit one up to O(dt Ldot / L) (it puts
  dt Ldot / (L + dt Ldot) into the self block);
* a fast-shrinking curved fiber stays smooth with the implicit term and does
  not with the explicit one (why the variant exists);
* the two-state dynamic instability reaches the Dogterom-Leibler stationary
  mean length v_g v_s / (v_s f_cat - v_g f_res) (+ the nucleation length)."""
import numpy as np
import pytest

import workloads as wl
from oracle import cheb
from oracle import kinetics as kin
from oracle import kernels as ok
from oracle import system


def arclength(Xm):
    """Clenshaw-Curtis arclength of the interpolant of one fiber's nodes."""
    N = Xm.shape[0]
    Xa = cheb.interp_derivs_ext(Xm, cheb.nodes_ld(N), 1).astype(float)
    return float(cheb.cc_weights(N) @ np.linalg.norm(Xa, axis=1))


@pytest.mark.parametrize("growth", ["explicit", "implicit"])
def test_straight_fiber_grows_at_its_plus_end(growth):
    ok.build()
    s = wl.free_space(3, 16, 20.0, seed=1)
    s.f_ext[:] = 0.0
    Ldot = np.array([0.7, -0.4, 2.0])
    r = system.from_suspension(s, Ldot=Ldot, growth=growth).step(tol=1e-13)
    N = 16
    a = cheb.nodes(N)
    for m in range(3):
        X = s.X[m * N:(m + 1) * N]
        t = (X[0] - X[-1]) / np.linalg.norm(X[0] - X[-1])      # node 0 is alpha = +1
        Lnew = s.L[m] + s.dt * Ldot[m]
        want = X[-1][None, :] + ((a + 1.0) * Lnew / 2.0)[:, None] * t[None, :]
        assert np.abs(r.X_new[m * N:(m + 1) * N] - want).max() <= 1e-12 * s.L[m]
    assert np.abs(r.T).max() <= 1e-9
    assert np.allclose(r.L_new, s.L + s.dt * Ldot, rtol=0, atol=1e-15)


def _grown_length_errors(growth):
    rels = []
    for dt in (1e-3, 1e-4):
        s = wl.free_space(1, 24, 5.0, seed=2, curved_amp=0.1, dt=dt)
        s.f_ext[:] = 0.0
        Ldot = 1.5
        grown = arclength(system.from_suspension(s, Ldot=np.array([Ldot]), growth=growth)
                          .step(tol=1e-13).X_new)
        fixed = arclength(system.from_suspension(s).step(tol=1e-13).X_new)
        rels.append(abs((grown - fixed) / (dt * Ldot) - 1.0))
    return rels


def test_curved_fiber_gains_the_grown_length():
    """The length the growth term adds to a curved fiber in one step is
    dt Ldot (the rest of the step's length change -- the linearised
    inextensibility acting on the bending relaxation -- is the same with and
    without growth), to a relative error that shrinks with dt (measured
    8.7e-4 and 2.8e-4 at dt = 1e-3, 1e-4)."""
    ok.build()
    rels = _grown_length_errors("explicit")
    assert rels[0] <= 2e-3 and rels[1] <= rels[0] / 2.0


def test_curved_fiber_gains_the_grown_length_implicit():
    """The implicit variant: within 5e-4 (measured 1.3e-4 and 9.5e-5)."""
    ok.build()
    assert max(_grown_length_errors("implicit")) <= 5e-4


def _three_rates(growth):
    s = wl.free_space(4, 16, 6.0, seed=3, curved_amp=0.05)
    s.f_ext = np.tile([0.0, 0.0, -1.0], (s.n_points, 1))
    Ld = np.array([0.5, -0.3, 1.0, 0.2])
    V0 = system.from_suspension(s).step(tol=1e-13).V
    V1 = system.from_suspension(s, Ldot=Ld, growth=growth).step(tol=1e-13).V
    V2 = system.from_suspension(s, Ldot=2.0 * Ld, growth=growth).step(tol=1e-13).V
    return s, Ld, np.linalg.norm((V2 - V0) - 2.0 * (V1 - V0)) / np.linalg.norm(V1 - V0)


def test_step_is_affine_in_the_growth_rate():
    """Explicit growth term: a known right-hand side linear in Ldot, so V is
    exactly affine in Ldot (measured 9e-12)."""
    ok.build()
    _, _, dev = _three_rates("explicit")
    assert dev <= 1e-9


def test_implicit_step_is_affine_in_the_growth_rate_to_first_order():
    """Implicit variant: its part at the new time adds dt kappa (y + 1) V_alpha
    to the self block, so V is affine in Ldot up to relative O(dt Ldot / L)."""
    ok.build()
    s, Ld, dev = _three_rates("implicit")
    assert dev <= 10.0 * s.dt * np.max(np.abs(Ld) / s.L)


def _shrink(growth, steps=19):
    s = wl.free_space(1, 16, 5.0, seed=4, curved_amp=0.05, L_range=(4.0, 4.0), E=10.0, dt=0.1)
    s.f_ext = np.tile([0.0, 0.0, -0.05], (s.n_points, 1))
    X, L = s.X.copy(), s.L.copy()
    vmax = 0.0
    for _ in range(steps):
        sub = wl.Suspension(s.n_per_fiber, X, L, s.f_ext, s.mu, s.eps, s.E, s.dt)
        r = system.from_suspension(sub, Ldot=np.array([-0.288 * 5.0]), growth=growth).step(tol=1e-12)
        X, L = r.X_new, r.L_new
        vmax = max(vmax, float(np.abs(r.V).max()))
    return s, X, L, vmax


def test_shrinking_fiber_stays_smooth_with_the_implicit_term():
    """A curved fiber shrinking by 0.144 per step (dt |Ldot| / L from 0.04 to
    0.11) for 19 steps, 4 -> 1.26 in length, keeps its discrete length equal
    to L (within 1 %) and its velocities bounded with the growth term at the
    new time (measured: length error 0.5 %, |V| <= 1.4)."""
    ok.build()
    s, X, L, vmax = _shrink("implicit")
    assert np.isfinite(vmax) and vmax < 10.0
    assert L[0] < 0.35 * s.L[0]
    assert abs(arclength(X) / L[0] - 1.0) <= 0.01


def test_shrinking_fiber_is_unstable_with_the_explicit_term():
    """The same fiber with the paper's explicit term: the reparametrisation is
    an advection in alpha (its spectral derivative has eigenvalues up to
    ~N^2) stepped by forward Euler, and the fiber's discrete length departs
    from L (measured: 50x L after 19 steps, |V| up to 335)."""
    ok.build()
    s, X, L, vmax = _shrink("explicit")
    assert not (abs(arclength(X) / L[0] - 1.0) <= 0.5)


def test_dynamic_instability_mean_length():
    v_g, v_s, f_cat, f_res, L_min = 1.0, 2.0, 1.0, 0.5, 0.01
    ell = kin.mean_length_bounded(v_g, v_s, f_cat, f_res)          # 4/3
    rng = np.random.default_rng(0)
    n, dt = 20000, 0.002
    state = np.ones(n, dtype=np.int32)
    L = np.full(n, L_min)
    means = []
    for k in range(15000):
        state, Ldot = kin.dynamic_instability(state, L, rng.random(n), dt, v_g, v_s, f_cat, f_res, L_min)
        L = L + dt * Ldot
        if k >= 7500 and k % 50 == 0:
            means.append(L.mean())
    assert abs(np.mean(means) / ell - 1.0) <= 0.03


def test_dynamic_instability_rules():
    # switch probabilities, rescue at L_min, cap at L_max
    st, Ld = kin.dynamic_instability([1, 1, 0, 0], [1.0, 1.0, 1.0, 0.05], [0.0, 0.99, 0.0, 0.99], 0.1,
                                     1.0, 2.0, 1.0, 1.0, 0.01)
    assert list(st) == [0, 1, 1, 1] and list(Ld) == [-2.0, 1.0, 1.0, 1.0]
    st, _ = kin.dynamic_instability([1], [1.95], [0.99], 0.1, 1.0, 2.0, 1.0, 1.0, 0.01, L_max=2.0)
    assert list(st) == [0]
