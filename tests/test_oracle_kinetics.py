"""Pins of fiber (de)polymerization (Sec. 2.4 kinetics; the dynamic
instability of Sec. 5) in the oracle:
* a force-free straight fiber with plus-end growth rate Ldot extends exactly:
  its minus end stays, its plus end advances by Ldot dt, tension zero;
* a curved fiber gains dt Ldot of arclength from the growth term (the
  material is inextensible; only the plus end adds length);
* the step is affine in Ldot up to O(dt Ldot / L) (the growth term is taken
  at the new time, which puts dt Ldot / (L + dt Ldot) into the self block);
* the two-state dynamic instability reaches the Dogterom-Leibler stationary
  mean length v_g v_s / (v_s f_cat - v_g f_res) (+ the nucleation length)."""
import numpy as np

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


def test_straight_fiber_grows_at_its_plus_end():
    ok.build()
    s = wl.free_space(3, 16, 20.0, seed=1)
    s.f_ext[:] = 0.0
    Ldot = np.array([0.7, -0.4, 2.0])
    r = system.from_suspension(s, Ldot=Ldot).step(tol=1e-13)
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


def test_curved_fiber_gains_the_grown_length():
    """The length a growth rate adds to a curved fiber in one step is dt Ldot
    (the rest of the step's length change -- the linearised inextensibility
    acting on the bending relaxation -- is the same with and without growth),
    to 5e-4 relative (measured 1.3e-4 and 9.5e-5 at dt = 1e-3, 1e-4)."""
    ok.build()
    rels = []
    for dt in (1e-3, 1e-4):
        s = wl.free_space(1, 24, 5.0, seed=2, curved_amp=0.1, dt=dt)
        s.f_ext[:] = 0.0
        Ldot = 1.5
        grown = arclength(system.from_suspension(s, Ldot=np.array([Ldot])).step(tol=1e-13).X_new)
        fixed = arclength(system.from_suspension(s).step(tol=1e-13).X_new)
        rels.append(abs((grown - fixed) / (dt * Ldot) - 1.0))
    assert max(rels) <= 5e-4


def test_step_is_affine_in_the_growth_rate_to_first_order():
    """The known part of the growth term is linear in Ldot; its part at the
    new time adds dt kappa (y + 1) V_alpha to the self block, so V is affine
    in Ldot up to relative O(dt Ldot / L)."""
    ok.build()
    s = wl.free_space(4, 16, 6.0, seed=3, curved_amp=0.05)
    s.f_ext = np.tile([0.0, 0.0, -1.0], (s.n_points, 1))
    Ld = np.array([0.5, -0.3, 1.0, 0.2])
    V0 = system.from_suspension(s).step(tol=1e-13).V
    V1 = system.from_suspension(s, Ldot=Ld).step(tol=1e-13).V
    V2 = system.from_suspension(s, Ldot=2.0 * Ld).step(tol=1e-13).V
    bound = 10.0 * s.dt * np.max(np.abs(Ld) / s.L)
    assert np.linalg.norm((V2 - V0) - 2.0 * (V1 - V0)) <= bound * np.linalg.norm(V1 - V0)


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


def test_shrinking_fiber_stays_smooth():
    """A curved fiber shrinking by 0.144 per step (dt |Ldot| / L from 0.04 to
    0.13) for 20 steps, 4 -> 1.12 in length, keeps its discrete length equal
    to L (within 1 %) and its velocities bounded: the reparametrisation term
    is taken at the new time (with it explicit, shrinking fibers blew up
    within tens of far milder steps)."""
    ok.build()
    s = wl.free_space(1, 16, 5.0, seed=4, curved_amp=0.05, L_range=(4.0, 4.0), E=10.0, dt=0.1)
    s.f_ext = np.tile([0.0, 0.0, -0.05], (s.n_points, 1))
    X, L = s.X.copy(), s.L.copy()
    for _ in range(20):
        sub = wl.Suspension(s.n_per_fiber, X, L, s.f_ext, s.mu, s.eps, s.E, s.dt)
        r = system.from_suspension(sub, Ldot=np.array([-0.288 * 5.0])).step(tol=1e-12)
        X, L = r.X_new, r.L_new
        assert np.isfinite(r.V).all() and np.abs(r.V).max() < 10.0
    assert L[0] < 0.3 * s.L[0]
    assert abs(arclength(X) / L[0] - 1.0) <= 0.01
