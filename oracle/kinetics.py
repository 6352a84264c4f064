"""Microtubule dynamic instability (oracle; test infrastructure -- only tests,
the smoke check and the benchmark's CPU baseline use this module).

Two-state model of Sec. 2.4 / Sec. 5 (kinetics): a fiber's plus end grows at
v_grow or shrinks at v_shrink and switches between the two at the catastrophe
rate f_cat (growing -> shrinking) and the rescue rate f_res (shrinking ->
growing).  One time step of length dt, given one uniform random number
u in [0, 1) per fiber (the random numbers are inputs, not drawn here):

    growing:   switch to shrinking if u < 1 - exp(-f_cat dt)
    shrinking: switch to growing   if u < 1 - exp(-f_res dt)
    a shrinking fiber that would pass below L_min is rescued (grows);
    a growing fiber that would pass L_max (> 0) switches to shrinking;
    Ldot = v_grow (growing) or -v_shrink (shrinking).

The load-dependent growth speed of the paper needs the plus-end force, which
is zero at a free end; v_grow is constant here.
"""
from __future__ import annotations

import math

import numpy as np


def dynamic_instability(state, L, u, dt, v_grow, v_shrink, f_cat, f_res, L_min, L_max=0.0):
    """Advance the per-fiber states (1 growing, 0 shrinking) by one step;
    returns (new_state, Ldot).  The rules above, applied to all fibers at
    once: the switch, then the rescue at L_min, else the cap at L_max (Sec. 2.4, Sec. 5)."""
    state = np.asarray(state, dtype=np.int32)
    L = np.asarray(L, dtype=float)
    u = np.asarray(u, dtype=float)
    p_cat = -math.expm1(-f_cat * dt)
    p_res = -math.expm1(-f_res * dt)
    flip = np.where(state == 1, u < p_cat, u < p_res)
    new = np.where(flip, 1 - state, state).astype(np.int32)
    rescue = (new == 0) & (L - v_shrink * dt < L_min)
    cap = ~rescue & (new == 1) & (L_max > 0.0) & (L + v_grow * dt > L_max)
    new = np.where(rescue, 1, np.where(cap, 0, new)).astype(np.int32)
    Ldot = np.where(new == 1, v_grow, -v_shrink).astype(float)
    return new, Ldot


def mean_length_bounded(v_grow, v_shrink, f_cat, f_res):
    """Stationary mean length of the two-state model in the bounded regime
    v_shrink f_cat > v_grow f_res with nucleation at zero length (Dogterom and
    Leibler, Phys. Rev. Lett. 70, 1993): exponential lengths of mean
    v_grow v_shrink / (v_shrink f_cat - v_grow f_res)."""
    den = v_shrink * f_cat - v_grow * f_res
    if den <= 0.0:
        raise ValueError("unbounded growth regime")
    return v_grow * v_shrink / den
