"""Pin of the whole discrete system on the sedimenting cloud of Sec. 4.3: the
mean settling velocity of a dilute cloud of N_F short fibers, centres uniform
in a ball of radius R0, approaches (N_F - 1)/N_F V_c + v_self, where
V_c = N_F F / (5 pi mu R0) is the Hadamard-Rybczynski speed of a drop with the
suspension's viscosity (the volume average of the flow of a uniformly forced
ball) and v_self = f0 [ (1/3) 2c + (2/3)(c + 2) ] / (8 pi mu) is one rod's
orientation-averaged slender-body settling speed, c = -ln(eps^2 e).  Neither
value comes from the implementation; the random sample makes the agreement
statistical (~1 %), gate 3 %."""
import math

import workloads as wl
from oracle import kernels as ok
from oracle import system


def closed_form(s):
    c = -math.log(s.eps ** 2 * math.e)
    v_self = abs(s.f_ext[0, 2]) * (2.0 * c / 3.0 + 2.0 * (c + 2.0) / 3.0) / (8.0 * math.pi * s.mu)
    M = s.n_fibers
    return (M - 1) / M * wl.cloud_velocity_scale(s) + v_self


def test_dilute_cloud_settles_at_the_drop_speed():
    ok.build()
    s = wl.sedimenting_cloud(0.15, M=256, N=16, seed=1)
    r = system.from_suspension(s).step(tol=1e-10)
    vz = -float(r.V[:, 2].mean())
    assert abs(vz / closed_form(s) - 1.0) <= 0.03
    # the horizontal mean velocity is zero up to the sample's fluctuations
    assert abs(float(r.V[:, 0].mean())) <= 0.03 * vz and abs(float(r.V[:, 1].mean())) <= 0.03 * vz
