"""The assembled self blocks B_m of Eq. prec (fs_get_self_block) for the
tensor-core build (split bf16 operands, fs_options.tc_blocks = 1, the
default) and the FP64 CUDA-core build: straight and curved fibers, 16 to 64
points, a ragged mix of point counts, local slender-body theory, and a
growing fiber with the implicit growth term.

Scale.  B = Rd + Rw S F sums products with cancellation (the tension rows
X_s . D_z w nearly vanish), and the operands themselves come out of
cancelling sums (the tension-column forces, the geometry), so an entry's
rounding is set by its row's product magnitude, max_j G_ij with
G = |Rd| + |Rw| |S| |F|.  Gates:
* library against the oracle, every entry within 2e-12 of its row's product
  magnitude (measured 1.3e-14, 5.6e-14, 4.5e-13 at N = 16, 32, 64, the same
  for both builds: it grows like N^2 with the rounding of the geometry's
  derivatives, double-double in the library, long double in the oracle);
* tensor-core build against the FP64 build, every entry within 1e-14 of its
  own product magnitude G_ij (measured 2.9e-15 on 64 cloud fibers): the
  emulated products are FP64-grade entry by entry."""
import numpy as np
import pytest

import workloads as wl
from oracle import system
from tests.gpu_helpers import dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402


def gpu_blocks(s, tc, lsb=False, Ldot=None, growth_implicit=False):
    opt = fs.fs_options_default()
    opt.tc_blocks = 1 if tc else 0
    opt.lsb = 1 if lsb else 0
    opt.growth_implicit = 1 if growth_implicit else 0
    h = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, options=opt)
    fs.fs_set_state(h, dev(s.X, torch), dev(s.L, torch), dev(s.f_ext, torch))
    if Ldot is not None:
        fs.fs_set_growth(h, np.asarray(Ldot, float))
    out = [fs.fs_get_self_block(h, m, int(s.n_per_fiber[m])) for m in range(s.n_fibers)]
    fs.fs_destroy(h)
    return out


def scale_of(fb):
    """G = |Rd| + |Rw| |S| |F|: the magnitude of the products an entry sums."""
    return np.abs(fb.Rd) + np.abs(fb.Rw) @ (np.abs(fb.S) @ np.abs(fb.F))


def row_rel(Bg, Bo, G):
    """Largest |difference| over its row's product magnitude max_j G_ij."""
    return float((np.abs(Bg - Bo) / np.maximum(G.max(axis=1, keepdims=True), 1e-300)).max())


def entry_rel(Ba, Bb, G):
    """Largest |difference| / G_ij over the entries whose products do not all
    vanish (below 1e-13 of the row, compared at that level)."""
    floor = 1e-13 * G.max(axis=1, keepdims=True)
    return float((np.abs(Ba - Bb) / np.maximum(np.maximum(G, floor), 1e-300)).max())


CASES = {
    "straight_16": lambda: wl.free_space(6, 16, 4.0, seed=1),
    "curved_32": lambda: wl.free_space(6, 32, 5.0, seed=2, curved_amp=0.05),
    "curved_64": lambda: wl.free_space(4, 64, 6.0, seed=3, curved_amp=0.05),
    "ragged": lambda: wl.free_space(5, np.array([16, 24, 32, 20, 64]), 5.0, seed=4, curved_amp=0.05),
}


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("name", sorted(CASES))
def test_blocks_match_oracle(name, tc):
    s = CASES[name]()
    sy = system.from_suspension(s)
    got = gpu_blocks(s, tc)
    worst = max(row_rel(g, fb.B, scale_of(fb)) for g, fb in zip(got, sy.fibers))
    print("%s tc=%d: worst difference / row product magnitude %.2e" % (name, tc, worst))
    assert worst <= 2e-12


@pytest.mark.parametrize("tc", [True, False])
def test_blocks_lsb_and_implicit_growth(tc):
    s = wl.free_space(4, 32, 5.0, seed=5, curved_amp=0.05)
    Ld = np.array([0.4, -0.3, 0.0, 1.0])
    sy = system.from_suspension(s, lsb=True)
    got = gpu_blocks(s, tc, lsb=True)
    assert max(row_rel(g, fb.B, scale_of(fb)) for g, fb in zip(got, sy.fibers)) <= 2e-12
    sy = system.from_suspension(s, Ldot=Ld, growth="implicit")
    got = gpu_blocks(s, tc, Ldot=Ld, growth_implicit=True)
    assert max(row_rel(g, fb.B, scale_of(fb)) for g, fb in zip(got, sy.fibers)) <= 2e-12


def test_tensor_core_build_equals_fp64_build():
    s = wl.cfg_cloud_mixed(0)
    sub = wl.Suspension(s.n_per_fiber[:64], s.X[:64 * 64], s.L[:64], s.f_ext[:64 * 64], s.mu, s.eps, s.E, s.dt)
    a = gpu_blocks(sub, True)
    b = gpu_blocks(sub, False)
    sy = system.from_suspension(sub)
    worst = max(entry_rel(x, y, scale_of(fb)) for x, y, fb in zip(a, b, sy.fibers))
    print("cloud fibers, tensor-core vs FP64 build: %.2e of the product magnitude" % worst)
    assert worst <= 1e-14
