"""The library's dynamic-instability step (host code, no GPU) against the
oracle's, bit for bit, on random states, lengths and random numbers over
many steps; and its argument checks."""
import numpy as np
import pytest

from oracle import kinetics as kin
from paper_1602_05650_gb300 import build


@pytest.fixture(scope="module")
def fs():
    build.build()
    import paper_1602_05650_gb300 as m
    return m


@pytest.mark.parametrize("L_max", [0.0, 3.0])
def test_matches_oracle_bitwise(fs, L_max):
    rng = np.random.default_rng(5)
    n = 5000
    state = rng.integers(0, 2, n).astype(np.int32)
    L = rng.uniform(0.05, 3.0, n)
    so, sl = state.copy(), state.copy()
    Lo = L.copy()
    args = (0.01, 1.0, 2.5, 0.8, 0.3, 0.05, L_max)
    for _ in range(200):
        u = rng.random(n)
        so, Ldo = kin.dynamic_instability(so, Lo, u, *args)
        sl, Ldl = fs.fs_dynamic_instability(sl, Lo, u, *args)
        assert np.array_equal(so, sl)
        assert np.array_equal(Ldo, Ldl)
        Lo = Lo + args[0] * Ldo
    assert Lo.min() > 0.0


def test_rejects_bad_arguments(fs):
    with pytest.raises(fs.FsError):
        fs.fs_dynamic_instability([1], [1.0], [0.5], -1.0, 1.0, 1.0, 1.0, 1.0, 0.1)
    with pytest.raises(fs.FsError):
        fs.fs_dynamic_instability([1], [1.0], [0.5], 0.1, -1.0, 1.0, 1.0, 1.0, 0.1)
    nan, inf = float("nan"), float("inf")
    for dt, vg, vs, fc, fr, lmin, lmax in ((0.1, nan, 1.0, 1.0, 1.0, 0.1, 0.0),
                                           (0.1, 1.0, 1.0, nan, 1.0, 0.1, 0.0),
                                           (0.1, 1.0, inf, 1.0, 1.0, 0.1, 0.0),
                                           (nan, 1.0, 1.0, 1.0, 1.0, 0.1, 0.0),
                                           (0.1, 1.0, 1.0, 1.0, 1.0, nan, 0.0)):
        with pytest.raises(fs.FsError):
            fs.fs_dynamic_instability([1], [1.0], [0.5], dt, vg, vs, fc, fr, lmin, lmax)
