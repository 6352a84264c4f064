"""Fast summation (treecode) of the Stokeslet far field against the oracle's
FP64 direct sum (the direct sum is the exact target: the expansion has a
truncation error that falls with its order and with the opening angle).

Measured on GB300 (relative 2-norm error over all targets, 19,200 points on
300 curved fibers, own-fiber pairs excluded): at theta = 0.5, orders 4, 6, 8
and 10 give 1.3e-3, 1.7e-4, 2.6e-5 and 4.6e-6; at order 8, theta = 0.7,
0.5 and 0.35 give 5.1e-4, 2.6e-5 and 2.2e-6.  The gates allow up to 1.5 to
2.3 times those numbers, and the error must fall with the order and with theta
(a wrong expansion coefficient or moment shift stalls the convergence:
before a missing charge-shift term was fixed, all orders sat at 3e-2).  Full
size: 1,048,576 points, order 8, theta 0.4: 5.7e-6 on 256 sampled targets."""
import numpy as np
import pytest

import workloads as wl
from oracle import kernels as ok
from tests.gpu_helpers import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    ok.build()
    h = fs.fs_create([], 1.0, 1e-3, 1.0, 1e-3)
    yield h
    fs.fs_destroy(h)


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


@pytest.fixture(scope="module")
def fibers():
    s = wl.free_space(300, 64, 20.0, seed=1, curved_amp=0.05)
    wf = s.f_ext * 0.02
    fid = s.fiber_id()
    ref = ok.stokeslet(s.X, s.X, wf, 1.0, fid, fid)
    return s, wf, fid, ref


def tree(h, X, W, T, Fs=None, Ft=None, order=8, theta=0.5):
    out = torch.empty_like(T)
    fs.fs_stokeslet_apply_tree(h, X, W, T, out, Fs, Ft, order=order, theta=theta)
    return out.cpu().numpy()


def test_error_falls_with_order(ctx, fibers):
    s, wf, fid, ref = fibers
    X, W, F = dev(s.X), dev(wf), dev(fid, torch.int32)
    gates = {4: 2e-3, 6: 3e-4, 8: 4e-5, 10: 1e-5}
    errs = []
    for order, gate in gates.items():
        e = rel(tree(ctx, X, W, X, F, F, order, 0.5), ref)
        print("order %d theta 0.5: %.3e" % (order, e))
        assert e <= gate
        errs.append(e)
    assert all(b < a / 2 for a, b in zip(errs, errs[1:]))


def test_error_falls_with_opening_angle(ctx, fibers):
    s, wf, fid, ref = fibers
    X, W, F = dev(s.X), dev(wf), dev(fid, torch.int32)
    errs = []
    for theta, gate in ((0.7, 7e-4), (0.5, 4e-5), (0.35, 5e-6)):
        e = rel(tree(ctx, X, W, X, F, F, 8, theta), ref)
        print("order 8 theta %.2f: %.3e" % (theta, e))
        assert e <= gate
        errs.append(e)
    assert errs[0] > errs[1] > errs[2]


def test_separate_targets_without_exclusion(ctx, fibers):
    s, wf, _, _ = fibers
    T = np.random.default_rng(3).uniform(0.0, 20.0, size=(5000, 3))
    ref = ok.stokeslet(T, s.X, wf, 1.0)
    e = rel(tree(ctx, dev(s.X), dev(wf), dev(T), order=8, theta=0.5), ref)
    assert e <= 1e-5


def test_small_inputs_are_exact_direct_sums(ctx):
    # fewer points than a leaf holds: the root is a leaf, every pair is direct
    rng = np.random.default_rng(5)
    for n in (1, 2, 33, 64):
        X = rng.uniform(-1.0, 1.0, size=(n, 3))
        wf = rng.normal(size=(n, 3))
        T = rng.uniform(-1.0, 1.0, size=(7, 3))
        ref = ok.stokeslet(T, X, wf, 1.0)
        assert rel(tree(ctx, dev(X), dev(wf), dev(T), order=4, theta=0.5), ref) <= 1e-6
    # self sum with exclusion of one fiber of 10 points: the result is zero
    X = rng.uniform(size=(10, 3))
    F = dev(np.zeros(10, dtype=np.int32), torch.int32)
    out = tree(ctx, dev(X), dev(rng.normal(size=(10, 3))), dev(X), F, F)
    assert np.abs(out).max() <= 1e-5
    # no targets / no sources
    empty = torch.empty((0, 3), dtype=torch.float64, device="cuda:0")
    assert tree(ctx, dev(X), dev(X), empty).shape == (0, 3)
    assert np.all(tree(ctx, empty, empty, dev(X)) == 0.0)


def test_bad_arguments_are_rejected(ctx):
    X = dev(np.random.default_rng(0).uniform(size=(100, 3)))
    out = torch.empty_like(X)
    for order, theta in ((5, 0.5), (12, 0.5), (8, 0.0), (8, 1.0)):
        with pytest.raises(fs.FsError):
            fs.fs_stokeslet_apply_tree(ctx, X, X, X, out, order=order, theta=theta)


def test_full_size_sampled_against_the_oracle(ctx):
    s = wl.cfg_large_matvec(0)
    wf = s.f_ext * 0.01
    fid = s.fiber_id()
    idx = np.linspace(0, s.n_points - 1, 256).astype(np.int64)
    ref = ok.stokeslet(s.X[idx], s.X, wf, 1.0, fid[idx], fid)
    X, F = dev(s.X), dev(fid, torch.int32)
    out = tree(ctx, X, dev(wf), X, F, F, order=8, theta=0.4)
    e = rel(out[idx], ref)
    print("1,048,576 points, order 8 theta 0.4: sampled error %.3e" % e)
    assert e <= 1e-5


@pytest.mark.parametrize("prec,tol", [(fs.FS_FP64, 1e-8), (fs.FS_MIXED, 1e-8)])
def test_step_with_the_treecode_far_field(prec, tol):
    """fs_step with tree_order set: every fiber-fiber far field is the
    treecode, so the step solves the treecode's system; its velocities differ
    from the direct step's by the treecode's error (here 6,400 points, order
    8, theta 0.4)."""
    from tests.gpu_helpers import gpu_step
    s = wl.free_space(200, 32, 15.0, seed=4, curved_amp=0.05)
    V_ref, _, _, _ = gpu_step(s, torch, prec=fs.FS_FP64, tol=1e-11)
    opt = fs.fs_options_default()
    opt.prec, opt.tol, opt.tree_order, opt.tree_theta = prec, tol, 8, 0.4
    h = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, options=opt)
    X = dev(s.X)
    fs.fs_set_state(h, X, dev(s.L), dev(s.f_ext))
    info = fs.fs_step(h)
    V = torch.empty_like(X)
    fs.fs_get_state(h, V=V)
    fs.fs_destroy(h)
    e = rel(V.cpu().numpy(), V_ref)
    print("tree step (prec %d): velocity difference %.3e, %d iterations" % (prec, e, info.iters))
    assert info.resid <= tol
    assert e <= 1e-4
