"""GPU parity of the direct sums (fs_stokeslet_apply, fs_stresslet_apply,
fs_surface_apply) against the oracle's plain FP64 C loops, element by element
on the same seeded inputs: sizes spanning several tiles with ragged tails,
fiber exclusion, the one-wave work split (runs of source tiles that end
inside a target block, several CTAs per block, many blocks per CTA), every
launch shape, edge cases and a sampled check at the 65,536-point cloud size.
Tolerances: FP64 arithmetic 1e-12 relative 2-norm; float-float 5e-11 (~2^-44
per pair, and coordinates carried as two floats, 2^-48 relative, which near
pairs of random points amplify); FP32 arithmetic 1e-6."""
import numpy as np
import pytest

import workloads as wl
from oracle import kernels as ok
from tests.gpu_helpers import dev, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402

FS_SUM_FF = 2
# FS_SUM_FP32_PLAIN keeps the coordinates of each thread's consecutive targets
# in a frame at its middle target: on fiber nodes (the sums of the step) the
# pair differences round relative to the fiber's extent, the accuracy of the
# hi/lo sum (1e-6).  Uniformly random points are not spatially grouped, so
# there the frame is the centre of the sources and the coordinates round to
# 2^-24 |x| (|x| <= side / 2 = 5), ~5e-7 absolute against pair distances of
# ~0.05 and more: 1e-5 relative.
TOL = {fs.FS_SUM_FP64: 1e-12, fs.FS_SUM_FP32: 1e-6, FS_SUM_FF: 5e-11, fs.FS_SUM_FP32_PLAIN: 1e-6}
TOL_RANDOM = dict(TOL)
TOL_RANDOM[fs.FS_SUM_FP32_PLAIN] = 1e-5


@pytest.fixture(scope="module")
def ctx():
    h = fs.fs_create([], 1.3, 1e-3, 1.0, 1e-3)
    yield h
    fs.fs_destroy(h)


def random_points(n, seed, side=10.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, side, (n, 3)), rng.normal(size=(n, 3))


def gpu_stokeslet(h, src, wf, tgt, prec, sf=None, tf=None):
    out = torch.empty((tgt.shape[0], 3), dtype=torch.float64, device="cuda:0")
    fs.fs_stokeslet_apply(h, dev(src, torch), dev(wf, torch), dev(tgt, torch), out,
                          None if sf is None else dev(sf, torch, torch.int32),
                          None if tf is None else dev(tf, torch, torch.int32), prec)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", [fs.FS_SUM_FP64, fs.FS_SUM_FP32, FS_SUM_FF, fs.FS_SUM_FP32_PLAIN])
@pytest.mark.parametrize("n_src,n_tgt", [(1, 1), (255, 3), (256, 257), (1000, 777), (5003, 129),
                                         (20000, 4100), (60000, 700), (700, 60000), (20011, 19997)])
def test_stokeslet_random_points(ctx, prec, n_src, n_tgt):
    src, wf = random_points(n_src, 1)
    tgt, _ = random_points(n_tgt, 2)
    got = gpu_stokeslet(ctx, src, wf, tgt, prec)
    ref = ok.stokeslet(tgt, src, wf, 1.3)
    assert rel(got, ref) <= TOL_RANDOM[prec]


@pytest.mark.parametrize("prec", [fs.FS_SUM_FP64, fs.FS_SUM_FP32, FS_SUM_FF, fs.FS_SUM_FP32_PLAIN])
@pytest.mark.parametrize("M,N,side", [(16, 32, 10.0), (97, 24, 12.0), (300, 64, 20.0)])
def test_stokeslet_fiber_exclusion(ctx, prec, M, N, side):
    s = wl.free_space(M, N, side, seed=3, curved_amp=0.05)
    fid = s.fiber_id()
    wf = s.f_ext * 0.03
    got = gpu_stokeslet(ctx, s.X, wf, s.X, prec, fid, fid)
    ref = ok.stokeslet(s.X, s.X, wf, 1.3, fid, fid)
    assert rel(got, ref) <= TOL[prec]
    assert np.all(np.isfinite(got))


@pytest.mark.parametrize("shape", [1, 2, 3])
def test_every_launch_shape_agrees(shape):
    opt = fs.fs_options_default()
    opt.tile_override = shape
    h = fs.fs_create([], 1.0, 1e-3, 1.0, 1e-3, options=opt)
    s = wl.free_space(40, 32, 10.0, seed=4)
    fid = s.fiber_id()
    for prec in (fs.FS_SUM_FP64, fs.FS_SUM_FP32, FS_SUM_FF, fs.FS_SUM_FP32_PLAIN):
        got = gpu_stokeslet(h, s.X, s.f_ext, s.X, prec, fid, fid)
        ref = ok.stokeslet(s.X, s.X, s.f_ext, 1.0, fid, fid)
        assert rel(got, ref) <= TOL[prec]
    fs.fs_destroy(h)


def test_empty_inputs(ctx):
    tgt, _ = random_points(10, 5)
    out = torch.full((10, 3), 7.0, dtype=torch.float64, device="cuda:0")
    e = torch.empty((0, 3), dtype=torch.float64, device="cuda:0")
    fs.fs_stokeslet_apply(ctx, e, e, dev(tgt, torch), out, None, None, fs.FS_SUM_FP32)
    torch.cuda.synchronize()
    assert torch.all(out == 0)
    fs.fs_stokeslet_apply(ctx, dev(tgt, torch), dev(tgt, torch), e, e, None, None, fs.FS_SUM_FP32)


def test_deterministic(ctx):
    s = wl.free_space(64, 32, 10.0, seed=6)
    fid = s.fiber_id()
    a = gpu_stokeslet(ctx, s.X, s.f_ext, s.X, fs.FS_SUM_FP32, fid, fid)
    b = gpu_stokeslet(ctx, s.X, s.f_ext, s.X, fs.FS_SUM_FP32, fid, fid)
    assert np.array_equal(a, b)


def test_cloud_size_sampled(ctx):
    """65,536-point curved-fiber cloud (1,024 x 64, [0,40]^3) with the launch
    configuration of the step: every target computed on the GPU, 512 sampled
    targets checked one by one against the oracle."""
    s = wl.cfg_cloud_mixed(0)
    fid = s.fiber_id()
    wf = s.f_ext * np.repeat(s.L / 64, 64)[:, None]
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(s.n_points, 512, replace=False))
    ref = ok.stokeslet(s.X[idx], s.X, wf, 1.3, fid[idx], fid)
    for prec in (fs.FS_SUM_FP32, fs.FS_SUM_FP64, FS_SUM_FF, fs.FS_SUM_FP32_PLAIN):
        got = gpu_stokeslet(ctx, s.X, wf, s.X, prec, fid, fid)
        err = rel(got[idx], ref)
        print("cloud 65,536 sampled: precision %d rel err %.3e" % (prec, err))
        assert err <= TOL[prec]


@pytest.mark.parametrize("prec", [fs.FS_SUM_FP64, fs.FS_SUM_FP32, FS_SUM_FF])
def test_stresslet_off_surface(ctx, prec):
    b = wl.sphere_quadrature(20.0, 8, 24)
    rng = np.random.default_rng(7)
    q = rng.normal(size=b.nodes.shape)
    d = rng.normal(size=(3000, 3))
    tgt = d / np.linalg.norm(d, axis=1, keepdims=True) * 18.0 * rng.uniform(0, 1, (3000, 1)) ** (1 / 3)
    out = torch.empty((3000, 3), dtype=torch.float64, device="cuda:0")
    fs.fs_stresslet_apply(ctx, dev(b.nodes, torch), dev(b.normals, torch), dev(b.weights, torch),
                          dev(q, torch), dev(tgt, torch), out, prec)
    torch.cuda.synchronize()
    ref = ok.stresslet(tgt, b.nodes, b.normals, b.weights, q)
    assert rel(out.cpu().numpy(), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [fs.FS_SUM_FP64, fs.FS_SUM_FP32, FS_SUM_FF])
def test_surface_operator(prec):
    b = wl.sphere_quadrature(20.0, 8, 16)
    s = wl.confined(2, 16, R=20.0, R_centres=5.0, n_theta=8, n_phi=16, seed=1)
    h = fs.fs_create(s.n_per_fiber, 1.0, 1e-3, 1.0, 1e-3, boundary=b)
    q = np.random.default_rng(8).normal(size=b.nodes.shape)
    out = torch.empty_like(dev(q, torch))
    fs.fs_surface_apply(h, dev(q, torch), out, prec)
    torch.cuda.synchronize()
    ref = ok.surface_self(b.nodes, b.normals, b.weights, q)
    assert rel(out.cpu().numpy(), ref) <= TOL[prec] * (10 if prec == fs.FS_SUM_FP32 else 1)
    fs.fs_destroy(h)
