"""GMRES restart cycles as CUDA graphs (fs_options.use_graph = 1): the
Givens rotations, the convergence test and the loop condition run on the
device inside a conditional WHILE node, one graph launch per cycle.  The step
must give the result of the host-driven cycle (use_graph = 0): the same
iteration counts and velocities within rounding (the device's hypot and
fused multiply-adds may differ from the host's in the last bit), for one
system, a batch of uneven systems, restarted cycles, and the mixed path.
The mixed path stops its inner solve at 1e-6 and corrects with a float-float
residual, so a last-bit change of its first solution moves the corrected one
within the band its tolerance leaves (measured 5e-9 in V at tol 1e-10): gate
1e-8 there.  FP64 path: one step agrees to 1e-12; over two steps the first
step's last-bit differences enter the second step's blocks, whose tensor-core
build rounds each entry to ~3e-15 of its products (measured 3.7e-11 at
N = 32): gate 1e-10 for the two-step case."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import dev, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402


def batch_step(ss, prec, tol, graph, restart=60, steps=1):
    opt = fs.fs_options_default()
    opt.prec = prec
    opt.tol = tol
    opt.use_graph = 1 if graph else 0
    opt.restart = restart
    fps = [s.n_fibers for s in ss]
    ppf = np.concatenate([s.n_per_fiber for s in ss])
    if len(ss) == 1:
        h = fs.fs_create(ppf, 1.0, 1e-3, 1.0, 1e-3, options=opt)
    else:
        h = fs.fs_create_batch(fps, ppf, 1.0, 1e-3, 1.0, 1e-3, options=opt)
    X = dev(np.concatenate([s.X for s in ss]), torch)
    L = dev(np.concatenate([s.L for s in ss]), torch)
    F = dev(np.concatenate([s.f_ext for s in ss]), torch)
    fs.fs_set_state(h, X, L, F)
    n0 = fs.fs_kernel_launches()
    infos = [fs.fs_step(h) for _ in range(steps)]
    launches = fs.fs_kernel_launches() - n0
    binfo = fs.fs_batch_info(h) if len(ss) > 1 else None
    V = torch.empty_like(X)
    fs.fs_get_state(h, V=V)
    fs.fs_destroy(h)
    return V.cpu().numpy(), infos, binfo, launches


def uneven():
    out = []
    for k, (M, N) in enumerate([(3, 16), (9, 32), (1, 24), (14, 16), (6, 32), (20, 24)]):
        s = wl.free_space(M, N, 3.0 + M ** (1 / 3), seed=70 + k, curved_amp=0.05)
        s.f_ext = np.tile([0.2 * k, -0.1, -1.0], (s.n_points, 1))
        out.append(s)
    return out


@pytest.mark.parametrize("prec,tol", [(fs.FS_FP64, 1e-12), (fs.FS_MIXED, 1e-10)])
def test_one_system_graph_equals_host_cycle(prec, tol):
    s = wl.free_space(24, 32, 6.0, seed=4, curved_amp=0.05)
    s.f_ext = np.tile([0.1, 0.0, -1.0], (s.n_points, 1))
    Vh, ih, _, lh = batch_step([s], prec, tol, graph=False, steps=2)
    Vg, ig, _, lg = batch_step([s], prec, tol, graph=True, steps=2)
    assert [i.iters for i in ig] == [i.iters for i in ih]
    assert rel(Vg, Vh) <= (1e-10 if prec == fs.FS_FP64 else 1e-8)
    assert lg > 0


@pytest.mark.parametrize("prec,tol", [(fs.FS_FP64, 1e-12), (fs.FS_MIXED, 1e-10)])
def test_uneven_batch_graph_equals_host_cycle(prec, tol):
    ss = uneven()
    Vh, _, bh, _ = batch_step(ss, prec, tol, graph=False)
    Vg, _, bg, _ = batch_step(ss, prec, tol, graph=True)
    assert list(bg["iters"]) == list(bh["iters"])
    assert all(bg["converged"])
    assert rel(Vg, Vh) <= (1e-12 if prec == fs.FS_FP64 else 1e-8)


def test_restarted_cycles():
    """restart = 3 forces several cycles per solve (restart vectors, per-system
    convergence across cycles)."""
    ss = uneven()
    Vh, _, bh, _ = batch_step(ss, fs.FS_FP64, 1e-12, graph=False, restart=3)
    Vg, _, bg, _ = batch_step(ss, fs.FS_FP64, 1e-12, graph=True, restart=3)
    assert list(bg["iters"]) == list(bh["iters"])
    assert max(bg["iters"]) > 3
    assert rel(Vg, Vh) <= 1e-11
