"""Sedimenting cloud of Sec. 4.3 on the GPU: parity with the oracle on a
256-fiber cloud, the closed-form settling speed of a dilute 1,024-fiber cloud
(see tests/test_oracle_sediment.py for its derivation), and the four fiber
lengths of the paper stepped together as one batch."""
import numpy as np
import pytest

import workloads as wl
from oracle import system
from tests.gpu_helpers import dev, gpu_step, rel
from tests.test_oracle_sediment import closed_form

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402


@pytest.mark.parametrize("prec,tol,gate", [(fs.FS_FP64, 1e-12, 1e-10), (fs.FS_MIXED, 1e-10, 1e-8)])
def test_cloud_matches_oracle(prec, tol, gate):
    s = wl.sedimenting_cloud(0.32, M=256, N=16, seed=2)
    ref = system.from_suspension(s).step(tol=1e-12)
    V, T, X, _ = gpu_step(s, torch, prec=prec, tol=tol)
    assert rel(V, ref.V) <= gate
    assert rel(X, ref.X_new) <= gate


def test_dilute_cloud_settles_at_the_drop_speed():
    s = wl.sedimenting_cloud(0.15, M=1024, N=16, seed=3)
    V, _, _, infos = gpu_step(s, torch, prec=fs.FS_MIXED, tol=1e-8)
    vz = -float(V[:, 2].mean())
    assert abs(vz / closed_form(s) - 1.0) <= 0.03


def test_four_lengths_batched_and_advanced():
    """The four lengths of the paper (L/R0 = 0.15, 0.25, 0.32, 0.40) as one
    batch, advanced 4 steps: the first step equals each cloud alone, every
    cloud settles (its centre of mass moves down by its mean velocity x dt),
    and longer fibers (denser clouds) settle faster."""
    clouds = [wl.sedimenting_cloud(Lr, M=256, N=16, seed=10 + k) for k, Lr in enumerate((0.15, 0.25, 0.32, 0.40))]
    opt = fs.fs_options_default()
    opt.tol = 1e-10
    h = fs.fs_create_batch([c.n_fibers for c in clouds], np.concatenate([c.n_per_fiber for c in clouds]),
                           1.0, 0.01, 3.2e-3, clouds[0].dt, options=opt)
    X = dev(np.concatenate([c.X for c in clouds]), torch)
    fs.fs_set_state(h, X, dev(np.concatenate([c.L for c in clouds]), torch),
                    dev(np.concatenate([c.f_ext for c in clouds]), torch))
    V = torch.empty_like(X)
    Xn = torch.empty_like(X)
    sizes = [c.n_points for c in clouds]
    speeds = []
    for step in range(4):
        x0 = X.clone() if step == 0 else Xn.clone()
        fs.fs_step(h)
        fs.fs_get_state(h, X=Xn, V=V)
        assert bool(torch.isfinite(Xn).all())
        o = 0
        for k, c in enumerate(clouds):
            v = V[o:o + sizes[k]].cpu().numpy()
            dz = (Xn[o:o + sizes[k], 2] - x0[o:o + sizes[k], 2]).mean().item()
            assert dz < 0.0
            assert abs(dz - c.dt * v[:, 2].mean()) <= 1e-12 * abs(dz) + 1e-15
            if step == 0:
                Va, _, _, _ = gpu_step(c, torch, prec=fs.FS_MIXED, tol=1e-10)
                assert rel(v, Va) <= 2e-8
                speeds.append(-v[:, 2].mean())
            o += sizes[k]
    fs.fs_destroy(h)
    assert speeds == sorted(speeds)
