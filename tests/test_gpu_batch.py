"""Batched independent systems (fs_create_batch): every system of an uneven
batch (different fiber counts and points per fiber) gives the same velocities
as the same system solved alone, within the solver tolerance, and matches the
oracle; smooth forcing, FP64 and mixed precision."""
import numpy as np
import pytest

import workloads as wl
from oracle import system
from tests.gpu_helpers import dev, gpu_step, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402


def systems():
    out = []
    for k, (M, N) in enumerate([(3, 16), (9, 32), (1, 24), (14, 16), (6, 32)]):
        s = wl.free_space(M, N, 3.0 + M ** (1 / 3), seed=20 + k, curved_amp=0.05)
        s.f_ext = np.tile([0.2 * k, -0.1, -1.0], (s.n_points, 1))
        out.append(s)
    return out


def run_batch(ss, prec, tol):
    opt = fs.fs_options_default()
    opt.prec = prec
    opt.tol = tol
    fps = [s.n_fibers for s in ss]
    ppf = np.concatenate([s.n_per_fiber for s in ss])
    h = fs.fs_create_batch(fps, ppf, 1.0, 1e-3, 1.0, 1e-3, options=opt)
    X = dev(np.concatenate([s.X for s in ss]), torch)
    L = dev(np.concatenate([s.L for s in ss]), torch)
    F = dev(np.concatenate([s.f_ext for s in ss]), torch)
    fs.fs_set_state(h, X, L, F)
    fs.fs_step(h)
    info = fs.fs_batch_info(h)
    V = torch.empty_like(X)
    fs.fs_get_state(h, V=V)
    fs.fs_destroy(h)
    out, o = [], 0
    for s in ss:
        out.append(V[o:o + s.n_points].cpu().numpy())
        o += s.n_points
    return out, info


@pytest.mark.parametrize("prec,tol,gate,ogate", [(fs.FS_FP64, 1e-12, 1e-10, 5e-9),
                                                 (fs.FS_MIXED, 1e-10, 2e-8, 1e-8)])
def test_batch_equals_alone_and_oracle(prec, tol, gate, ogate):
    """alone vs in the batch: gate; vs the oracle: ogate.  These curved systems
    have cond(A) ~2e9: the oracle's own FP64 solutions of one system -- its
    GMRES, a dense LU solve of A, a dense LU solve of P^-1 A -- differ by up
    to 8.5e-10 (9 x 32 fibers) and 3.2e-9 (6 x 32), so FP64 ogate = 5e-9.
    Mixed: the batch's work-list far field and the single system's one-wave
    far field add the FP32 terms in different orders, so the two solves are
    two different roundings, each within ogate of the oracle: gate 2 x ogate."""
    ss = systems()
    Vb, info = run_batch(ss, prec, tol)
    assert np.all(info["converged"] == 1)
    for k, s in enumerate(ss):
        Va, _, _, _ = gpu_step(s, torch, prec=prec, tol=tol)
        assert rel(Vb[k], Va) <= gate, k
        ref = system.from_suspension(s).step(tol=1e-12)
        assert rel(Vb[k], ref.V) <= ogate, k


def test_batch_of_one_equals_single_context():
    s = systems()[1]
    Vb, info = run_batch([s], fs.FS_FP64, 1e-12)
    Va, _, _, infos = gpu_step(s, torch, prec=fs.FS_FP64, tol=1e-12)
    assert rel(Vb[0], Va) <= 1e-13
