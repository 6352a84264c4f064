"""Helpers shared by the GPU tests: run the library on a workloads.Suspension."""
import numpy as np

import paper_1602_05650_gb300 as fs


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a, torch, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda:0")


def make_ctx(s, prec=fs.FS_FP64, tol=1e-12, lsb=False, delta_over_L=0.01, restart=60, max_iter=300,
             relax=None, profile=False, growth_implicit=False):
    opt = fs.fs_options_default()
    opt.growth_implicit = 1 if growth_implicit else 0
    if relax is not None:
        opt.relax = 1 if relax else 0
    opt.profile = 1 if profile else 0
    opt.prec = prec
    opt.tol = tol
    opt.lsb = 1 if lsb else 0
    opt.delta_over_L = delta_over_L
    opt.restart = restart
    opt.max_iter = max_iter
    return fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, boundary=s.boundary, options=opt)


def gpu_step(s, torch, steps=1, **kw):
    h = make_ctx(s, **kw)
    X = dev(s.X, torch)
    fs.fs_set_state(h, X, dev(s.L, torch), dev(s.f_ext, torch))
    infos = [fs.fs_step(h) for _ in range(steps)]
    V = torch.empty_like(X)
    T = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
    Xn = torch.empty_like(X)
    fs.fs_get_state(h, X=Xn, T=T, V=V)
    fs.fs_destroy(h)
    return V.cpu().numpy(), T.cpu().numpy(), Xn.cpu().numpy(), infos
