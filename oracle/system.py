"""Global linear system of one implicit step and its GMRES solve (oracle).

Sec. 3.2-3.3: the linearised backward-Euler step gives A u = b
(Eq. sche-linear-eq) with fiber blocks (4N_m unknowns each) and, under
confinement, the periphery double-layer density q0 (3 unknowns per surface
node).  Coupling between bodies is the complementary velocity
(Eqs. complementary-uc, complementary-uf):

* fiber m nodes:  ubar = sum over other fibers of the Stokeslet line integral
  (Clenshaw-Curtis sources W f) + T_Gamma0[q0] (Eq. cortex-vel);
* surface rows:   -q0/2 + T[q0] + N[q0] + (fiber Stokeslets at the nodes) = 0
  (Eq. main-cortex-density), singular part by subtraction (Sec. 3.1.2).

Preconditioner (Eq. prec): exact fiber self-blocks B_m (LU with partial
pivoting) and the scalar diagonal of the surface self-block; left
preconditioned GMRES (Saad) with x0 = 0, modified Gram-Schmidt and Givens
rotations, stopping when ||P^-1(b - A u)|| <= tol ||P^-1 b||.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg

from . import kernels
from .fiber import Fiber


@dataclasses.dataclass
class StepResult:
    V: np.ndarray          # [N_tot, 3] fiber velocity at the nodes
    T: np.ndarray          # [N_tot] tension at the nodes
    X_new: np.ndarray      # [N_tot, 3] X + dt V
    q: Optional[np.ndarray]  # [n_s, 3] periphery density
    u: np.ndarray          # full unknown vector
    iters: int
    resid: float
    L_new: Optional[np.ndarray] = None   # [M] L + dt Ldot


class System:
    def __init__(self, X, L, n_per_fiber, f_ext, mu=1.0, eps=1e-3, E=1.0, dt=1e-3,
                 delta_over_L=0.01, lsb=False, boundary=None, Ldot=None):
        self.mu = mu
        self.n_per = np.asarray(n_per_fiber, dtype=np.int64)
        self.ptr = np.concatenate([[0], np.cumsum(self.n_per)])
        self.X = np.asarray(X, float)
        self.fibers: List[Fiber] = []
        for m in range(len(self.n_per)):
            a, b = self.ptr[m], self.ptr[m + 1]
            self.fibers.append(Fiber(self.X[a:b], float(L[m]), np.asarray(f_ext[a:b], float), mu,
                                     eps, E, dt, delta_over_L * float(L[m]), lsb,
                                     0.0 if Ldot is None else float(Ldot[m])))
        self.L = np.asarray(L, float)
        self.Ldot = np.zeros(len(self.n_per)) if Ldot is None else np.asarray(Ldot, float)
        self.uptr = np.concatenate([[0], np.cumsum(4 * self.n_per)])
        self.fid = np.repeat(np.arange(len(self.n_per), dtype=np.int32), self.n_per)
        self.Wall = np.concatenate([f.W for f in self.fibers]) if self.fibers else np.zeros(0)
        self.boundary = boundary
        self.n_s = 0 if boundary is None else boundary.nodes.shape[0]
        self.n_unknowns = int(self.uptr[-1]) + 3 * self.n_s
        self.lu = [scipy.linalg.lu_factor(f.B) for f in self.fibers]
        if boundary is not None:
            self.sdiag = kernels.surface_diag(boundary.nodes, boundary.normals, boundary.weights).reshape(-1)

    # --------------------------------------------------------------- pieces
    def _split(self, u):
        us = [u[self.uptr[m]:self.uptr[m + 1]] for m in range(len(self.fibers))]
        q = u[self.uptr[-1]:].reshape(-1, 3) if self.n_s else None
        return us, q

    def _couplings(self, f_nodes: np.ndarray, q):
        """Complementary velocities for nodal fiber forces f_nodes [N_tot,3]
        and density q: (ubar at fiber nodes [N_tot,3], fiber Stokeslets at the
        surface nodes [n_s,3] or None)."""
        wf = f_nodes * self.Wall[:, None]
        ub = kernels.stokeslet(self.X, self.X, wf, self.mu, self.fid, self.fid)
        us = None
        if self.n_s:
            b = self.boundary
            if q is not None:
                ub = ub + kernels.stresslet(self.X, b.nodes, b.normals, b.weights, q)
            us = kernels.stokeslet(b.nodes, self.X, wf, self.mu)
        return ub, us

    def matvec(self, u: np.ndarray) -> np.ndarray:
        us, q = self._split(u)
        f = np.concatenate([fb.f_lin(um) for fb, um in zip(self.fibers, us)])
        ub, usurf = self._couplings(f, q)
        out = np.zeros_like(u)
        for m, fb in enumerate(self.fibers):
            a, b = self.ptr[m], self.ptr[m + 1]
            out[self.uptr[m]:self.uptr[m + 1]] = fb.B @ us[m] + fb.rows_from_ubar(ub[a:b])
        if self.n_s:
            bd = self.boundary
            out[self.uptr[-1]:] = (kernels.surface_self(bd.nodes, bd.normals, bd.weights, q)
                                   + usurf).reshape(-1)
        return out

    def rhs(self) -> np.ndarray:
        f = np.concatenate([fb.f_known for fb in self.fibers])
        ub, usurf = self._couplings(f, None)
        b = np.zeros(self.n_unknowns)
        for m, fb in enumerate(self.fibers):
            a, c = self.ptr[m], self.ptr[m + 1]
            b[self.uptr[m]:self.uptr[m + 1]] = -(fb.rows_known() + fb.rows_from_ubar(ub[a:c]))
        if self.n_s:
            b[self.uptr[-1]:] = -usurf.reshape(-1)
        return b

    def precond(self, v: np.ndarray) -> np.ndarray:
        out = np.empty_like(v)
        for m in range(len(self.fibers)):
            sl = slice(self.uptr[m], self.uptr[m + 1])
            out[sl] = scipy.linalg.lu_solve(self.lu[m], v[sl])
        if self.n_s:
            out[self.uptr[-1]:] = v[self.uptr[-1]:] / self.sdiag
        return out

    # ---------------------------------------------------------------- GMRES
    def gmres(self, b: np.ndarray, tol: float, max_iter: int = 300, matvec=None):
        A = matvec or self.matvec
        r0 = self.precond(b)
        beta = np.linalg.norm(r0)
        n = b.shape[0]
        if beta == 0.0:
            return np.zeros(n), 0, 0.0
        Vb = [r0 / beta]
        H = np.zeros((max_iter + 1, max_iter))
        cs, sn = np.zeros(max_iter), np.zeros(max_iter)
        g = np.zeros(max_iter + 1)
        g[0] = beta
        j = 0
        for j in range(max_iter):
            w = self.precond(A(Vb[j]))
            for i in range(j + 1):                        # modified Gram-Schmidt
                H[i, j] = w @ Vb[i]
                w = w - H[i, j] * Vb[i]
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            for i in range(j):                            # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            if abs(g[j + 1]) <= tol * beta or hn == 0.0:
                break
            Vb.append(w / hn)
        k = j + 1
        y = scipy.linalg.solve_triangular(H[:k, :k], g[:k])
        x = np.zeros(n)
        for i in range(k):
            x += y[i] * Vb[i]
        return x, k, abs(g[k]) / beta

    def step(self, tol: float = 1e-10, max_iter: int = 300) -> StepResult:
        b = self.rhs()
        u, its, res = self.gmres(b, tol, max_iter)
        us, q = self._split(u)
        V = np.concatenate([fb.velocity_nodes(um) for fb, um in zip(self.fibers, us)])
        T = np.concatenate([fb.tension_nodes(um) for fb, um in zip(self.fibers, us)])
        dt = self.fibers[0].dt if self.fibers else 0.0
        return StepResult(V=V, T=T, X_new=self.X + dt * V, q=q, u=u, iters=its, resid=res,
                          L_new=self.L + dt * self.Ldot)


def from_suspension(s, delta_over_L=0.01, lsb=False, Ldot=None) -> System:
    """Build the system from a workloads.Suspension (Ldot: per-fiber length
    rates, None = fixed lengths)."""
    return System(s.X, s.L, s.n_per_fiber, s.f_ext, s.mu, s.eps, s.E, s.dt, delta_over_L, lsb,
                  s.boundary, Ldot)
