"""Global linear system of one implicit step and its GMRES solve (oracle;
test infrastructure -- only the tests, the smoke check and the benchmark's
CPU-baseline legs use it).

Sec. 3.2-3.3: the linearised backward-Euler step gives A u = b
(Eq. sche-linear-eq) with fiber blocks (4N_m unknowns each) and, under
confinement, the periphery double-layer density q0 (3 unknowns per surface
node).  Coupling between bodies is the complementary velocity
(Eqs. complementary-uc, complementary-uf):

* fiber m nodes:  ubar = sum over other fibers of the Stokeslet line integral
  (Clenshaw-Curtis sources W f) + T_Gamma0[q0] (Eq. cortex-vel);
* surface rows:   -q0/2 + T[q0] + N[q0] + (fiber Stokeslets at the nodes) = 0
  (Eq. main-cortex-density), singular part by subtraction (Sec. 3.1.2).

With a rigid body (Sec. 2.2, Eqs. main-nsb-second-kind, main-nsb-rgbt,
main-nsb-rgbr) the unknowns add its surface density q1 (3 per node) and its
translational and angular velocities U, Omega; fibers may be clamped or
hinged to it at their minus ends (Sec. 2.3), and the force and torque they
exert on it (Eqs. f-ext, t-ext) drive its Stokeslet and rotlet:

* body rows:   -q1/2 + T_pv[q1] + G(y - X^P) F + R(y - X^P) L - U
               - Omega x (y - X^P) + (fiber Stokeslets, periphery double
               layer at y) = 0;
* constraints: mean of q1 over the surface - U = 0,
               mean of (y - X^P) x q1 - Omega = 0;
* every other target feels T[q1] + G F + R L (Eq. main-nsb-vel);
* F = F^E + sum of the attached ends' forces, L likewise (Fiber.end_load).

Unknown vector: fibers (4N_m each), periphery q0, body q1, then U, Omega.

Preconditioner (Eq. prec): exact fiber self-blocks B_m (LU with partial
pivoting) and the scalar diagonal of the surface and body self-blocks
(-1 on the U, Omega rows); left preconditioned GMRES (Saad) with x0 = 0,
modified Gram-Schmidt and Givens rotations, stopping when
||P^-1(b - A u)|| <= tol ||P^-1 b||.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg

from . import kernels
from .fiber import FREE, Fiber


def point_flow(x: np.ndarray, centre: np.ndarray, F: np.ndarray, Lt: np.ndarray, mu: float) -> np.ndarray:
    """G(x - c) F + R(x - c) L at the points x (Eqs. oseen, rotlet):
    G = (I + rhat rhat) / (8 pi mu |r|), R L = L x rhat / (8 pi mu |r|^2)."""
    r = np.asarray(x, float) - centre[None, :]
    rn = np.linalg.norm(r, axis=1)
    h = r / rn[:, None]
    c = 1.0 / (8.0 * np.pi * mu)
    return c * ((F[None, :] + h * (h @ F)[:, None]) / rn[:, None]
                + np.cross(Lt[None, :], h) / (rn * rn)[:, None])


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
    U: Optional[np.ndarray] = None       # [3] body translational velocity
    Omega: Optional[np.ndarray] = None   # [3] body angular velocity
    centre_new: Optional[np.ndarray] = None   # [3] X^P + dt U
    q1: Optional[np.ndarray] = None      # [n_b, 3] body density


class System:
    """The coupled implicit system of all fibers, the periphery and the body
    (Eqs. sche-linear-eq, complementary-uf, complementary-uc)."""

    def __init__(self, X, L, n_per_fiber, f_ext, mu=1.0, eps=1e-3, E=1.0, dt=1e-3,
                 delta_over_L=0.01, lsb=False, boundary=None, Ldot=None, body=None, attach=None,
                 growth="explicit"):
        self.mu = mu
        self.dt = dt
        self.n_per = np.asarray(n_per_fiber, dtype=np.int64)
        self.ptr = np.concatenate([[0], np.cumsum(self.n_per)])
        self.X = np.asarray(X, float)
        self.fibers: List[Fiber] = []
        for m in range(len(self.n_per)):
            a, b = self.ptr[m], self.ptr[m + 1]
            self.fibers.append(Fiber(self.X[a:b], float(L[m]), np.asarray(f_ext[a:b], float), mu,
                                     eps, E, dt, delta_over_L * float(L[m]), lsb,
                                     0.0 if Ldot is None else float(Ldot[m]),
                                     FREE if attach is None else int(attach[m]), growth))
        self.L = np.asarray(L, float)
        self.Ldot = np.zeros(len(self.n_per)) if Ldot is None else np.asarray(Ldot, float)
        self.uptr = np.concatenate([[0], np.cumsum(4 * self.n_per)])
        self.fid = np.repeat(np.arange(len(self.n_per), dtype=np.int32), self.n_per)
        self.Wall = np.concatenate([f.W for f in self.fibers]) if self.fibers else np.zeros(0)
        self.boundary = boundary
        self.n_s = 0 if boundary is None else boundary.nodes.shape[0]
        self.body = body
        self.n_b = 0 if body is None else body.nodes.shape[0]
        if attach is not None and body is None and np.any(np.asarray(attach) != FREE):
            raise ValueError("attached fibers need a body")
        self.q1_off = int(self.uptr[-1]) + 3 * self.n_s
        self.rb_off = self.q1_off + 3 * self.n_b
        self.n_unknowns = self.rb_off + (6 if body is not None else 0)
        self.lu = [scipy.linalg.lu_factor(f.B) for f in self.fibers]
        if boundary is not None:
            self.sdiag = kernels.surface_diag(boundary.nodes, boundary.normals, boundary.weights).reshape(-1)
        if body is not None:
            self.Xp = np.asarray(body.centre, float)
            self.area = float(np.sum(body.weights))
            self.bdiag = kernels.body_diag(body.nodes, body.normals, body.weights).reshape(-1)

    # --------------------------------------------------------------- pieces
    def _split(self, u):
        us = [u[self.uptr[m]:self.uptr[m + 1]] for m in range(len(self.fibers))]
        q = u[self.uptr[-1]:self.q1_off].reshape(-1, 3) if self.n_s else None
        return us, q

    def _split_body(self, u):
        """(q1 [n_b, 3], U, Omega) of the body part of u."""
        return (u[self.q1_off:self.rb_off].reshape(-1, 3), u[self.rb_off:self.rb_off + 3],
                u[self.rb_off + 3:self.rb_off + 6])

    def _body_load(self, us, known: bool):
        """(F, L) of the body: the attached ends' forces and torques (known
        part plus the external load, or the part linear in the unknowns)."""
        bd = self.body
        F = np.array(bd.force, float) if known else np.zeros(3)
        L = np.array(bd.torque, float) if known else np.zeros(3)
        for m, fb in enumerate(self.fibers):
            if fb.attach != FREE:
                dF, dL = fb.end_load(None if known else us[m], self.Xp, known)
                F, L = F + dF, L + dL
        return F, L

    def _fields(self, f_nodes, q0, q1, F, Lt):
        """Complementary velocities for nodal fiber forces f_nodes [N_tot,3],
        periphery density q0, body density q1 and body load (F, Lt): (at the
        fiber nodes, at the periphery nodes or None, at the body nodes or
        None).  Each surface's own double layer is left to its rows; the
        body's own Stokeslet and rotlet are included at its nodes."""
        wf = f_nodes * self.Wall[:, None]
        ub = kernels.stokeslet(self.X, self.X, wf, self.mu, self.fid, self.fid)
        us = ubody = None
        if self.n_s:
            b = self.boundary
            if q0 is not None:
                ub = ub + kernels.stresslet(self.X, b.nodes, b.normals, b.weights, q0)
            us = kernels.stokeslet(b.nodes, self.X, wf, self.mu)
        if self.body is not None:
            bd = self.body
            ubody = kernels.stokeslet(bd.nodes, self.X, wf, self.mu) + point_flow(bd.nodes, self.Xp, F, Lt,
                                                                                 self.mu)
            ub = ub + point_flow(self.X, self.Xp, F, Lt, self.mu)
            if q1 is not None:
                ub = ub + kernels.stresslet(self.X, bd.nodes, bd.normals, bd.weights, q1)
            if self.n_s:
                b = self.boundary
                us = us + point_flow(b.nodes, self.Xp, F, Lt, self.mu)
                if q1 is not None:
                    us = us + kernels.stresslet(b.nodes, bd.nodes, bd.normals, bd.weights, q1)
                if q0 is not None:
                    ubody = ubody + kernels.stresslet(bd.nodes, b.nodes, b.normals, b.weights, q0)
        return ub, us, ubody

    def _couplings(self, f_nodes: np.ndarray, q):
        """Complementary velocities of a body-free system for nodal fiber
        forces f_nodes [N_tot,3] and density q: (ubar at fiber nodes [N_tot,3],
        fiber Stokeslets at the surface nodes [n_s,3] or None)."""
        ub, us, _ = self._fields(f_nodes, q, None, None, None)
        return ub, us

    def matvec(self, u: np.ndarray) -> np.ndarray:
        """A u: each fiber's rows with the far field of the others, and the
        surface rows (Eq. sche-linear-eq)."""
        us, q = self._split(u)
        f = np.concatenate([fb.f_lin(um) for fb, um in zip(self.fibers, us)]) if self.fibers \
            else np.zeros((0, 3))
        if self.body is not None:
            q1, U, Om = self._split_body(u)
            F, Lt = self._body_load(us, known=False)
        else:
            q1 = F = Lt = None
        ub, usurf, ubody = self._fields(f, q, q1, F, Lt)
        out = np.zeros_like(u)
        for m, fb in enumerate(self.fibers):
            a, b = self.ptr[m], self.ptr[m + 1]
            r = fb.B @ us[m] + fb.rows_from_ubar(ub[a:b])
            if fb.attach != FREE:
                r = r + fb.rigid_rows(U, Om, self.Xp)
            out[self.uptr[m]:self.uptr[m + 1]] = r
        if self.n_s:
            bd = self.boundary
            out[self.uptr[-1]:self.q1_off] = (kernels.surface_self(bd.nodes, bd.normals, bd.weights, q)
                                              + usurf).reshape(-1)
        if self.body is not None:
            bd = self.body
            rel = bd.nodes - self.Xp[None, :]
            rows = kernels.body_self(bd.nodes, bd.normals, bd.weights, q1) + ubody - U[None, :] \
                - np.cross(Om[None, :], rel)
            out[self.q1_off:self.rb_off] = rows.reshape(-1)
            w = bd.weights[:, None]
            out[self.rb_off:self.rb_off + 3] = np.sum(w * q1, axis=0) / self.area - U
            out[self.rb_off + 3:self.rb_off + 6] = np.sum(w * np.cross(rel, q1), axis=0) / self.area - Om
        return out

    def rhs(self) -> np.ndarray:
        """Right-hand side b from the known force, the free-end data and the
        body's load (Sec. 3.2, Eq. sche-linear-eq)."""
        f = np.concatenate([fb.f_known for fb in self.fibers]) if self.fibers else np.zeros((0, 3))
        F = Lt = None
        if self.body is not None:
            F, Lt = self._body_load(None, known=True)
        ub, usurf, ubody = self._fields(f, None, None, F, Lt)
        b = np.zeros(self.n_unknowns)
        for m, fb in enumerate(self.fibers):
            a, c = self.ptr[m], self.ptr[m + 1]
            b[self.uptr[m]:self.uptr[m + 1]] = -(fb.rows_known() + fb.rows_from_ubar(ub[a:c]))
        if self.n_s:
            b[self.uptr[-1]:self.q1_off] = -usurf.reshape(-1)
        if self.body is not None:
            b[self.q1_off:self.rb_off] = -ubody.reshape(-1)
        return b

    def precond(self, v: np.ndarray) -> np.ndarray:
        """P^-1 v: per-fiber block solves and Jacobi on the surface unknowns
        (Eq. prec)."""
        out = np.empty_like(v)
        for m in range(len(self.fibers)):
            sl = slice(self.uptr[m], self.uptr[m + 1])
            out[sl] = scipy.linalg.lu_solve(self.lu[m], v[sl])
        if self.n_s:
            out[self.uptr[-1]:self.q1_off] = v[self.uptr[-1]:self.q1_off] / self.sdiag
        if self.body is not None:
            out[self.q1_off:self.rb_off] = v[self.q1_off:self.rb_off] / self.bdiag
            out[self.rb_off:] = -v[self.rb_off:]
        return out

    # ---------------------------------------------------------------- GMRES
    def gmres(self, b: np.ndarray, tol: float, max_iter: int = 300, matvec=None):
        """GMRES on the preconditioned system (Sec. 3.3)."""
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
        """One implicit step: assemble, solve, read V and T (Sec. 3.2-3.3)."""
        b = self.rhs()
        u, its, res = self.gmres(b, tol, max_iter)
        return self.result(u, its, res)

    def exact_step(self) -> StepResult:
        """The step with the exact solution of the assembled FP64 system
        (oracle.exact: dense assembly, LU and refinement with double-double
        residuals) instead of GMRES; small systems only."""
        from . import exact
        A, b = exact.assemble(self)
        u, _ = exact.solve_refined(A, b)
        return self.result(u, 0, 0.0)

    def result(self, u: np.ndarray, its: int = 0, res: float = 0.0) -> StepResult:
        """V, T, X+ (and the body's motion) from the unknowns u."""
        us, q = self._split(u)
        V = np.concatenate([fb.velocity_nodes(um) for fb, um in zip(self.fibers, us)]) \
            if self.fibers else np.zeros((0, 3))
        T = np.concatenate([fb.tension_nodes(um) for fb, um in zip(self.fibers, us)]) \
            if self.fibers else np.zeros(0)
        dt = self.dt
        res_ = StepResult(V=V, T=T, X_new=self.X + dt * V, q=q, u=u, iters=its, resid=res,
                          L_new=self.L + dt * self.Ldot)
        if self.body is not None:
            q1, U, Om = self._split_body(u)
            res_.U, res_.Omega, res_.q1 = U.copy(), Om.copy(), q1.copy()
            res_.centre_new = self.Xp + dt * U
        return res_


def from_suspension(s, delta_over_L=0.01, lsb=False, Ldot=None, growth="explicit") -> System:
    """Build the system from a workloads.Suspension (Ldot: per-fiber length
    rates, None = fixed lengths; growth: "explicit" = the growth term at the
    current time as in Eq. discrete-rhs, "implicit" = at the new time; a
    rigid body and the fibers' minus-end conditions when the suspension has
    them)."""
    return System(s.X, s.L, s.n_per_fiber, s.f_ext, s.mu, s.eps, s.E, s.dt, delta_over_L, lsb,
                  s.boundary, Ldot, getattr(s, "body", None), getattr(s, "attach", None), growth)
