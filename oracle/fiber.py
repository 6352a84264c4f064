"""Per-fiber discretisation of the implicit step (oracle; test infrastructure).

Unknowns per fiber (4N), following the representation of Eq. cheb-basis with
the velocity V = (X+ - X)/dt solved for directly (exact change of variables of
the backward-Euler update, Sec. 3.2):

    V_a(alpha) = sum_{j<N-4} sigma_{a,j} I^4 T_j(alpha) + sum_{k<4} p_{a,k} T_k(alpha)
    T(alpha)   = sum_{j<N-2} tau_j I^2 T_j(alpha) + q_0 + q_1 alpha

laid out as u_m = [c_x, c_y, c_z, d] with c_a = [sigma_a, p_a] (N each) and
d = [tau, q_0, q_1] (N).

Force at the nodes (Sec. 3.2, discrete force of set:time-stepping, with the
force balance of Eq. force-balance):
    f = -E D_s^4 X+ + D_s(T X_s) + f^E,   D_s = (2/L) D_alpha   (Sec. 3.1.3)
so with X+ = X + dt V and D_alpha^4 V = sigma:
    f = [-E dt g^4 sigma + g D_alpha(T X_s)] + [f^E - E g^4 X_aaaa],  g = 2/L.

Velocity expression at the nodes (Eq. main-sb-local):
    w = M f + K_delta[f] + ubar   (ubar: other fibers and the periphery)
    M f = (1/8 pi mu)[c (I + X_s X_s) + 2 (I - X_s X_s)] f,  c = -ln(eps^2 e)
    K_delta (Eq. sb-stokes-reg) by Clenshaw-Curtis quadrature on the nodes.

Rows (4N), rectangular collocation:
    velocity   (N-4 per component, first-kind points y):  -V(y) + [P_y w](y) = 0,
               with a growing or shrinking fiber (length rate Ldot, plus end
               at alpha = 1) the nodes sit at fixed alpha = 2 s / L - 1, so
               they move with the material velocity w plus the
               reparametrisation term R (Sec. 2.4, Eq. chain-rule, with the
               sign that advances the plus end):
               growth="explicit" (default; Eq. discrete-rhs, R at the current
               time):  -V(y) + [P_y w](y) + (y + 1)(Ldot / L) X_alpha(y) = 0;
               growth="implicit" (named variant, R at the new time):
                 -V(y) + [P_y w](y) + (y + 1) kappa X+_alpha(y) = 0,
                 kappa = Ldot / (L + dt Ldot), X+ = X + dt V
    free ends  (Eq. bc-free, on X+):  V''(+-1) + X''(+-1)/dt = 0,
                                      V'''(+-1) + X'''(+-1)/dt = 0
    tension    (N-2 first-kind points z):  X_s(z) . [D_z w](z) = 0
               (inextensibility X_s . V_s = 0 of Eq. main-inextensibility
                imposed on the velocity expression)
    tension ends: T(+1) = T(-1) = 0 (Eq. bc-free)

rows(u) = B u + Rw (S f_known + ubar) + const, where
    f_lin = F u,  S = M + K_delta (3N x 3N),  B = Rd + Rw S F.
"""
from __future__ import annotations

import math

import numpy as np

from . import cheb


class FiberOps:
    """Matrices that depend only on the number of points N (Sec. 3.1.3-3.2)."""

    def __init__(self, N: int):
        if N < 6:
            raise ValueError("need N >= 6 points per fiber")
        self.N = N
        a = cheb.nodes(N)
        self.alpha = a
        self.y = cheb.first_kind(N - 4)
        self.z = cheb.first_kind(N - 2)
        BV = cheb.basis_V(N)
        BT = cheb.basis_T(N)
        pm = np.array([1.0, -1.0])
        self.V_y = cheb.basis_matrix(BV, self.y)            # (N-4, N)
        self.V1_y = cheb.basis_matrix(BV, self.y, 1)        # (N-4, N): alpha-derivative at y
        self.V_nodes = cheb.basis_matrix(BV, a)             # (N, N)
        self.V0_pm = cheb.basis_matrix(BV, pm)              # (2, N): V at alpha = +1, -1
        self.V1_pm = cheb.basis_matrix(BV, pm, 1)           # (2, N)
        self.V2_pm = cheb.basis_matrix(BV, pm, 2)           # (2, N)
        self.V3_pm = cheb.basis_matrix(BV, pm, 3)           # (2, N)
        self.sig_nodes = cheb.basis_matrix(BV, a, 4)        # (N, N): sigma at nodes
        self.T_nodes = cheb.basis_matrix(BT, a)             # (N, N)
        self.T_pm = cheb.basis_matrix(BT, pm)               # (2, N)
        self.D1 = cheb.nodal_deriv_matrix(N, a, 1)          # (N, N)
        self.P_y = cheb.nodal_deriv_matrix(N, self.y, 0)    # (N-4, N)
        self.D_z = cheb.nodal_deriv_matrix(N, self.z, 1)    # (N-2, N)
        self.w = cheb.cc_weights(N)


_OPS = {}


def ops_for(N: int) -> FiberOps:
    """The FiberOps of N points, built once per N (Sec. 3.1.3-3.2)."""
    if N not in _OPS:
        _OPS[N] = FiberOps(N)
    return _OPS[N]


def stokeslet_tensor(r: np.ndarray, mu: float) -> np.ndarray:
    """G(r) = (I + rhat rhat)/(8 pi mu |r|) (Eq. oseen), r: [..., 3] -> [..., 3, 3]."""
    rn = np.linalg.norm(r, axis=-1)
    h = r / rn[..., None]
    return (np.eye(3) + h[..., :, None] * h[..., None, :]) / (8.0 * math.pi * mu * rn[..., None, None])


FREE, CLAMPED, HINGED = 0, 1, 2      # minus-end condition (Sec. 2.3)


class Fiber:
    """Explicit geometry and operator matrices of one fiber (Sec. 3.2: geometry
    frozen at the current step, forces implicit)."""

    def __init__(self, X: np.ndarray, L: float, f_ext: np.ndarray, mu: float, eps: float,
                 E: float, dt: float, delta: float, lsb: bool = False, Ldot: float = 0.0,
                 attach: int = FREE, growth: str = "explicit"):
        if growth not in ("explicit", "implicit"):
            raise ValueError("growth must be 'explicit' or 'implicit'")
        N = X.shape[0]
        op = ops_for(N)
        self.N, self.op, self.L = N, op, L
        self.mu, self.E, self.dt = mu, E, dt
        g = 2.0 / L
        # geometry: derivatives of the interpolant of X, in extended precision
        # (they amplify rounding by up to ~N^8, and the fiber block is
        # ill-conditioned, so double-precision evaluation would leave O(1e-8)
        # rounding noise in the step's velocities)
        Nld = cheb.nodes_ld(N)
        pm = np.array([1.0, -1.0], dtype=cheb.LD)
        self.t = g * cheb.interp_derivs_ext(X, Nld, 1)        # X_s at nodes
        self.tz = g * cheb.interp_derivs_ext(X, cheb.first_kind_ld(N - 2), 1)   # X_s at z
        X2 = cheb.interp_derivs_ext(X, pm, 2)                 # X_aa at alpha = +1, -1
        X3 = cheb.interp_derivs_ext(X, pm, 3)
        Xaaaa = cheb.interp_derivs_ext(X, Nld, 4)
        Xa_y = np.asarray(cheb.interp_derivs_ext(X, cheb.first_kind_ld(N - 4), 1), dtype=float) \
            if Ldot != 0.0 else None                            # X_alpha at the y points
        self.f_known = f_ext - E * g ** 4 * Xaaaa              # [N, 3]
        self.W = op.w * L / 2.0                                # source weights
        s = (op.alpha + 1.0) * L / 2.0
        c_log = -math.log(eps * eps * math.e)

        # F: u -> f_lin at nodes, component-major [a*N + k]
        F = np.zeros((3 * N, 4 * N))
        D1T = g * op.D1
        for a in range(3):
            F[a * N:(a + 1) * N, a * N:(a + 1) * N] = -E * dt * g ** 4 * op.sig_nodes
            F[a * N:(a + 1) * N, 3 * N:4 * N] = D1T @ (self.t[:, a:a + 1] * op.T_nodes)
        # S = M + K_delta on nodal forces; blocks S[a*N + k, b*N + j] = S_kj[a, b]
        I3 = np.eye(3)
        tt = self.t[:, :, None] * self.t[:, None, :]                    # [N, 3, 3]
        Mk = (c_log * (I3 + tt) + 2.0 * (I3 - tt)) / (8.0 * math.pi * mu)
        blocks = np.zeros((N, N, 3, 3))
        blocks[np.arange(N), np.arange(N)] = Mk
        if not lsb:
            off = ~np.eye(N, dtype=bool)
            r = X[:, None, :] - X[None, :, :]                                # r = X(s_k) - X(s_j)
            r[~off] = 1.0                                                    # placeholder, unused
            rn = np.linalg.norm(r, axis=-1)
            G = stokeslet_tensor(r, mu)                                      # [N, N, 3, 3]
            reg = rn / np.sqrt(rn * rn + delta * delta)                      # |r| / sqrt(|r|^2 + delta^2)
            blocks += np.where(off[:, :, None, None], (reg * self.W[None, :])[:, :, None, None] * G, 0.0)
            ds = s[:, None] - s[None, :]
            sub = np.where(off, self.W[None, :] / (8.0 * math.pi * mu * np.sqrt(ds * ds + delta * delta)), 0.0)
            blocks[np.arange(N), np.arange(N)] -= sub.sum(axis=1)[:, None, None] * (I3 + tt)
        S = blocks.transpose(2, 0, 3, 1).reshape(3 * N, 3 * N)
        # Rw: nodal w -> rows; Rd: direct rows; const
        Rw = np.zeros((4 * N, 3 * N))
        Rd = np.zeros((4 * N, 4 * N))
        const = np.zeros(4 * N)
        for a in range(3):
            r0 = a * N
            Rw[r0:r0 + N - 4, a * N:(a + 1) * N] = op.P_y
            Rd[r0:r0 + N - 4, a * N:(a + 1) * N] = -op.V_y
            Rd[r0 + N - 4:r0 + N - 2, a * N:(a + 1) * N] = op.V2_pm
            Rd[r0 + N - 2:r0 + N, a * N:(a + 1) * N] = op.V3_pm
            const[r0 + N - 4:r0 + N - 2] = X2[:, a] / dt
            const[r0 + N - 2:r0 + N] = X3[:, a] / dt
            if Ldot != 0.0 and growth == "explicit":
                # growth (Sec. 2.4, Eq. chain-rule; Sec. 3.2, Eq. discrete-rhs):
                # at fixed alpha the nodes move with the material velocity plus
                # (alpha + 1)(Ldot / L) X_alpha, taken at the current time:
                # -V + w + (y + 1)(Ldot / L) X_alpha(y) = 0
                const[r0:r0 + N - 4] = (op.y + 1.0) * (Ldot / L) * Xa_y[:, a]
            elif Ldot != 0.0:
                # the same term at the new time (length L + dt Ldot, positions
                # X + dt V): -V + w + (y + 1) kappa (X_alpha + dt V_alpha)(y) = 0
                kappa = Ldot / (L + dt * Ldot)
                const[r0:r0 + N - 4] = (op.y + 1.0) * kappa * Xa_y[:, a]
                Rd[r0:r0 + N - 4, a * N:(a + 1) * N] += dt * kappa * (op.y + 1.0)[:, None] * op.V1_y
            Rw[3 * N:4 * N - 2, a * N:(a + 1) * N] = self.tz[:, a:a + 1] * op.D_z
        Rd[4 * N - 2:4 * N, 3 * N:4 * N] = op.T_pm
        # minus end (alpha = -1, s = 0) attached to a rigid body (Sec. 2.3,
        # Eqs. BC2-1, BC2-2, BC2-T); the body's U, Omega enter through
        # rigid_rows.  The V_aaa(-1) rows become the position condition
        # V(-1) = U + Omega x (X(-1) - X^P); clamped: the V_aa(-1) rows become
        # g V_a(-1) = Omega x X_s(-1) (hinged keeps X+_aa(-1) = 0, torque
        # free); the T(-1) = 0 row becomes the tangential projection of the
        # velocity expression at the end, X_s . w(-1) = X_s . (U + Omega x r).
        self.attach = attach
        self.X_end = np.asarray(X[N - 1], float)
        self.X2m = np.asarray(X2[1], dtype=float)          # X_aa(-1)
        self.X3m = np.asarray(X3[1], dtype=float)          # X_aaa(-1)
        if attach != FREE:
            for a in range(3):
                r0 = a * N
                Rd[r0 + N - 1, :] = 0.0
                Rd[r0 + N - 1, a * N:(a + 1) * N] = op.V0_pm[1]
                const[r0 + N - 1] = 0.0
                if attach == CLAMPED:
                    Rd[r0 + N - 3, :] = 0.0
                    Rd[r0 + N - 3, a * N:(a + 1) * N] = g * op.V1_pm[1]
                    const[r0 + N - 3] = 0.0
                Rw[4 * N - 1, a * N + N - 1] = self.t[N - 1, a]
            Rd[4 * N - 1, :] = 0.0
            const[4 * N - 1] = 0.0
        self.F, self.S, self.Rw, self.Rd, self.const = F, S, Rw, Rd, const
        self.B = Rd + Rw @ S @ F

    # ------------------------------------------------------------------ helpers
    @staticmethod
    def to_cm(v: np.ndarray) -> np.ndarray:
        """[N, 3] -> component-major [3N]."""
        return v.T.reshape(-1)

    @staticmethod
    def from_cm(v: np.ndarray) -> np.ndarray:
        return v.reshape(3, -1).T

    def f_lin(self, u: np.ndarray) -> np.ndarray:
        """Nodal force of the unknowns u, -E dt D_s^4 V + D_s(T X_s) (Eq.
        main-elastic-force, Sec. 3.2)."""
        return self.from_cm(self.F @ u)

    def rows_from_ubar(self, ubar: np.ndarray) -> np.ndarray:
        """Rw applied to a nodal velocity field [N, 3] (Sec. 3.2, Eq. sche-linear-eq)."""
        return self.Rw @ self.to_cm(ubar)

    def rows_known(self) -> np.ndarray:
        """Constant rows from the known force and the free-end data (Sec. 3.2, Eq. bc-free)."""
        return self.Rw @ (self.S @ self.to_cm(self.f_known)) + self.const

    def velocity_nodes(self, u: np.ndarray) -> np.ndarray:
        """V at the nodes from the unknowns u (Eq. cheb-basis)."""
        N = self.N
        return np.stack([self.op.V_nodes @ u[a * N:(a + 1) * N] for a in range(3)], axis=1)

    def rigid_rows(self, U: np.ndarray, Om: np.ndarray, Xp: np.ndarray) -> np.ndarray:
        """Terms of the attached-end rows in the body's U, Omega (zero for a
        free fiber) (Eqs. BC2-1, BC2-2, BC2-T)."""
        N = self.N
        out = np.zeros(4 * N)
        if self.attach == FREE:
            return out
        te = np.asarray(self.t[N - 1], float)
        v = U + np.cross(Om, self.X_end - Xp)
        for a in range(3):
            out[a * N + N - 1] = -v[a]
        if self.attach == CLAMPED:
            w = np.cross(Om, te)
            for a in range(3):
                out[a * N + N - 3] = -w[a]
        out[4 * N - 1] = -te @ v
        return out

    def end_load(self, u, Xp: np.ndarray, known: bool):
        """(force, torque about Xp) that the attached end exerts on the body,
        from the rod's force and moment balance: F^I(0) = -E X+_sss + T X_s and
        (X(0) - X^P) x F^I(0) + E X_s x X+_ss at s = 0 (Sec. 2.3, Eqs. f-ext,
        t-ext), X+ = X + dt V.  known: the part without unknowns (u ignored);
        else the part linear in u."""
        N, op, g, dt, E = self.N, self.op, 2.0 / self.L, self.dt, self.E
        te = np.asarray(self.t[N - 1], float)
        if known:
            X3, X2, Tm = self.X3m, self.X2m, 0.0
        else:
            X3 = dt * np.array([op.V3_pm[1] @ u[a * N:(a + 1) * N] for a in range(3)])
            X2 = dt * np.array([op.V2_pm[1] @ u[a * N:(a + 1) * N] for a in range(3)])
            Tm = op.T_pm[1] @ u[3 * N:4 * N]
        F = -E * g ** 3 * X3 + Tm * te
        L = np.cross(self.X_end - Xp, F) + E * g ** 2 * np.cross(te, X2)
        return F, L

    def tension_nodes(self, u: np.ndarray) -> np.ndarray:
        """T at the nodes from the unknowns u (Eq. cheb-basis)."""
        N = self.N
        return self.op.T_nodes @ u[3 * N:4 * N]
