"""Seeded synthetic inputs for fiber-suspension steps.

This module is shared by the CPU oracle, the tests and the benchmark.  It
holds no arithmetic of the numerical method (no Chebyshev transforms, no
quadrature rules of the method, no kernels): it only places fibers in space,
draws external forces and lays out the spherical boundary's quadrature nodes.
The paper computes the surface's Jacobian and normals in a preprocessing step
outside the solver (Sec. 3.1.1, Eq. patch-gl-quad), so they are inputs here too.

Every generator takes a seed and returns plain numpy float64/int32 arrays.

Workloads (shapes follow the paper's experiments: confined arrays of 32-2048
fibers with 31 points (Table 2), a sedimenting cloud of 1024 free fibers
(Sec. 4.3)):

* ``free_space``: M fibers, N Chebyshev points each, centres uniform in a
  cube, orientations uniform on the sphere, lengths uniform in [1, 3],
  optional smooth initial curvature, i.i.d. N(0,1) external force per node.
* ``confined``: the same inside a sphere of radius R, centres uniform in a
  ball of radius R_c, with the sphere's 4x4 Gauss-Legendre patch nodes.
* ``batched``: independent free-space systems with log-uniform fiber counts
  and mixed points per fiber.
* ``aster``: a rigid sphere with fibers attached at their minus ends, pointing
  outwards, inside a spherical periphery of six body radii (Table 2), driven
  by a force on the sphere.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Boundary:
    """Quadrature description of a sphere of radius R centred at the origin."""
    R: float
    nodes: np.ndarray     # [n, 3]
    normals: np.ndarray   # [n, 3] outward unit normals
    weights: np.ndarray   # [n]   Gauss-Legendre weight x surface Jacobian


@dataclasses.dataclass
class RigidBody:
    """A rigid sphere: centre, radius, quadrature nodes on its surface
    (absolute positions), outward normals, weights, and the external force
    and torque applied to it."""
    centre: np.ndarray    # [3]
    radius: float
    nodes: np.ndarray     # [n, 3]
    normals: np.ndarray   # [n, 3]
    weights: np.ndarray   # [n]
    force: np.ndarray     # [3]
    torque: np.ndarray    # [3]


# minus-end conditions of a fiber (codes shared with the library's interface)
FREE, CLAMPED, HINGED = 0, 1, 2

# Microtubule parameters of the paper's simulation table (Sec. 4, taken there
# from Kimura and Onami 2005), in um, s and pN: plus-end growth and shrinkage
# speeds (um/s), catastrophe and rescue rates (1/s), bending modulus
# (pN um^2) and cytoplasm viscosity (pN s / um^2 = Pa s).
MICROTUBULE = {"v_grow": 0.12, "v_shrink": 0.288, "f_cat": 0.014, "f_res": 0.014, "E": 10.0, "mu": 1.0}


@dataclasses.dataclass
class Suspension:
    """One fiber suspension: all arrays fiber-major, nodes of fiber m at
    rows ptr[m]:ptr[m+1]."""
    n_per_fiber: np.ndarray   # [M] int32, points per fiber
    X: np.ndarray             # [N_tot, 3] node positions
    L: np.ndarray             # [M] fiber lengths
    f_ext: np.ndarray         # [N_tot, 3] external force per unit length
    mu: float = 1.0
    eps: float = 1e-3
    E: float = 1.0
    dt: float = 1e-3
    boundary: Optional[Boundary] = None
    body: Optional[RigidBody] = None
    attach: Optional[np.ndarray] = None   # [M] int32 minus-end condition (FREE/CLAMPED/HINGED)

    @property
    def ptr(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_per_fiber)]).astype(np.int64)

    @property
    def n_fibers(self) -> int:
        return int(self.n_per_fiber.shape[0])

    @property
    def n_points(self) -> int:
        return int(self.X.shape[0])

    def fiber_id(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_fibers, dtype=np.int32), self.n_per_fiber)


def collocation_alpha(n: int) -> np.ndarray:
    """Positions of the n collocation points in the fiber parameter,
    alpha_k = cos(k pi / (n-1)), k = 0..n-1 (Sec. 3.1.3); k = 0 is alpha = +1."""
    return np.cos(np.pi * np.arange(n) / (n - 1))


def _unit_vectors(rng: np.random.Generator, m: int) -> np.ndarray:
    d = rng.normal(size=(m, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _curved_fiber(rng, centre, direction, length, alpha, amp, n_modes=4, n_gl=96):
    """Centreline whose unit tangent is normalise(t0 + sum_k g_k cos(k acos a)),
    g_k ~ N(0, amp^2) per component, integrated from the midpoint with
    Gauss-Legendre quadrature so that |dX/ds| = 1 and the arclength is L."""
    g = rng.normal(scale=amp, size=(n_modes, 3))
    xg, wg = np.polynomial.legendre.leggauss(n_gl)

    def tangent(a):
        a = np.clip(a, -1.0, 1.0)
        th = np.arccos(a)
        t = direction[None, :] + sum(np.cos((k + 1) * th)[:, None] * g[k][None, :]
                                     for k in range(n_modes))
        return t / np.linalg.norm(t, axis=1, keepdims=True)

    pts = np.empty((alpha.shape[0], 3))
    for i, a in enumerate(alpha):
        # integrate tangent over [0, a] in the parameter; ds = (L/2) d alpha
        half = 0.5 * a
        nodes = half * (xg + 1.0)
        pts[i] = centre + (length / 2.0) * half * (wg[:, None] * tangent(nodes)).sum(0)
    return pts


def free_space(M: int, N, side: float, seed: int = 0, curved_amp: float = 0.0,
               L_range=(1.0, 3.0), mu=1.0, eps=1e-3, E=1.0, dt=1e-3,
               centre_offset=None, min_gap: float = 0.0) -> Suspension:
    """M fibers in the cube [0, side]^3 (N may be an int or a per-fiber array).
    min_gap > 0: straight chords at least min_gap x (mean length) apart
    (random sequential addition)."""
    rng = np.random.default_rng(seed)
    n_per = np.full(M, N, dtype=np.int32) if np.isscalar(N) else np.asarray(N, np.int32)
    if min_gap > 0.0:
        L = rng.uniform(L_range[0], L_range[1], size=M)
        centres, dirs = _place_separated(rng, M, L, lambda: rng.uniform(0.0, side, size=3), min_gap)
    else:
        centres = rng.uniform(0.0, side, size=(M, 3))
        dirs = _unit_vectors(rng, M)
        L = rng.uniform(L_range[0], L_range[1], size=M)
    if centre_offset is not None:
        centres = centres + np.asarray(centre_offset)[None, :]
    return _assemble(rng, n_per, centres, dirs, L, curved_amp, mu, eps, E, dt, None)


def _assemble(rng, n_per, centres, dirs, L, curved_amp, mu, eps, E, dt, boundary):
    Xs = []
    for m in range(n_per.shape[0]):
        a = collocation_alpha(int(n_per[m]))
        if curved_amp > 0.0:
            Xs.append(_curved_fiber(rng, centres[m], dirs[m], L[m], a, curved_amp))
        else:
            Xs.append(centres[m][None, :] + (a[:, None] * L[m] / 2.0) * dirs[m][None, :])
    X = np.concatenate(Xs, axis=0)
    f_ext = rng.normal(size=X.shape)
    return Suspension(n_per_fiber=n_per, X=X, L=L, f_ext=f_ext, mu=mu, eps=eps, E=E,
                      dt=dt, boundary=boundary)


def sphere_quadrature(R: float, n_theta: int, n_phi: int, q: int = 4) -> Boundary:
    """Uniform (theta, phi) patches on a sphere with a q x q Gauss-Legendre grid
    on each (Sec. 3.1.1, Eq. patch-gl-quad): weight = nu_i nu_j J, with
    J = R^2 sin(theta) times the patch's parameter-box half-widths."""
    x, w = np.polynomial.legendre.leggauss(q)
    dth = math.pi / n_theta
    dph = 2.0 * math.pi / n_phi
    nodes, normals, weights = [], [], []
    for it in range(n_theta):
        th = (it + 0.5 + 0.5 * x) * dth
        for ip in range(n_phi):
            ph = (ip + 0.5 + 0.5 * x) * dph
            TH, PH = np.meshgrid(th, ph, indexing="ij")
            WW = np.outer(w, w) * (0.5 * dth) * (0.5 * dph) * R * R * np.sin(TH)
            n = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1)
            nodes.append((R * n).reshape(-1, 3))
            normals.append(n.reshape(-1, 3))
            weights.append(WW.reshape(-1))
    return Boundary(R=R, nodes=np.concatenate(nodes), normals=np.concatenate(normals),
                    weights=np.concatenate(weights))


def confined(M: int, N: int, R: float = 20.0, R_centres: float = 18.0,
             n_theta: int = 16, n_phi: int = 48, seed: int = 0, L_range=(1.0, 3.0),
             mu=1.0, eps=1e-3, E=1.0, dt=1e-3) -> Suspension:
    """M straight fibers with centres uniform in a ball of radius R_centres,
    inside a no-slip sphere of radius R (16 x 48 patches x 16 = 12,288 nodes
    by default)."""
    rng = np.random.default_rng(seed)
    n_per = np.full(M, N, dtype=np.int32)
    d = _unit_vectors(rng, M)
    rad = R_centres * rng.uniform(0.0, 1.0, size=M) ** (1.0 / 3.0)
    centres = d * rad[:, None]
    dirs = _unit_vectors(rng, M)
    L = rng.uniform(L_range[0], L_range[1], size=M)
    b = sphere_quadrature(R, n_theta, n_phi)
    return _assemble(rng, n_per, centres, dirs, L, 0.0, mu, eps, E, dt, b)


def batched(n_systems: int, seed: int = 0, fibers_range=(8, 512),
            points_choices=(16, 32, 64), density_ref=(16, 10.0)) -> List[Suspension]:
    """Independent free-space systems: fiber count log-uniform in fibers_range,
    one points-per-fiber value per system, cube side scaled to keep the fiber
    density of `density_ref` = (fibers, side)."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi = math.log(fibers_range[0]), math.log(fibers_range[1])
    for s in range(n_systems):
        M = int(round(math.exp(rng.uniform(lo, hi))))
        N = int(rng.choice(points_choices))
        side = density_ref[1] * (M / density_ref[0]) ** (1.0 / 3.0)
        out.append(free_space(M, N, side, seed=int(rng.integers(1 << 31))))
    return out


def _segment_distances(p, u, h, P, U, H):
    """Closest distances between the segment p +- h u and the segments
    P[k] +- H[k] U[k] (u, U unit vectors)."""
    w = p[None, :] - P
    b = U @ u
    d = w @ u
    e = np.einsum("ij,ij->i", U, w)
    den = 1.0 - b * b
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(den > 1e-12, (b * e - d) / den, 0.0)
    s = np.clip(s, -h, h)
    t = np.clip(b * s + e, -H, H)
    s = np.clip(b * t - d, -h, h)
    diff = w + s[:, None] * u[None, :] - t[:, None] * U
    return np.linalg.norm(diff, axis=1)


def _place_separated(rng, M, L, sample_centre, min_gap):
    """Random sequential addition of M straight segments of lengths L with
    centres from sample_centre() and uniform orientations, each at least
    min_gap x (mean of the two lengths) from all earlier ones."""
    centres = np.zeros((M, 3))
    dirs = np.zeros((M, 3))
    k = tries = 0
    while k < M:
        tries += 1
        if tries > 1000 * M:
            raise RuntimeError("could not place the fibers with this gap")
        c = sample_centre()
        u = _unit_vectors(rng, 1)[0]
        if k and np.any(_segment_distances(c, u, L[k] / 2.0, centres[:k], dirs[:k], L[:k] / 2.0)
                        < min_gap * 0.5 * (L[k] + L[:k])):
            continue
        centres[k], dirs[k] = c, u
        k += 1
    return centres, dirs


def sedimenting_cloud(L_over_R: float, M: int = 1024, N: int = 16, seed: int = 0, R0: float = 1.0,
                      f0: float = 1.0, dt: float = 1e-4, min_gap: float = 0.1) -> Suspension:
    """The sedimenting cloud of Sec. 4.3: M straight free fibers of equal
    length L = L_over_R R0, centres uniform in a ball of radius R0,
    orientations uniform on S^2, gravity f^E = -f0 z (per unit length),
    eps = 0.01, E = 3.2e-3 f0 R0^3, mu = 1.  Fibers are placed by random
    sequential addition with centrelines at least min_gap L apart (about one
    node spacing at 16 points): the direct quadrature of the far field is
    not accurate for closer fibers and such pairs go unstable (near-singular
    quadrature is not used here).  The paper gives no time step; dt = 1e-4
    (the cloud moves ~0.003 R0 per step)."""
    rng = np.random.default_rng(seed)
    n_per = np.full(M, N, dtype=np.int32)
    L = np.full(M, L_over_R * R0)
    centres, dirs = _place_separated(rng, M, L, lambda: _unit_vectors(rng, 1)[0] * R0 * rng.uniform() ** (1.0 / 3.0),
                                     min_gap)
    s = _assemble(rng, n_per, centres, dirs, L, 0.0, 1.0, 0.01, 3.2e-3 * f0 * R0 ** 3, dt, None)
    s.f_ext = np.tile([0.0, 0.0, -f0], (s.n_points, 1))
    return s


def cloud_velocity_scale(s: Suspension, R0: float = 1.0) -> float:
    """V_c = N_F F / (5 pi mu R0), F = |f^E| L the weight of one fiber: the
    settling speed of a spherical drop of the suspension's viscosity
    (Hadamard-Rybczynski with equal viscosities), Sec. 4.3."""
    F = float(np.abs(s.f_ext[0, 2])) * float(s.L[0])
    return s.n_fibers * F / (5.0 * math.pi * s.mu * R0)


# Named workloads (sizes of the paper-shaped benchmark cases).
def cfg_small_fp64(seed: int = 0) -> Suspension:
    """16 straight fibers x 32 points in [0,10]^3 (512 points)."""
    return free_space(16, 32, 10.0, seed=seed)


def cfg_cloud_mixed(seed: int = 0) -> Suspension:
    """1,024 curved fibers x 64 points in [0,40]^3 (65,536 points)."""
    return free_space(1024, 64, 40.0, seed=seed, curved_amp=0.05)


def cfg_confined(seed: int = 0) -> Suspension:
    """2,000 fibers x 32 points inside a radius-20 sphere with 12,288 nodes."""
    return confined(2000, 32, seed=seed)


def cfg_large_matvec(seed: int = 0) -> Suspension:
    """8,192 fibers x 128 points in [0,80]^3 (1,048,576 points)."""
    return free_space(8192, 128, 80.0, seed=seed)


def sphere_body(centre, radius: float, n_theta: int, n_phi: int, force=(0.0, 0.0, 0.0),
                torque=(0.0, 0.0, 0.0), q: int = 4) -> RigidBody:
    """A rigid sphere with the periphery's patch quadrature (q x q
    Gauss-Legendre nodes on n_theta x n_phi (theta, phi) patches)."""
    c = np.asarray(centre, dtype=np.float64)
    b = sphere_quadrature(radius, n_theta, n_phi, q)
    return RigidBody(centre=c, radius=float(radius), nodes=b.nodes + c[None, :], normals=b.normals,
                     weights=b.weights, force=np.asarray(force, dtype=np.float64),
                     torque=np.asarray(torque, dtype=np.float64))


def _attachment_dirs(n: int, n_theta: int, n_phi: int) -> np.ndarray:
    """n near-uniform unit vectors, each at the centre of a distinct cell of a
    refined (theta, phi) patch grid, so that no attachment point falls on a
    Gauss-Legendre node: Fibonacci-sphere directions, each moved to the
    nearest unused cell centre (k x k cells per patch, k the smallest with
    at least two cells per fiber)."""
    k = 1
    while n_theta * n_phi * k * k < 2 * n:
        k += 1
    th = (np.arange(n_theta * k) + 0.5) * math.pi / (n_theta * k)
    ph = (np.arange(n_phi * k) + 0.5) * 2.0 * math.pi / (n_phi * k)
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    cand = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    used = np.zeros(cand.shape[0], dtype=bool)
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = np.zeros((n, 3))
    for i in range(n):
        z = 1.0 - (2.0 * i + 1.0) / n
        r = math.sqrt(max(0.0, 1.0 - z * z))
        d = np.array([r * math.cos(golden * i), r * math.sin(golden * i), z])
        score = cand @ d
        score[used] = -np.inf
        j = int(np.argmax(score))
        used[j] = True
        out[i] = cand[j]
    return out


def aster(n_fibers: int, N: int = 32, radius: float = 1.0, L: Optional[float] = None,
          R_periphery: Optional[float] = 6.0, body_grid=(8, 16), periphery_grid=(12, 24),
          attach: int = CLAMPED, force=None, torque=(0.0, 0.0, 0.0), fiber_force_std: float = 0.0,
          tilt: float = 0.0, seed: int = 0, mu=1.0, eps=1e-3, E=1.0, dt=1e-2) -> Suspension:
    """Fibers of length L (default 2 radius) attached at their minus ends
    (alpha = -1, the last node) to a rigid sphere of the given radius centred
    at the origin, pointing outwards (tilted from the normal by an angle
    uniform in [0, tilt]); a spherical periphery of radius R_periphery x
    radius (None: free space); a force on the sphere (default along z, of
    size E / (32 L^2): 1/32 of the elastic force scale, Table 2) and
    optional i.i.d. N(0, fiber_force_std^2) force per node on the fibers."""
    rng = np.random.default_rng(seed)
    L = 2.0 * radius if L is None else float(L)
    d = _attachment_dirs(n_fibers, body_grid[0], body_grid[1])
    dirs = d.copy()
    if tilt > 0.0:
        for m in range(n_fibers):
            p = np.cross(d[m], rng.normal(size=3))
            p /= np.linalg.norm(p)
            a = rng.uniform(0.0, tilt)
            dirs[m] = math.cos(a) * d[m] + math.sin(a) * p
    alpha = collocation_alpha(N)
    X = np.concatenate([radius * d[m][None, :] + ((alpha + 1.0) * L / 2.0)[:, None] * dirs[m][None, :]
                        for m in range(n_fibers)]) if n_fibers else np.zeros((0, 3))
    f_ext = fiber_force_std * rng.normal(size=X.shape) if fiber_force_std > 0.0 else np.zeros(X.shape)
    if force is None:
        force = (0.0, 0.0, E / (32.0 * L * L))
    body = sphere_body((0.0, 0.0, 0.0), radius, body_grid[0], body_grid[1], force, torque)
    bnd = None
    if R_periphery is not None:
        bnd = sphere_quadrature(R_periphery * radius, periphery_grid[0], periphery_grid[1])
    return Suspension(n_per_fiber=np.full(n_fibers, N, dtype=np.int32), X=X,
                      L=np.full(n_fibers, L), f_ext=f_ext, mu=mu, eps=eps, E=E, dt=dt, boundary=bnd,
                      body=body, attach=np.full(n_fibers, attach, dtype=np.int32))


def table2_aster(n_fibers: int, seed: int = 0, N: int = 31, grid=(16, 32)) -> Suspension:
    """The confined aster of Table 2: a sphere of radius r = 1 inside a
    no-slip sphere of radius 6, n_fibers fibers of length 2r with N = 31
    points clamped to it, a force of 1/32 of the elastic scale E / L^2 on the
    sphere only; eps = 1e-3, E = mu = 1.  dt = 2.5e-4 tau_E, inside the
    paper's stable range for every fiber count (tau_E = 8 pi mu L^4 / c,
    c = -ln(eps^2 e), the caption's elastic relaxation time).  Surface grids
    of 16 x 32 patches (8,192 nodes) on both spheres."""
    eps, L, mu = 1e-3, 2.0, 1.0
    tau_e = 8.0 * math.pi * mu * L ** 4 / (-math.log(eps * eps * math.e))
    return aster(n_fibers, N=N, radius=1.0, L=L, R_periphery=6.0, body_grid=grid, periphery_grid=grid,
                 attach=CLAMPED, seed=seed, mu=mu, eps=eps, E=1.0, dt=2.5e-4 * tau_e)
