"""Seeded synthetic inputs for the EQP-IFT hot path.

This module builds meshes, bases (Phi, Psi), empirical-quadrature weight sets
(rho), parameters (mu) and evaluation points (w, tau). It holds none of the
method's arithmetic: no residual, flux, Jacobian, reduction or solver step. Both
the CUDA library's tests and the CPU oracle's tests take their inputs from here.

Random numbers come from a counter-based splitmix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) and the
Box-Muller transform for normals, so every array is a pure function of
(seed, stream, index).

The paper's meshes and snapshots (space-time Burgers, NACA0012; Sec. 4) are not
available, so these synthetic workloads stand in for them:

* Burgers 1-D: d/dx(u^2/2) = 0.5 exp(mu x) on [0, 1], u(0) = 1, p = 2, 200
  uniform elements; Phi = QR of a seeded Gaussian 600 x 5; Psi = the raw modes
  sin(k pi X), k = 1, 2 at the 201 vertices; mu ~ U[1, 2].
* Euler 2-D: unit square, n x n cells each cut along the same diagonal
  (2 n^2 triangles), Mach-2 free stream (rho = 1, P = 1, c = sqrt(gamma));
  Phi = QR([U_pert, G]) with U_pert = U_inf (1 + 1e-2 xi) and G a seeded
  Gaussian; Psi = orthonormalised smooth bump modes that vanish on the boundary.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """n outputs of splitmix64 for the key (seed, stream), as uint64."""
    with np.errstate(over="ignore"):
        base = _mix(np.array([(seed * 0x100000001B3 + stream * 0x9E37) & 0xFFFFFFFFFFFFFFFF],
                             dtype=np.uint64))[0]
        ctr = np.arange(1, n + 1, dtype=np.uint64)
        return _mix(base + ctr * _GOLDEN)


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


# ---------------------------------------------------------------------------
# Meshes
# ---------------------------------------------------------------------------

def interval_mesh(n_elems: int, a: float = 0.0, b: float = 1.0):
    """Uniform 1-D mesh: vertices (n_elems+1,), elements (n_elems, 2) left-to-right."""
    X = np.linspace(a, b, n_elems + 1)
    ev = np.stack([np.arange(n_elems), np.arange(1, n_elems + 1)], axis=1).astype(np.int32)
    return X, ev


def square_tri_mesh(n: int):
    """Unit square, n x n cells, each cut along the diagonal from (i, j) to (i+1, j+1).

    Returns vertices ((n+1)^2, 2) row-major in (i, j) with i fastest, and
    counter-clockwise triangles (2 n^2, 3), two per cell in cell order.
    """
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    X = np.stack([ii.ravel() / n, jj.ravel() / n], axis=1).astype(np.float64)

    def vid(i, j):
        return j * (n + 1) + i

    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    ci = ci.ravel()
    cj = cj.ravel()
    v00, v10, v01, v11 = vid(ci, cj), vid(ci + 1, cj), vid(ci, cj + 1), vid(ci + 1, cj + 1)
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    ev = np.empty((2 * n * n, 3), dtype=np.int32)
    ev[0::2] = t1
    ev[1::2] = t2
    return X, ev


def square_tri_mesh_q2(n: int, curve: float = 0.0):
    """Six-node (q = 2) triangles: the triangles of square_tri_mesh with a node at the
    midpoint of every edge (per element: the three vertices, then the midpoints of edges
    0-1, 1-2 and 2-0), after which every node moves by the smooth map
    x -> x + curve / (2 pi) (sin(pi x) sin(pi y), sin(pi x) sin(2 pi y)).
    The map fixes the boundary of the unit square and bends the interior edges into
    parabolas; curve = 0 leaves straight-sided elements with midpoint nodes.
    """
    X, ev = square_tri_mesh(n)
    nv = X.shape[0]
    ne = ev.shape[0]
    ev6 = np.empty((ne, 6), dtype=np.int32)
    ev6[:, :3] = ev
    edge_id = {}
    mids = []
    for e in range(ne):
        for k in range(3):
            a, b = int(ev[e, k]), int(ev[e, (k + 1) % 3])
            key = (a, b) if a < b else (b, a)
            if key not in edge_id:
                edge_id[key] = nv + len(mids)
                mids.append(0.5 * (X[a] + X[b]))
            ev6[e, 3 + k] = edge_id[key]
    Xq = np.concatenate([X, np.asarray(mids)], axis=0)
    if curve:
        x, y = Xq[:, 0], Xq[:, 1]
        d = np.stack([np.sin(math.pi * x) * np.sin(math.pi * y), np.sin(math.pi * x) * np.sin(2 * math.pi * y)],
                     axis=1)
        Xq = Xq + curve / (2 * math.pi) * d
    return Xq, ev6


def boundary_elements(X: np.ndarray, ev: np.ndarray, tol: float = 1e-12):
    """Per side of the unit square (x=0, x=1, y=0, y=1), the elements with an edge on it."""
    out = []
    for c, val in ((0, 0.0), (0, 1.0), (1, 0.0), (1, 1.0)):
        on = np.abs(X[:, c] - val) < tol
        cnt = on[ev].sum(axis=1)
        out.append(np.nonzero(cnt >= 2)[0])
    return out


def triangle_areas(X: np.ndarray, ev: np.ndarray) -> np.ndarray:
    """Signed areas of triangles (input validation of generated meshes only)."""
    a, b, c = X[ev[:, 0]], X[ev[:, 1]], X[ev[:, 2]]
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))


def freestream_state(gamma: float, mach: float, alpha: float) -> np.ndarray:
    """Conserved free-stream state (rho, rho u, rho v, rho E) with rho = 1, P = 1, c = sqrt(gamma)."""
    c = math.sqrt(gamma)
    vx, vy = mach * c * math.cos(alpha), mach * c * math.sin(alpha)
    return np.array([1.0, vx, vy, 1.0 / (gamma - 1.0) + 0.5 * (vx * vx + vy * vy)])


def _orthonormal_columns(A: np.ndarray) -> np.ndarray:
    """Q of A = QR with diag(R) > 0 (unique for full column rank). Tall matrices
    use Cholesky QR applied twice (Gram matrix, Cholesky factor, triangular
    solve), which is BLAS-3 and orthogonal to rounding for the well-conditioned
    bases generated here; small ones use Householder QR."""
    if A.shape[0] < 100000 or A.shape[1] == 0:
        Q, R = np.linalg.qr(A)
        s = np.sign(np.diag(R))
        s[s == 0] = 1.0
        return Q * s
    Q = A
    for _ in range(2):
        L = np.linalg.cholesky(Q.T @ Q)  # Q^T Q = L L^T, R = L^T
        Q = Q @ np.linalg.inv(L.T)
    return Q


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

PROB_BURGERS1D = 1
PROB_EULER2D = 2


@dataclass
class Workload:
    """A complete synthetic problem instance."""

    name: str
    problem: int
    p: int
    X: np.ndarray            # n_verts x dim reference nodes (all geometry nodes)
    ev: np.ndarray           # n_elems x (dim+1) int32 (q = 2: n_elems x 6, vertices then edge midpoints)
    Phi: np.ndarray          # N_u x k_u, row-major, element-major rows
    Psi: np.ndarray          # N_x x k_x
    gamma: float = 1.4
    kappa: float = 0.0
    mus: np.ndarray = field(default_factory=lambda: np.zeros((1, 2)))   # queries x n_mu
    w_eval: np.ndarray = None   # evaluation point(s) for assembly tests
    tau_eval: np.ndarray = None
    U_guess: np.ndarray = None  # per-query constant state used by the paper's initialisation
    rho_sets: list = None       # per query: (elems int32, rho float64) or None for rho = 1
    q: int = 1                  # geometry degree (2: curved six-node triangles)

    @property
    def dim(self):
        return 1 if self.problem == PROB_BURGERS1D else 2

    @property
    def m(self):
        return 1 if self.problem == PROB_BURGERS1D else 4

    @property
    def n_elems(self):
        return self.ev.shape[0]

    @property
    def n_verts(self):
        return self.X.shape[0]

    @property
    def nb(self):
        return self.p + 1 if self.dim == 1 else (self.p + 1) * (self.p + 2) // 2

    @property
    def nu(self):
        return self.nb * self.m

    @property
    def ku(self):
        return self.Phi.shape[1]

    @property
    def kx(self):
        return self.Psi.shape[1]


def burgers_workload(n_elems: int = 200, p: int = 2, k_u: int = 5, seed: int = 1, n_mu: int = 1,
                     name: str = "burgers1d") -> Workload:
    """1-D steady Burgers with a parameterised source, DG degree p (Phi: QR of a Gaussian)."""
    X, ev = interval_mesh(n_elems)
    Nu = n_elems * (p + 1)
    Phi = _orthonormal_columns(normal(seed, 11, Nu * k_u).reshape(Nu, k_u))
    Psi = np.stack([np.sin(k * math.pi * X) for k in (1, 2)], axis=1)
    mus = (1.0 + uniform(seed, 12, n_mu)).reshape(n_mu, 1)
    h = 1.0 / n_elems
    tau = 0.1 * h * (2.0 * uniform(seed, 13, 2) - 1.0)
    w = normal(seed, 14, k_u)
    return Workload(name=name, problem=PROB_BURGERS1D, p=p, X=X, ev=ev, Phi=Phi, Psi=Psi, mus=mus,
                    w_eval=w, tau_eval=tau, U_guess=np.ones(1), rho_sets=None)


def _bump_modes(X: np.ndarray, k_x: int) -> np.ndarray:
    """Displacement modes that vanish on the boundary of the unit square, vertex-major (N_x x k_x)."""
    x, y = X[:, 0], X[:, 1]
    s = np.sin
    pi = math.pi
    fam = [
        (s(pi * x) * s(pi * y), 0),
        (s(pi * x) * s(pi * y), 1),
        (s(2 * pi * x) * s(pi * y), 0),
        (s(pi * x) * s(2 * pi * y), 1),
        (s(pi * x) * s(2 * pi * y), 0),
        (s(2 * pi * x) * s(pi * y), 1),
        (s(2 * pi * x) * s(2 * pi * y), 0),
        (s(2 * pi * x) * s(2 * pi * y), 1),
    ]
    if k_x > len(fam):
        raise ValueError("at most 8 mesh modes")
    Nx = 2 * X.shape[0]
    M = np.zeros((Nx, k_x))
    for c in range(k_x):
        f, comp = fam[c]
        M[comp::2, c] = f
    return M


def euler_workload(n: int = 100, p: int = 2, k_u: int = 20, k_x: int = 4, seed: int = 2,
                   mach: float = 2.0, alpha: float = 0.0, n_mu: int = 1, mu_box: bool = False,
                   gamma: float = 1.4, name: str = "euler2d", q: int = 1, curve: float = 0.0) -> Workload:
    """2-D steady Euler on the unit square with a Mach-2 free stream.

    Phi = QR([U_pert, G]) with U_pert = U_inf (1 + 1e-2 xi), G ~ N(0, 1); the
    first column is U_pert/|U_pert| with positive sign. Psi = QR of smooth bump
    modes. The evaluation point (w, tau) keeps every triangle's area above half
    its reference value. q = 2: curved six-node triangles (square_tri_mesh_q2 with
    the given curve); the mesh modes act on every geometry node.
    """
    X, ev = square_tri_mesh(n) if q == 1 else square_tri_mesh_q2(n, curve)
    ne = ev.shape[0]
    nb = (p + 1) * (p + 2) // 2
    Nu = ne * nb * 4
    U_inf = freestream_state(gamma, mach, alpha)
    xi = normal(seed, 21, Nu)
    U_pert = np.tile(U_inf, ne * nb) * (1.0 + 1e-2 * xi)
    G = normal(seed, 22, Nu * (k_u - 1)).reshape(Nu, k_u - 1)
    Phi = _orthonormal_columns(np.concatenate([U_pert[:, None], G], axis=1))
    Psi = _orthonormal_columns(_bump_modes(X, k_x))
    nrm = float(np.linalg.norm(U_pert))
    zeta = normal(seed, 23, k_u - 1)
    w = np.concatenate([[nrm], 1e-3 * nrm * zeta])
    # mesh-motion amplitude: scale a seeded direction until every area ratio > 0.5
    d = normal(seed, 24, k_x)
    d /= np.linalg.norm(d)
    A0 = triangle_areas(X, ev)
    h = 1.0 / n
    amp = 0.2 * h * math.sqrt(X.shape[0])  # Psi columns have unit 2-norm over all vertices
    for _ in range(60):
        Xd = X + (Psi @ (amp * d)).reshape(-1, 2)
        if np.min(triangle_areas(Xd, ev) / A0) > 0.5:
            break
        amp *= 0.5
    tau = amp * d
    if mu_box:
        mus = mu_box_samples(seed, 25, n_mu)
    else:
        mus = np.tile(np.array([[mach, alpha]]), (n_mu, 1))
    return Workload(name=name, problem=PROB_EULER2D, p=p, X=X, ev=ev, Phi=Phi, Psi=Psi, gamma=gamma,
                    mus=mus, w_eval=w, tau_eval=tau, U_guess=U_inf, rho_sets=None, q=q)


MU_BOX_LO = np.array([1.8, math.radians(-2.0)])
MU_BOX_WIDTH = np.array([0.4, math.radians(4.0)])


def mu_box_samples(seed: int, stream: int, n: int) -> np.ndarray:
    """n parameter points (Mach, angle) uniform in [1.8, 2.2] x [-2 deg, 2 deg]."""
    u = uniform(seed, stream, 2 * n).reshape(n, 2)
    return MU_BOX_LO + MU_BOX_WIDTH * u


def eq_weight_sets(wl: Workload, n_sets: int, seed: int, lo: int = 100, hi: int = 2000,
                   rho_lo: float = 0.5, rho_hi: float = 50.0):
    """Per-query sparse weight sets: counts log-uniform in [lo, hi], at least one element
    on each boundary side, element ids sorted, values uniform in [rho_lo, rho_hi]."""
    ne = wl.n_elems
    bnd = boundary_elements(wl.X, wl.ev) if wl.dim == 2 else [np.array([0]), np.array([ne - 1])]
    u = uniform(seed, 31, n_sets)
    counts = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    counts = np.clip(counts, lo, min(hi, ne))
    sets = []
    for q in range(n_sets):
        c = int(counts[q])
        # one element per boundary side, then a seeded draw without replacement
        ub = uniform(seed, 1000 + 2 * q, len(bnd))
        chosen = {int(b[int(ub[i] * len(b))]) for i, b in enumerate(bnd)}
        keys = uniform(seed, 1001 + 2 * q, ne)
        order = np.argsort(keys, kind="stable")
        for e in order:
            if len(chosen) >= c:
                break
            chosen.add(int(e))
        elems = np.array(sorted(chosen), dtype=np.int32)
        rho = rho_lo + (rho_hi - rho_lo) * uniform(seed, 5000 + q, len(elems))
        sets.append((elems, rho))
    return sets


def replicate_guess(wl: Workload, U_const: np.ndarray) -> np.ndarray:
    """A constant state at every DOF (the state whose projection starts the solver)."""
    return np.tile(np.asarray(U_const, dtype=np.float64), wl.n_elems * wl.nb)
