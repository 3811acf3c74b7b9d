"""Pins of the oracle's curved (q = 2) geometry: the six-node quadratic element map
with the mapping Jacobian G, its determinant g and the scaled face normals taken
at every quadrature point (Eq. p2r-flux), and the distortion of Eq. dist_elem1
integrated with the volume rule.

* midpoint nodes on straight edges reproduce the straight-sided (q = 1) residual,
  its state Jacobians and the distortion; the mesh Jacobians agree through the
  chain rule of midpoint = average of the two vertices;
* free-stream preservation on curved, deformed meshes: the cofactor g G^{-T} of a
  quadratic map is linear in the master coordinates, so the volume and face
  integrals of a constant state are exact and cancel (Piola identity);
* central finite differences of every element Jacobian on a curved mesh;
* App. A on a curved mesh: the elemental weighted sums equal the same quantities
  formed from the globally assembled residual and Jacobians.
"""

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import workloads as W

GAMMA = 1.4


def _rng_state(O, seed, mu, scale=0.05):
    rng = np.random.default_rng(seed)
    U = np.tile(orc.freestream(GAMMA, mu), O.Nu // 4)
    return U * (1.0 + scale * rng.normal(size=U.shape))


def _interior_shift(X, amp, n, seed):
    rng = np.random.default_rng(seed)
    interior = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    d = rng.uniform(-1, 1, size=X.shape) * amp / n
    d[~interior] = 0.0
    return X + d


@pytest.mark.parametrize("p", [1, 2, 3])
def test_straight_q2_equals_q1(p):
    n = 3
    X1, ev1 = W.square_tri_mesh(n)
    X2, ev2 = W.square_tri_mesh_q2(n, curve=0.0)
    O1 = orc.Oracle(orc.PROB_EULER2D, p, X1, ev1, gamma=GAMMA, kappa=0.1)
    O2 = orc.Oracle(orc.PROB_EULER2D, p, X2, ev2, gamma=GAMMA, kappa=0.1, q=2)
    assert O2.nxe == 12 and O1.nxe == 6
    mu = np.array([2.0, 0.02])
    U = _rng_state(O1, 3, mu)
    # deform the vertices; the midpoints follow as averages, so the q = 2 elements stay straight
    x1 = _interior_shift(X1, 0.3, n, seed=5)
    x2 = np.concatenate([x1, np.zeros((X2.shape[0] - X1.shape[0], 2))])
    for e in range(ev2.shape[0]):
        for k in range(3):
            a, b = ev2[e, k], ev2[e, (k + 1) % 3]
            x2[ev2[e, 3 + k]] = 0.5 * (x1[a] + x1[b])
    for e in (0, 5, 11, 17):
        Ue, Up, xe1 = O1.gather(U, x1.ravel(), e)
        _, _, xe2 = O2.gather(U, x2.ravel(), e)
        r1 = O1.element(e, Ue, Up, xe1, mu)
        r2 = O2.element(e, Ue, Up, xe2, mu)
        sc = np.abs(r1["R"]).max()
        assert np.abs(r2["R"] - r1["R"]).max() <= 1e-12 * sc
        for key in ("JU", "JUp"):
            assert np.abs(r2[key] - r1[key]).max() <= 1e-12 * np.abs(r1[key]).max(), key
        # x_mid(k) = (x_k + x_{k+1}) / 2: d/dx_v (q = 1) = d/dx_v + 1/2 sum of the adjacent midpoints (q = 2)
        Jx2 = r2["Jx"].reshape(O1.nu, 6, 2)
        dN2 = r2["dN"].reshape(6, 2)
        Jchain = Jx2[:, :3, :].copy()
        dNchain = dN2[:3].copy()
        for k in range(3):
            for v in (k, (k + 1) % 3):
                Jchain[:, v, :] += 0.5 * Jx2[:, 3 + k, :]
                dNchain[v] += 0.5 * dN2[3 + k]
        assert np.abs(Jchain.reshape(O1.nu, 6) - r1["Jx"]).max() <= 1e-11 * np.abs(r1["Jx"]).max()
        assert abs(r2["N"] - r1["N"]) <= 1e-12 * max(abs(r1["N"]), 1e-30) + 1e-15
        assert np.abs(dNchain.ravel() - r1["dN"]).max() <= 1e-11 * np.abs(r1["dN"]).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_freestream_preservation_curved(p):
    n = 4
    X, ev = W.square_tri_mesh_q2(n, curve=0.4)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA, q=2)
    mu = np.array([2.0, 0.03])
    Uinf = orc.freestream(GAMMA, mu)
    x = _interior_shift(X, 0.1, n, seed=p)  # moves midpoints off their chords as well
    U = np.tile(Uinf, O.Nu // 4)
    R, N, bad = O.residual(U, x.ravel(), mu)
    f, _ = orc.euler_flux(GAMMA, Uinf)
    assert bad == 0
    assert np.abs(R).max() <= 1e-12 * np.abs(f).max(), np.abs(R).max()
    # and the edges really are curved: some midpoint is off its chord by a visible amount
    off = []
    for e in range(ev.shape[0]):
        for k in range(3):
            a, b, m = ev[e, k], ev[e, (k + 1) % 3], ev[e, 3 + k]
            off.append(np.linalg.norm(x[m] - 0.5 * (x[a] + x[b])))
    assert max(off) > 1e-2 / n


def _fd_check(fun, x0, J, h=1e-6, rtol=1e-6, atol=1e-9):
    # atol: the rounding of central differences of O(1) values with h = 1e-6
    scale = max(np.abs(J).max(), 1e-30)
    for j in range(x0.size):
        xp, xm = x0.copy(), x0.copy()
        hh = h * max(1.0, abs(x0[j]))
        xp[j] += hh
        xm[j] -= hh
        col = (fun(xp) - fun(xm)) / (2 * hh)
        assert np.abs(col - J[:, j]).max() <= rtol * scale + atol, (j, np.abs(col - J[:, j]).max(), scale)


@pytest.mark.parametrize("p", [1, 2])
def test_curved_jacobians_finite_differences(p):
    n = 3
    X, ev = W.square_tri_mesh_q2(n, curve=0.4)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA, kappa=0.1, q=2)
    mu = np.array([2.0, 0.02])
    U = _rng_state(O, 9, mu)
    x = _interior_shift(X, 0.1, n, seed=4).ravel()
    for e in (0, 4, 9, 13):
        Ue, Up, xe = O.gather(U, x, e)
        out = O.element(e, Ue, Up, xe, mu)
        _fd_check(lambda v: O.element(e, v, Up, xe, mu, jac=False)["R"], Ue, out["JU"])
        _fd_check(lambda v: O.element(e, Ue, v, xe, mu, jac=False)["R"], Up, out["JUp"])
        _fd_check(lambda v: O.element(e, Ue, Up, v, mu, jac=False)["R"], xe, out["Jx"])
        _fd_check(lambda v: np.array([O.element(e, Ue, Up, v, mu, jac=False)["N"]]), xe, out["dN"][None, :])


def test_curved_elemental_equals_global():
    wl = W.euler_workload(n=3, p=2, k_u=6, k_x=3, seed=4, q=2, curve=0.4)
    O = orc.Oracle.from_workload(wl, kappa=0.1)
    mu = wl.mus[0]
    w, tau = wl.w_eval, wl.tau_eval
    rng = np.random.default_rng(1)
    elems = np.sort(rng.choice(O.n_elems, 7, replace=False)).astype(np.int32)
    rho = rng.uniform(0.5, 50, 7)
    rho_e = np.zeros(O.n_elems)
    rho_e[elems] = rho
    r = O.reduced(wl.Phi, wl.Psi, w, tau, mu, rho_set=(elems, rho))
    U = wl.Phi @ w
    x = wl.X.ravel() + wl.Psi @ tau
    R, N, bad = O.residual(U, x, mu)
    assert bad == 0
    dRdU, dRdx, dNdx = O.jacobian_dense(U, x, mu)
    Wd = np.repeat(rho_e, O.nu)
    A = np.concatenate([dRdU @ wl.Phi, dRdx @ wl.Psi], axis=1)
    B = np.concatenate([np.zeros((O.n_elems, wl.ku)), dNdx @ wl.Psi], axis=1)
    S = wl.Phi.T @ (dRdU.T @ (Wd * R))
    T = wl.Psi.T @ (dRdx.T @ (Wd * R) + dNdx.T @ (rho_e * N))
    H = A.T @ (Wd[:, None] * A) + B.T @ (rho_e[:, None] * B)
    J = 0.5 * (R @ (Wd * R) + N @ (rho_e * N))
    np.testing.assert_allclose(r["S"], S, rtol=1e-12, atol=1e-12 * np.abs(S).max())
    np.testing.assert_allclose(r["T"], T, rtol=1e-12, atol=1e-12 * np.abs(T).max())
    np.testing.assert_allclose(r["H"], H, rtol=1e-12, atol=1e-12 * np.abs(H).max())
    assert abs(r["J"] - J) <= 1e-13 * J
    assert abs(wl.X.shape[0] - (16 + 33)) == 0  # 16 vertices and 33 edges of the 3 x 3 mesh
