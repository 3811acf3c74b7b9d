"""p-convergence pins of the oracle's discretisation (Sec. 2.3, nodal DG).

With Phi = I and Psi z = 0 the method reduces to the underlying DG model
(Sec. 2.3 with x = X). Its solution of a smooth problem must converge at the
optimal rate p + 1 in L2. Two exact solutions fix the problem:

* Burgers: d/dx(u^2/2) = 0.5 exp(mu x), u(0) = 1 has u = sqrt(1 + (exp(mu x) - 1)/mu);
* Euler: a parallel shear flow along d = (cos 0.4, sin 0.4) with density and
  speed varying across the stream and uniform pressure is a steady solution.
"""

import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as orc
from paper_2305_15661_gb300 import workloads as W

GAMMA = 1.4


def burgers_exact(x, mu):
    return np.sqrt(1.0 + (np.exp(mu * x) - 1.0) / mu)


def shear_exact(x, y, gamma=GAMMA, th=0.4):
    s = -math.sin(th) * x + math.cos(th) * y
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * s)
    q = 1.5 + 0.25 * np.cos(2 * math.pi * s)
    return np.stack([rho, rho * q * math.cos(th), rho * q * math.sin(th),
                     1.0 / (gamma - 1.0) + 0.5 * rho * q * q], axis=-1)


def newton(res, jac, U, tol=1e-11, maxit=20):
    for _ in range(maxit):
        R = res(U)
        if np.linalg.norm(R) < tol:
            return U
        U = U - jac(U, R)
    assert np.linalg.norm(res(U)) < tol * 10
    return U


def burgers_error(p, ne, mu):
    X, ev = W.interval_mesh(ne)
    O = orc.Oracle(orc.PROB_BURGERS1D, p, X, ev)
    nodes, _ = O.ref_nodes()
    xn = (X[ev[:, 0]][:, None] + nodes[:, 0][None, :] / ne).ravel()
    U = burgers_exact(xn, mu)
    mu_a = np.array([mu])
    U = newton(lambda U: O.residual(U, X, mu_a)[0],
               lambda U, R: np.linalg.solve(O.jacobian_dense(U, X, mu_a)[0], R), U)
    gx, gw = np.polynomial.legendre.leggauss(10)
    t = 0.5 * (1 + gx)
    phi, _ = O.ref_basis(t[:, None])
    err = 0.0
    for e in range(ne):
        xq = X[e] + t / ne
        uh = phi @ U[e * O.nb:(e + 1) * O.nb]
        err += np.sum(0.5 * gw / ne * (uh - burgers_exact(xq, mu)) ** 2)
    return math.sqrt(err)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_burgers_p_convergence(p):
    mu = 1.5
    errs = [burgers_error(p, ne, mu) for ne in (8, 16, 32)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > p + 1 - 0.25, (errs, rates)


def euler_error(p, n):
    X, ev = W.square_tri_mesh(n)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA, bc_mode=orc.BC_SHEAR_TEST)
    nodes, _ = O.ref_nodes()
    A = X[ev[:, 0]]
    B = X[ev[:, 1]]
    C = X[ev[:, 2]]
    P = A[:, None, :] + nodes[None, :, 0:1] * (B - A)[:, None, :] + nodes[None, :, 1:2] * (C - A)[:, None, :]
    U = shear_exact(P[..., 0], P[..., 1]).ravel()
    mu = np.array([0.0, 0.0])
    x = X.ravel()

    def jsolve(U, R):
        return spla.spsolve(O.jacobian_sparse(U, x, mu).tocsc(), R)

    U = newton(lambda U: O.residual(U, x, mu)[0], jsolve, U, tol=1e-10)
    # L2 error with a collapsed Gauss rule of 8 x 8 points
    gx, gw = np.polynomial.legendre.leggauss(8)
    a, b = np.meshgrid(gx, gx, indexing="xy")
    wa, wb = np.meshgrid(gw, gw, indexing="xy")
    r = (0.25 * (1 + a) * (1 - b)).ravel()
    s = (0.5 * (1 + b)).ravel()
    wq = (wa * wb * (1 - b) / 8).ravel()
    phi, _ = O.ref_basis(np.stack([r, s], axis=1))
    err = 0.0
    for e in range(O.n_elems):
        J = np.stack([B[e] - A[e], C[e] - A[e]], axis=1)
        det = abs(np.linalg.det(J))
        pts = A[e][None, :] + np.stack([r, s], axis=1) @ J.T
        Uh = phi @ U[e * O.nu:(e + 1) * O.nu].reshape(O.nb, 4)
        err += np.sum(wq * det * np.sum((Uh - shear_exact(pts[:, 0], pts[:, 1])) ** 2, axis=1))
    return math.sqrt(err)


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2])
def test_euler_shear_flow_p_convergence(p):
    errs = [euler_error(p, n) for n in (4, 8, 16)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > p + 1 - 0.35, (errs, rates)
