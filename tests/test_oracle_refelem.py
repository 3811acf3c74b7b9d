"""Pins of the oracle's reference element: quadrature, nodes and Lagrange basis.

The paper fixes only "nodal DG" (Sec. 2.3). The readings here: equispaced
Lagrange nodes (triangles: vertices, then edge-interior nodes edge by edge, then
interior nodes), Gauss-Legendre with p+2 points on intervals and faces, and the
collapsed (Duffy) Gauss rule with (p+2)^2 points on triangles. These tests pin them against
numpy's Gauss-Legendre routine and against exact integrals and interpolation
identities.
"""

import math

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import workloads as W


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8])
def test_gauss_legendre_matches_numpy(n):
    x, w = orc.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=1e-15)
    np.testing.assert_allclose(w, wr, atol=1e-15)


def _tri_oracle(p):
    X, ev = W.square_tri_mesh(1)
    return orc.Oracle(orc.PROB_EULER2D, p, X, ev)


def _line_oracle(p):
    X, ev = W.interval_mesh(2)
    return orc.Oracle(orc.PROB_BURGERS1D, p, X, ev)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_triangle_rule_exact_monomials(p):
    O = _tri_oracle(p)
    vq, vw, ft, fw = O.ref_quadrature()
    n1d = p + 2
    assert len(vw) == n1d * n1d
    # collapsed Gauss rule with n points per direction integrates total degree 2n-2 exactly
    for a in range(2 * n1d - 1):
        for b in range(2 * n1d - 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = np.sum(vw * vq[:, 0] ** a * vq[:, 1] ** b)
            assert abs(got - exact) < 1e-15, (a, b, got, exact)
    # face rule on [0, 1] exact for degree 2n-1
    for a in range(2 * n1d):
        assert abs(np.sum(fw * ft ** a) - 1.0 / (a + 1)) < 1e-15


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_interval_rule_exact_monomials(p):
    O = _line_oracle(p)
    vq, vw, ft, fw = O.ref_quadrature()
    for a in range(2 * (p + 2)):
        assert abs(np.sum(vw * vq[:, 0] ** a) - 1.0 / (a + 1)) < 1e-15


@pytest.mark.parametrize("dim,p", [(1, 0), (1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3), (2, 4)])
def test_lagrange_basis_identities(dim, p):
    O = _line_oracle(p) if dim == 1 else _tri_oracle(p)
    nodes, fn = O.ref_nodes()
    nb = O.nb
    # Lagrange property phi_i(node_j) = delta_ij
    phi, _ = O.ref_basis(nodes)
    np.testing.assert_allclose(phi, np.eye(nb), atol=1e-12)
    # partition of unity, zero-sum gradients and reproduction of every monomial of degree <= p
    rng = np.random.default_rng(0)
    if dim == 1:
        pts = rng.uniform(0, 1, size=(20, 1))
        monos = [(a,) for a in range(p + 1)]
    else:
        r = rng.uniform(0, 1, size=(20, 2))
        pts = np.where(r.sum(1, keepdims=True) > 1, 1 - r, r)
        monos = [(a, b) for a in range(p + 1) for b in range(p + 1 - a)]
    phi, dphi = O.ref_basis(pts)
    np.testing.assert_allclose(phi.sum(1), 1.0, atol=1e-12)
    np.testing.assert_allclose(dphi.sum(1), 0.0, atol=1e-10)
    for mono in monos:
        f_nodes = np.prod(nodes ** np.array(mono), axis=1)
        f_pts = np.prod(pts ** np.array(mono), axis=1)
        np.testing.assert_allclose(phi @ f_nodes, f_pts, atol=1e-12)
        for d in range(dim):
            e = np.array(mono)
            if e[d] == 0:
                g = np.zeros(len(pts))
            else:
                e2 = e.copy()
                e2[d] -= 1
                g = e[d] * np.prod(pts ** e2, axis=1)
            np.testing.assert_allclose(dphi[:, :, d] @ f_nodes, g, atol=1e-10)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_triangle_face_nodes_lie_on_edges_in_order(p):
    O = _tri_oracle(p)
    nodes, fn = O.ref_nodes()
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    assert fn.shape == (3, p + 1)
    for k in range(3):
        a, b = V[k], V[(k + 1) % 3]
        for j, node in enumerate(fn[k]):
            np.testing.assert_allclose(nodes[node], a + (j / p) * (b - a), atol=1e-15)
    # vertices first, then edge-interior nodes, then interior nodes
    np.testing.assert_allclose(nodes[:3], V)
    # basis functions of nodes off an edge vanish on that edge
    t = np.linspace(0, 1, 7)
    for k in range(3):
        a, b = V[k], V[(k + 1) % 3]
        pts = a + t[:, None] * (b - a)
        phi, _ = O.ref_basis(pts)
        off = [i for i in range(O.nb) if i not in fn[k]]
        assert np.max(np.abs(phi[:, off])) < 1e-13


def test_neighbors_of_structured_mesh():
    X, ev = W.square_tri_mesh(3)
    O = orc.Oracle(orc.PROB_EULER2D, 2, X, ev)
    nbr, nbf = O.neighbors()
    # every interior edge is shared by exactly two elements, consistently
    for e in range(O.n_elems):
        for k in range(3):
            e2, k2 = nbr[e, k], nbf[e, k]
            if e2 < 0:
                a, b = X[ev[e, k]], X[ev[e, (k + 1) % 3]]
                on_bnd = any(abs(a[c] - v) < 1e-12 and abs(b[c] - v) < 1e-12 for c in (0, 1) for v in (0.0, 1.0))
                assert on_bnd
            else:
                assert nbr[e2, k2] == e and nbf[e2, k2] == k
                assert ev[e, k] == ev[e2, (k2 + 1) % 3] and ev[e, (k + 1) % 3] == ev[e2, k2]
    n_bnd = int((nbr < 0).sum())
    assert n_bnd == 4 * 3
