"""Pins of the oracle's element residual, Jacobians and distortion term.

* free-stream preservation on deformed meshes (the transformed law of Sec. 2.2
  is equivalent to the physical one for any diffeomorphism; q = 1 and exact
  quadrature make the constant state an exact discrete solution);
* the reference-domain residual (Eq. p2r-flux) equals a physical-space DG
  residual written directly from Eq. claw-phys on the mapped mesh, and at
  z = 0 it is that standard DG residual on the reference mesh (Sec. 2.3);
* discrete conservation: interior face fluxes cancel between neighbours;
* a closed form for one Burgers element of degree 0;
* central finite differences of dR_e/dU_e, dR_e/dU_e', dR_e/dx_e, dN_e/dx_e;
* closed forms of the distortion of Eqs. dist_elem0-dist_elem1.
"""

import math

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import workloads as W

GAMMA = 1.4


def deformed_vertices(X, ev, amp, seed, n):
    """Random interior-vertex displacement keeping every area above half its reference."""
    rng = np.random.default_rng(seed)
    interior = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    d = rng.uniform(-1, 1, size=X.shape) * amp / n
    d[~interior] = 0.0
    x = X + d
    A0 = W.triangle_areas(X, ev)
    assert np.min(W.triangle_areas(x, ev) / A0) > 0.15
    return x


def random_state(O, seed, base, scale=0.05):
    rng = np.random.default_rng(seed)
    U = np.tile(base, O.Nu // len(base))
    return U * (1.0 + scale * rng.normal(size=U.shape))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_freestream_preservation_deformed(p):
    n = 4
    X, ev = W.square_tri_mesh(n)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA)
    mu = np.array([2.0, 0.03])
    Uinf = orc.freestream(GAMMA, mu)
    x = deformed_vertices(X, ev, 0.3, seed=p, n=n)
    U = np.tile(Uinf, O.Nu // 4)
    R, N, bad = O.residual(U, x.ravel(), mu)
    f, _ = orc.euler_flux(GAMMA, Uinf)
    scale = np.abs(f).max() / n
    assert bad == 0
    assert np.abs(R).max() <= 1e-12 * scale * 100, np.abs(R).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_reference_domain_equals_physical_dg(p):
    n = 3
    X, ev = W.square_tri_mesh(n)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA)
    mu = np.array([2.0, -0.02])
    U = random_state(O, 7, orc.freestream(GAMMA, mu))
    for xx in (X, deformed_vertices(X, ev, 0.35, seed=11, n=n)):
        x = xx.ravel()
        for e in range(O.n_elems):
            Ue, Up, xe = O.gather(U, x, e)
            Rref = O.element(e, Ue, Up, xe, mu, jac=False)["R"]
            Rphys = O.element_physical(e, Ue, Up, xe, mu)
            np.testing.assert_allclose(Rref, Rphys, rtol=1e-12, atol=1e-13 * np.abs(Rphys).max())


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_burgers_reference_equals_physical(p):
    X, ev = W.interval_mesh(6)
    O = orc.Oracle(orc.PROB_BURGERS1D, p, X, ev)
    rng = np.random.default_rng(p)
    U = 1.0 + 0.3 * rng.normal(size=O.Nu)
    x = X + np.concatenate([[0], 0.04 * rng.uniform(-1, 1, 5), [0]])
    mu = np.array([1.4])
    for e in range(O.n_elems):
        Ue, Up, xe = O.gather(U, x, e)
        np.testing.assert_allclose(O.element(e, Ue, Up, xe, mu, jac=False)["R"],
                                   O.element_physical(e, Ue, Up, xe, mu), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_interior_fluxes_cancel(p):
    # sum_i R_e[i] = boundary flux of e (partition of unity, S = 0); summed over all
    # elements the interior face fluxes cancel exactly when the neighbour traces are
    # taken at the matching points, so the total equals the boundary flux alone
    n = 3
    X, ev = W.square_tri_mesh(n)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA)
    mu = np.array([2.0, 0.0])
    Uinf = orc.freestream(GAMMA, mu)
    U = random_state(O, 5, Uinf, scale=0.1)
    x = deformed_vertices(X, ev, 0.3, seed=3, n=n).ravel()
    R, _, _ = O.residual(U, x, mu)
    total = R.reshape(-1, O.nb, 4).sum(axis=(0, 1))
    # boundary flux computed here from traces, the face rule and the Roe flux
    nbr, _ = O.neighbors()
    nodes, fn = O.ref_nodes()
    gx, gw = np.polynomial.legendre.leggauss(p + 2)
    tq, wq = 0.5 * (1 + gx), 0.5 * gw
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    xv = x.reshape(-1, 2)
    bflux = np.zeros(4)
    for e in range(O.n_elems):
        for k in range(3):
            if nbr[e, k] >= 0:
                continue
            a, b = xv[ev[e, k]], xv[ev[e, (k + 1) % 3]]
            ed = b - a
            nt = np.array([ed[1], -ed[0]])
            pts = V[k] + tq[:, None] * (V[(k + 1) % 3] - V[k])
            phi, _ = O.ref_basis(pts)
            Uq = phi @ U[e * O.nu:(e + 1) * O.nu].reshape(O.nb, 4)
            for q in range(len(tq)):
                bflux += wq[q] * orc.euler_roe(GAMMA, Uq[q], Uinf, nt)
    np.testing.assert_allclose(total, bflux, rtol=1e-12, atol=1e-12 * np.abs(bflux).max())


def test_burgers_single_element_degree_zero_closed_form():
    # one element on [0, 1], p = 0, constant state u > 0: the inflow face gives
    # -f(1), the outflow face f(u), the source -int 0.5 exp(mu x) dx (Gauss rule with p+2 points)
    X, ev = W.interval_mesh(1)
    O = orc.Oracle(orc.PROB_BURGERS1D, 0, X, ev)
    gx, gw = np.polynomial.legendre.leggauss(2)
    for u in (0.4, 1.0, 1.7):
        for mu in (1.0, 1.6):
            src = np.sum(0.5 * gw * 0.5 * np.exp(mu * 0.5 * (1 + gx)))
            out = O.element(0, np.array([u]), np.zeros(2), np.array([0.0, 1.0]), np.array([mu]))
            assert abs(out["R"][0] - (0.5 * u * u - 0.5 - src)) < 1e-15
            assert abs(out["JU"][0, 0] - u) < 1e-15
    # a moved right end scales the source integral with the element length
    x1 = 0.9
    src = np.sum(0.5 * gw * x1 * 0.5 * np.exp(1.3 * x1 * 0.5 * (1 + gx)))
    out = O.element(0, np.array([1.2]), np.zeros(2), np.array([0.0, x1]), np.array([1.3]))
    assert abs(out["R"][0] - (0.72 - 0.5 - src)) < 1e-15


def _fd_check(fun, x0, J, h_rel=1e-6, rtol=1e-7, atol=1e-10):
    for j in range(len(x0)):
        h = h_rel * max(1.0, abs(x0[j]))
        xp = x0.copy()
        xm = x0.copy()
        xp[j] += h
        xm[j] -= h
        col = (fun(xp) - fun(xm)) / (2 * h)
        scale = np.abs(J).max()
        assert np.abs(col - J[:, j]).max() <= rtol * scale + atol, (j, np.abs(col - J[:, j]).max(), scale)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_euler_jacobians_finite_differences(p):
    n = 3
    X, ev = W.square_tri_mesh(n)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA, kappa=0.1)
    mu = np.array([2.0, 0.02])
    U = random_state(O, 9, orc.freestream(GAMMA, mu), scale=0.05)
    x = deformed_vertices(X, ev, 0.3, seed=4, n=n).ravel()
    for e in (0, 4, 9, 17):
        Ue, Up, xe = O.gather(U, x, e)
        out = O.element(e, Ue, Up, xe, mu)
        _fd_check(lambda v: O.element(e, v, Up, xe, mu, jac=False)["R"], Ue, out["JU"])
        _fd_check(lambda v: O.element(e, Ue, v, xe, mu, jac=False)["R"], Up, out["JUp"])
        _fd_check(lambda v: O.element(e, Ue, Up, v, mu, jac=False)["R"], xe, out["Jx"])
        _fd_check(lambda v: np.array([O.element(e, Ue, Up, v, mu, jac=False)["N"]]), xe, out["dN"][None, :])


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_burgers_jacobians_finite_differences(p):
    X, ev = W.interval_mesh(5)
    O = orc.Oracle(orc.PROB_BURGERS1D, p, X, ev)
    rng = np.random.default_rng(10 + p)
    U = 1.0 + 0.3 * rng.normal(size=O.Nu)
    x = X + np.concatenate([[0], 0.04 * rng.uniform(-1, 1, 4), [0]])
    mu = np.array([1.7])
    for e in range(5):
        Ue, Up, xe = O.gather(U, x, e)
        out = O.element(e, Ue, Up, xe, mu)
        _fd_check(lambda v: O.element(e, v, Up, xe, mu, jac=False)["R"], Ue, out["JU"])
        _fd_check(lambda v: O.element(e, Ue, v, xe, mu, jac=False)["R"], Up, out["JUp"])
        _fd_check(lambda v: O.element(e, Ue, Up, v, mu, jac=False)["R"], xe, out["Jx"])


def test_distortion_closed_forms():
    # eta_e = |Omega_0e| (|G|_F^2 / g)^2 for straight-sided triangles (d = 2):
    # 4 |Omega_0e| for any similarity (so N_e = 0), (2 + s^2)^2 |Omega_0e| for a shear
    X, ev = W.square_tri_mesh(1)
    kappa = 0.37
    O = orc.Oracle(orc.PROB_EULER2D, 2, X, ev, gamma=GAMMA, kappa=kappa)
    U = np.tile(orc.freestream(GAMMA, np.array([2.0, 0.0])), O.Nu // 4)
    mu = np.array([2.0, 0.0])
    area = 0.5
    th, sc = 0.7, 1.9
    Rm = sc * np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    for e in range(2):
        Ue, Up, xe = O.gather(U, X.ravel(), e)
        xs = (Rm @ xe.reshape(3, 2).T).T.ravel() + 0.3
        assert abs(O.element(e, Ue, Up, xs, mu, jac=False)["N"]) < 1e-13
        s = 0.45
        Gs = np.array([[1.0, s], [0.0, 1.0]])
        xsh = (Gs @ xe.reshape(3, 2).T).T.ravel()
        expect = kappa * area * ((2 + s * s) ** 2 - 4.0)
        assert abs(O.element(e, Ue, Up, xsh, mu, jac=False)["N"] - expect) < 1e-13
        # compressions below eps: g is clipped at eps = 1e-8, so eta = |Omega| (|G|^2 / eps)^2
        Gc = np.array([[1e-9, 0.0], [0.0, 1.0]])
        xc = (Gc @ xe.reshape(3, 2).T).T.ravel()
        expect = kappa * area * (((1e-18 + 1.0) / 1e-8) ** 2 - 4.0)
        got = O.element(e, Ue, Up, xc, mu, jac=False)["N"]
        assert abs(got - expect) <= 1e-12 * abs(expect)
    # in 1-D the distortion is constant (|G|^2 / g^2 = 1), so N_e = 0
    Xl, evl = W.interval_mesh(2)
    Ol = orc.Oracle(orc.PROB_BURGERS1D, 1, Xl, evl, kappa=kappa)
    out = Ol.element(0, np.ones(2), np.ones(2), np.array([0.0, 0.3]), np.array([1.0]))
    assert abs(out["N"]) < 1e-15 and np.abs(out["dN"]).max() < 1e-14


def test_nonphysical_flagged():
    X, ev = W.square_tri_mesh(2)
    O = orc.Oracle(orc.PROB_EULER2D, 1, X, ev, gamma=GAMMA)
    mu = np.array([2.0, 0.0])
    U = np.tile(orc.freestream(GAMMA, mu), O.Nu // 4)
    Ue, Up, xe = O.gather(U, X.ravel(), 0)
    xe_inv = xe.reshape(3, 2)[[0, 2, 1]].ravel()  # reversed orientation: g < 0
    assert O.element(0, Ue, Up, xe_inv, mu, jac=False)["nonphysical"]
    Ue2 = Ue.copy()
    Ue2[0] = -0.1  # negative density at a node
    assert O.element(0, Ue2, Up, xe, mu, jac=False)["nonphysical"]
    assert not O.element(0, Ue, Up, xe, mu, jac=False)["nonphysical"]
