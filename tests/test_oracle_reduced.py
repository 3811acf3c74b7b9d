"""Pins of the oracle's weighted reduced residuals, Gauss-Newton blocks and objective.

* App. A: with rho = 1 (Remark rom-eqp-ones) and for sparse rho, the elemental
  sums equal the same quantities formed from the globally assembled residual,
  Jacobians and distortion (Eqs. ift-res, hdm_elem_jac1, hdm_elem_jac2):
  S = Phi^T dR/dU^T W R, T = Psi^T (dR/dx^T W R + dN/dx^T W_e N),
  H = [dR/dU Phi, dR/dx Psi]^T W [..] + the distortion block, J = (R^T W R + N^T W_e N)/2.
* first-order optimality identity (App. A): [S; T] is the gradient of J, checked
  by central differences along random directions;
* the weighted quantities are linear in rho.
"""

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import workloads as W

GAMMA = 1.4


def small_euler(n=3, p=2, ku=6, kx=3, seed=4, kappa=0.1):
    wl = W.euler_workload(n=n, p=p, k_u=ku, k_x=kx, seed=seed)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    return wl, O


def global_route(O, wl, w, tau, mu, rho_e):
    U = wl.Phi @ w
    x = wl.X.ravel() + wl.Psi @ tau
    R, N, bad = O.residual(U, x, mu)
    assert bad == 0
    dRdU, dRdx, dNdx = O.jacobian_dense(U, x, mu)
    Wd = np.repeat(rho_e, O.nu)  # rho_e on every DOF of element e
    A = np.concatenate([dRdU @ wl.Phi, dRdx @ wl.Psi], axis=1)
    B = np.concatenate([np.zeros((O.n_elems, wl.ku)), dNdx @ wl.Psi], axis=1)
    S = wl.Phi.T @ (dRdU.T @ (Wd * R))
    T = wl.Psi.T @ (dRdx.T @ (Wd * R) + dNdx.T @ (rho_e * N))
    H = A.T @ (Wd[:, None] * A) + B.T @ (rho_e[:, None] * B)
    J = 0.5 * (R @ (Wd * R) + N @ (rho_e * N))
    return S, T, H, J


@pytest.mark.parametrize("sparse", [False, True])
def test_elemental_equals_global_euler(sparse):
    wl, O = small_euler()
    mu = wl.mus[0]
    w, tau = wl.w_eval, wl.tau_eval
    if sparse:
        rng = np.random.default_rng(0)
        elems = np.sort(rng.choice(O.n_elems, 7, replace=False)).astype(np.int32)
        rho = rng.uniform(0.5, 50, 7)
        rho_e = np.zeros(O.n_elems)
        rho_e[elems] = rho
        rs = (elems, rho)
    else:
        rho_e = np.ones(O.n_elems)
        rs = None
    r = O.reduced(wl.Phi, wl.Psi, w, tau, mu, rho_set=rs)
    S, T, H, J = global_route(O, wl, w, tau, mu, rho_e)
    np.testing.assert_allclose(r["S"], S, rtol=1e-12, atol=1e-12 * np.abs(S).max())
    np.testing.assert_allclose(r["T"], T, rtol=1e-12, atol=1e-12 * np.abs(T).max())
    np.testing.assert_allclose(r["H"], H, rtol=1e-12, atol=1e-12 * np.abs(H).max())
    assert abs(r["J"] - J) <= 1e-13 * J


def test_elemental_equals_global_burgers():
    wl = W.burgers_workload(n_elems=12, p=2, k_u=4)
    O = orc.Oracle.from_workload(wl)
    mu = wl.mus[0]
    w = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess) + 0.1 * wl.w_eval
    r = O.reduced(wl.Phi, wl.Psi, w, wl.tau_eval, mu)
    S, T, H, J = global_route(O, wl, w, wl.tau_eval, mu, np.ones(O.n_elems))
    np.testing.assert_allclose(r["S"], S, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(r["T"], T, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(r["H"], H, rtol=1e-12, atol=1e-13)
    assert abs(r["J"] - J) <= 1e-13 * J


@pytest.mark.parametrize("prob", ["euler", "burgers"])
def test_gradient_is_derivative_of_objective(prob):
    if prob == "euler":
        wl, O = small_euler()
        rng = np.random.default_rng(1)
        elems = np.sort(rng.choice(O.n_elems, 9, replace=False)).astype(np.int32)
        rs = (elems, rng.uniform(0.5, 50, 9))
        w, tau = wl.w_eval, wl.tau_eval
    else:
        wl = W.burgers_workload(n_elems=20, p=2, k_u=5)
        O = orc.Oracle.from_workload(wl)
        rs = None
        w = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess) + 0.1 * wl.w_eval
        tau = wl.tau_eval
    mu = wl.mus[0]
    r = O.reduced(wl.Phi, wl.Psi, w, tau, mu, rho_set=rs)
    g = np.concatenate([r["S"], r["T"]])
    rng = np.random.default_rng(2)
    for _ in range(4):
        d = rng.normal(size=wl.ku + wl.kx)
        d /= np.linalg.norm(d)
        h = 1e-6 * max(1.0, np.linalg.norm(np.concatenate([w, tau])))
        Jp, _ = O.objective(wl.Phi, wl.Psi, w + h * d[:wl.ku], tau + h * d[wl.ku:], mu, rho_set=rs)
        Jm, _ = O.objective(wl.Phi, wl.Psi, w - h * d[:wl.ku], tau - h * d[wl.ku:], mu, rho_set=rs)
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g @ d) <= 1e-7 * np.linalg.norm(g) + 1e-12, (fd, g @ d)


def test_linear_in_rho():
    wl, O = small_euler()
    mu = wl.mus[0]
    rng = np.random.default_rng(3)
    elems = np.arange(O.n_elems, dtype=np.int32)
    r1 = rng.uniform(0, 2, O.n_elems)
    r2 = rng.uniform(0, 2, O.n_elems)
    a = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, mu, rho_set=(elems, r1))
    b = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, mu, rho_set=(elems, r2))
    c = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, mu, rho_set=(elems, r1 + 2 * r2))
    for key in ("S", "T", "H"):
        np.testing.assert_allclose(c[key], a[key] + 2 * b[key], rtol=1e-13, atol=1e-13 * np.abs(c[key]).max())
    assert abs(c["J"] - (a["J"] + 2 * b["J"])) <= 1e-13 * c["J"]


def test_dense_rho_one_equals_explicit_list():
    wl, O = small_euler()
    mu = wl.mus[0]
    a = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, mu)
    elems = np.arange(O.n_elems, dtype=np.int32)
    b = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, mu, rho_set=(elems, np.ones(O.n_elems)))
    for key in ("S", "T", "H"):
        np.testing.assert_array_equal(a[key], b[key])
    assert a["J"] == b["J"]


def test_threads_do_not_change_result():
    wl, O = small_euler(n=6)
    mu = wl.mus[0]
    a = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, mu, nthreads=1)
    b = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, mu, nthreads=4)
    for key in ("S", "T", "H"):
        np.testing.assert_array_equal(a[key], b[key])
