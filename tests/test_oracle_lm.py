"""Pins of the oracle's Levenberg-Marquardt solver (Sec. 3.2.3, Remark rem:solver).

* one Burgers element of degree 0 with a 1 x 1 basis: the residual is the
  closed form u^2/2 - 1/2 - Q[s], so the Gauss-Newton iteration with the
  line-search reading is written out here by hand and must match the oracle's
  iterates, iteration count and final point;
* two Burgers elements of degree 0 with one state and one mesh unknown: the
  damped step (H + diag(0, lambda)) dz = -g of Eqs. lmstep and levmarq-step and
  the lambda schedule (lambda_0 = 1e-4, lambda/10 after a full step, 10 lambda
  after a shortened one) are written out by hand (tests/hand_lm.py) and must give
  the oracle's steps, lambdas, step lengths and point;
* on the Burgers and Euler workloads: convergence to the optimality tolerance,
  monotone decrease of J, symmetric positive definite H at the solution, and the
  tau = 0 initialisation;
* a zero column of Phi (an exactly singular w block): every factorisation takes
  one diagonal shift, and the solve matches the one without that column.
"""

import math

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import workloads as W

EPS = np.finfo(float).eps


def scalar_gn(phi, src, w0, tol, max_iters=100):
    """Hand-written scalar Gauss-Newton with the solver's line-search reading."""
    R = lambda w: 0.5 * (phi * w) ** 2 - 0.5 - src
    dR = lambda w: phi * phi * w
    J = lambda w: 0.5 * R(w) ** 2

    def phase(w):
        g0 = abs(dR(w) * R(w))
        thresh = tol * max(1.0, g0)
        it = 0
        while abs(dR(w) * R(w)) > thresh and it < max_iters:
            g = dR(w) * R(w)
            d = -g / dR(w) ** 2
            slope = g * d
            a = 1.0
            for _ in range(31):
                wt = w + a * d
                if J(wt) <= J(w) + 1e-4 * a * slope + 16 * EPS * abs(J(w)):
                    break
                a *= 0.5
            w = wt
            it += 1
        return w, it

    w, it0 = phase(w0)
    w, it1 = phase(w)
    return w, it0, it1


@pytest.mark.parametrize("phi,mu", [(0.8, 1.0), (1.3, 1.7), (0.5, 2.0)])
def test_scalar_gauss_newton_by_hand(phi, mu):
    X, ev = W.interval_mesh(1)
    O = orc.Oracle(orc.PROB_BURGERS1D, 0, X, ev)
    gx, gw = np.polynomial.legendre.leggauss(2)
    src = np.sum(0.5 * gw * 0.5 * np.exp(mu * 0.5 * (1 + gx)))
    Phi = np.array([[phi]])
    Psi = np.zeros((2, 0))
    w0 = phi * 1.0  # Phi^T U_guess with U_guess = 1
    res = O.solve(Phi, Psi, np.array([mu]), np.array([w0]), tol=1e-12)
    w_ref, it0, it1 = scalar_gn(phi, src, w0, 1e-12)
    assert res["status"] == 0
    assert res["init_iters"] == it0 and res["iters"] == it1
    assert abs(res["w"][0] - w_ref) <= 1e-14 * abs(w_ref)
    # the converged state is the exact outflow value of the quadrature-integrated source
    assert abs((phi * res["w"][0]) ** 2 / 2 - 0.5 - src) < 1e-12


def _check_solution(O, wl, res, mu, tol, rho_set=None):
    assert res["status"] == 0, res
    g = math.hypot(res["normS"], res["normT"])
    assert g <= tol * max(1.0, res["g0"])
    h = res["hist"]
    assert np.all(np.diff(h) <= 16 * EPS * np.abs(h[:-1])), np.diff(h)
    r = O.reduced(wl.Phi, wl.Psi, res["w"], res["tau"], mu, rho_set=rho_set)
    assert abs(r["J"] - res["J"]) <= 1e-14 * res["J"]
    ev = np.linalg.eigvalsh(r["H"])
    assert ev.min() > 0.0
    np.testing.assert_allclose(r["H"], r["H"].T, rtol=0, atol=1e-14 * np.abs(r["H"]).max())


def test_burgers_workload_converges():
    wl = W.burgers_workload()
    O = orc.Oracle.from_workload(wl)
    mu = wl.mus[0]
    wg = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess)
    res = O.solve(wl.Phi, wl.Psi, mu, wg, tol=1e-10)
    _check_solution(O, wl, res, mu, 1e-10)
    assert res["init_iters"] > 0 and res["iters"] > 0


def test_euler_small_workload_converges_sparse_rho():
    wl = W.euler_workload(n=8, p=2, k_u=8, k_x=4, seed=6)
    O = orc.Oracle.from_workload(wl)
    sets = W.eq_weight_sets(wl, 1, seed=7, lo=20, hi=40)
    mu = wl.mus[0]
    wg = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess)
    res = O.solve(wl.Phi, wl.Psi, mu, wg, rho_set=sets[0], tol=1e-8)
    _check_solution(O, wl, res, mu, 1e-8, rho_set=sets[0])


def test_init_phase_is_the_tau_free_solve():
    # the initialisation of Remark rem:solver is LM over w with tau = 0: a solve with an
    # empty mesh basis runs exactly that iteration, so the J histories coincide over it
    wl = W.burgers_workload(n_elems=40)
    O = orc.Oracle.from_workload(wl)
    mu = wl.mus[0]
    wg = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess)
    full = O.solve(wl.Phi, wl.Psi, mu, wg, tol=1e-10)
    free = O.solve(wl.Phi, np.zeros((wl.Psi.shape[0], 0)), mu, wg, tol=1e-10)
    assert free["status"] == 0 and free["iters"] == 0
    assert full["init_iters"] == free["init_iters"] > 0
    n = full["init_iters"] + 1
    np.testing.assert_array_equal(full["hist"][:n], free["hist"][:n])
    assert full["J"] <= free["J"]


def test_given_start_skips_init():
    wl = W.burgers_workload(n_elems=40)
    O = orc.Oracle.from_workload(wl)
    mu = wl.mus[0]
    wg = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess)
    full = O.solve(wl.Phi, wl.Psi, mu, wg, tol=1e-10)
    warm = O.solve(wl.Phi, wl.Psi, mu, full["w"], tau0=full["tau"], do_init=False, tol=1e-10)
    assert warm["init_iters"] == 0
    assert warm["iters"] <= 1
    np.testing.assert_allclose(warm["w"], full["w"], rtol=1e-9)


# -- damping placement and lambda schedule (Eqs. levmarq-step and lmstep) -----------

@pytest.mark.parametrize("z0", [(0.4, 0.0), (1.5, 3.0), (0.9, -4.0)])
def test_damped_two_unknown_step_by_hand(z0):
    """Two Burgers elements of degree 0, one state and one mesh unknown (tests/hand_lm.py):
    the oracle's accepted steps, the lambda each used, the step lengths and the final
    point equal the hand-derived LM. The start (0.4, 0) needs a halved first step, so
    both lambda updates are taken. The same hand iteration with the damping moved to the
    w block, or with the two lambda updates swapped, leaves the oracle's path by far more
    than the tolerance, so either mistake in the oracle would fail here."""
    import hand_lm as HL
    phi, eps, mu = np.array([0.8, 1.1]), 0.02, 1.4
    X, ev = W.interval_mesh(2)
    O = orc.Oracle(orc.PROB_BURGERS1D, 0, X, ev)
    Phi = phi[:, None]
    Psi = np.array([[0.0], [eps], [0.0]])  # one mode moving the interior vertex
    res = O.solve(Phi, Psi, np.array([mu]), np.array([z0[0]]), tau0=np.array([z0[1]]), do_init=False,
                  tol=1e-12, trace=True)
    ref = HL.lm(z0, phi, eps, mu, 1e-12)
    tr = res["trace"]
    assert res["status"] == 0 and res["iters"] == len(ref) == tr.shape[0]
    assert np.all(tr[:, 0] == 1.0)
    np.testing.assert_array_equal(tr[:, 1], ref[:, 0])  # lambda: exact powers of ten
    np.testing.assert_array_equal(tr[:, 2], ref[:, 1])  # alpha: exact powers of two
    np.testing.assert_allclose(tr[:, 3:], ref[:, 2:], rtol=0, atol=1e-12)
    if z0 == (0.4, 0.0):
        assert ref[0, 1] < 1.0 and ref[1, 0] == 1e-3 and ref[2, 0] == 1e-4
    for wrong in (dict(damp="w"), dict(schedule="inverted")):
        alt = HL.lm(z0, phi, eps, mu, 1e-12, **wrong)
        n = min(len(alt), len(ref))
        assert len(alt) != len(ref) or np.abs(alt[:n, 2:] - ref[:n, 2:]).max() > 1e-3, wrong


def test_zero_basis_column_takes_the_shifted_factorisation():
    # A zero column of Phi gives H a zero row and column, so every factorisation of
    # the w block meets a zero pivot and is retried with the diagonal shift
    # 1e-14 tr(M)/k (times 10 per further retry). That shift is far below the other
    # pivots, so one retry succeeds, the zero column's coefficient stays exactly 0,
    # and the solve takes the same steps to the same optimum as the problem without
    # that column.
    wl = W.euler_workload(n=8, p=2, k_u=8, k_x=4, seed=6)
    mu = wl.mus[0]
    U0 = W.replicate_guess(wl, wl.U_guess)
    O = orc.Oracle.from_workload(wl)
    Pz = wl.Phi.copy()
    Pz[:, -1] = 0.0
    rz = O.solve(Pz, wl.Psi, mu, Pz.T @ U0, tol=1e-8)
    P7 = np.ascontiguousarray(wl.Phi[:, :-1])
    r7 = O.solve(P7, wl.Psi, mu, P7.T @ U0, tol=1e-8)
    assert rz["status"] == 0 and r7["status"] == 0
    assert r7["shifts"] == 0
    assert rz["shifts"] == rz["init_iters"] + rz["iters"] > 0  # one retry per factorisation
    assert (rz["init_iters"], rz["iters"]) == (r7["init_iters"], r7["iters"])
    assert rz["w"][-1] == 0.0
    z = np.concatenate([rz["w"][:-1], rz["tau"]])
    z7 = np.concatenate([r7["w"], r7["tau"]])
    assert np.linalg.norm(z - z7) <= 1e-10 * np.linalg.norm(z7)
    assert abs(rz["J"] - r7["J"]) <= 1e-12 * r7["J"]
