"""Pins of the oracle's snapshot alignment (Eq. align0): min over (w, x) of
(1/2)|[R(Phi w, x; mu); N(x)]|^2 with the free mesh coordinates unknown.

* a case with a known minimum: the free stream lies in span(Phi), so R(Phi w, x) = 0
  for w = w_inf and any admissible mesh (free-stream preservation), and N(X) = 0;
  from a perturbed start the iteration must drive the objective to zero and w to
  w_inf (the only state in span(Phi) with a zero residual);
* the gradient J^T F it uses is the derivative of (1/2)|F|^2 along random
  directions in (w, x_free) (central differences);
* a generic problem converges to the first-order condition.
"""

import numpy as np

import oracle as orc
from paper_2305_15661_gb300 import workloads as W

GAMMA = 1.4


def interior_mask(X):
    inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    return np.repeat(inner, 2)


def freestream_basis(O, mu, k, seed):
    Uinf = np.tile(orc.freestream(GAMMA, mu), O.Nu // 4)
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(np.concatenate([Uinf[:, None], rng.normal(size=(O.Nu, k - 1))], axis=1))
    if Q[:, 0] @ Uinf < 0:
        Q[:, 0] *= -1
    return Q, Q.T @ Uinf


def test_known_minimum_free_stream():
    n = 3
    X, ev = W.square_tri_mesh(n)
    O = orc.Oracle(orc.PROB_EULER2D, 1, X, ev, gamma=GAMMA, kappa=0.1)
    mu = np.array([2.0, 0.02])
    Phi, w_inf = freestream_basis(O, mu, 4, seed=1)
    mask = interior_mask(X)
    rng = np.random.default_rng(2)
    x0 = X.ravel() + mask * rng.uniform(-0.05, 0.05, size=X.size) / n
    w0 = w_inf + 1e-3 * np.linalg.norm(w_inf) * rng.normal(size=w_inf.size)
    r = O.align(Phi, mu, w0, x0, mask, tol=1e-12, max_iters=60)
    assert r["status"] == 0
    F0 = np.concatenate(O.residual(Phi @ w0, x0, mu)[:2])
    # the state part is exact (w = w_inf, R = 0 on the aligned mesh); the distortion
    # part decays with the tolerance (18 element equations on 8 free coordinates)
    assert r["J"] <= 1e-12 * (0.5 * F0 @ F0)
    R, _, bad = O.residual(Phi @ r["w"], r["x"], mu)
    assert bad == 0 and np.abs(R).max() <= 1e-12
    np.testing.assert_allclose(r["w"], w_inf, rtol=0, atol=1e-12 * np.linalg.norm(w_inf))
    # fixed coordinates stay where they were
    assert np.array_equal(r["x"][~mask], x0[~mask])


def test_gradient_is_derivative_of_objective():
    wl = W.euler_workload(n=3, p=1, k_u=5, k_x=2, seed=4)
    O = orc.Oracle.from_workload(wl, kappa=0.1)
    mu = wl.mus[0]
    mask = interior_mask(wl.X)
    free = np.nonzero(mask)[0]
    w, x = wl.w_eval, wl.X.ravel() + wl.Psi @ wl.tau_eval

    def Jfun(w, x):
        R, N, _ = O.residual(wl.Phi @ w, x, mu)
        return 0.5 * (R @ R + N @ N)

    R, N, _ = O.residual(wl.Phi @ w, x, mu)
    dRdU, dRdx, dNdx = O.jacobian_dense(wl.Phi @ w, x, mu)
    g = np.concatenate([wl.Phi.T @ (dRdU.T @ R), (dRdx.T @ R + dNdx.T @ N)[free]])
    rng = np.random.default_rng(5)
    for _ in range(3):
        d = rng.normal(size=g.size)
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[free] += h * d[wl.ku:]
        xm[free] -= h * d[wl.ku:]
        fd = (Jfun(w + h * d[:wl.ku], xp) - Jfun(w - h * d[:wl.ku], xm)) / (2 * h)
        assert abs(fd - g @ d) <= 1e-6 * max(abs(g @ d), np.linalg.norm(g) * np.linalg.norm(d) * 1e-3)


def test_generic_alignment_reaches_first_order_condition():
    wl = W.euler_workload(n=3, p=1, k_u=5, k_x=2, seed=4)
    O = orc.Oracle.from_workload(wl, kappa=0.1)
    mask = interior_mask(wl.X)
    mu = np.array([2.1, 0.01])
    r = O.align(wl.Phi, mu, wl.w_eval, wl.X.ravel(), mask, tol=1e-8, max_iters=100)
    assert r["status"] == 0
    assert r["gnorm"] <= 1e-8 * max(1.0, r["g0"])
    F0 = np.concatenate(O.residual(wl.Phi @ wl.w_eval, wl.X.ravel(), mu)[:2])
    assert r["J"] < 0.5 * F0 @ F0


def test_mesh_row_damping_by_hand():
    """Two Burgers elements of degree 0 with the interior vertex free (tests/hand_lm.py
    with eps = 1): Oracle.align's accepted steps, lambdas, step lengths and point equal
    the hand-derived LM damped on the mesh row only. Damping the state row instead, or
    swapping the lambda updates, leaves that path by far more than the tolerance."""
    import hand_lm as HL
    phi, mu = np.array([0.8, 1.1]), 1.4
    X, ev = W.interval_mesh(2)
    O = orc.Oracle(orc.PROB_BURGERS1D, 0, X, ev)
    mask = np.array([False, True, False])
    for z0 in [(0.4, 0.0), (1.5, 0.1), (1.9, -0.2)]:
        x0 = X.copy()
        x0[1] = 0.5 + z0[1]
        r = O.align(phi[:, None], np.array([mu]), np.array([z0[0]]), x0, mask, tol=1e-12, max_iters=100,
                    trace=True)
        ref = HL.lm(z0, phi, 1.0, mu, 1e-12)
        tr = r["trace"]
        assert r["status"] == 0 and r["iters"] == len(ref) == tr.shape[0]
        np.testing.assert_array_equal(tr[:, 0], ref[:, 0])
        np.testing.assert_array_equal(tr[:, 1], ref[:, 1])
        np.testing.assert_allclose(tr[:, 2], ref[:, 2], rtol=0, atol=1e-12)
        np.testing.assert_allclose(tr[:, 3], 0.5 + ref[:, 3], rtol=0, atol=1e-12)
        assert r["x"][0] == 0.0 and r["x"][2] == 1.0
        for wrong in (dict(damp="w"), dict(schedule="inverted")):
            alt = HL.lm(z0, phi, 1.0, mu, 1e-12, **wrong)
            n = min(len(alt), len(ref))
            assert len(alt) != len(ref) or np.abs(alt[:n, 2:] - ref[:n, 2:]).max() > 1e-6, wrong
