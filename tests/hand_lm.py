"""A two-unknown Levenberg-Marquardt problem written out by hand (Sec. 3.2.3).

The problem is steady 1-D Burgers, u u_x = s(x; mu) with s = 0.5 e^{mu x}, on two
elements of degree 0 over [0, 1] with the interior vertex at x_1. With one state
value per element (u_1, u_2 > 0, so the Roe flux upwinds exactly: the interface
flux is f(u_1) = u_1^2/2, the inflow flux f(1) = 1/2, the outflow flux f(u_2)),
the element residuals are, for the 2-point Gauss rule Q[a, b] of the source,

    R_1 = u_1^2/2 - 1/2 - Q[0, x_1],     R_2 = u_2^2/2 - u_1^2/2 - Q[x_1, 1].

The tests use it twice:
* reduced (Eq. lmstep): U = phi w with phi a 2-vector, x_1 = 1/2 + eps tau; the
  unknowns (w, tau) are damped on the tau block only (Eq. levmarq-step);
* alignment (Eq. align0): the same residual with x_1 itself the free unknown
  (eps = 1, x_1 = 1/2 + tau), damped on the mesh row.

Everything here is derived in closed form from the two formulas above; nothing
calls the oracle.
"""

import numpy as np

EPS = np.finfo(float).eps
_gx, _gw = np.polynomial.legendre.leggauss(2)
XI, WQ = 0.5 * (1.0 + _gx), 0.5 * _gw


def source_rule(a, b, mu):
    """2-point Gauss rule for the integral of 0.5 e^{mu x} over [a, b]."""
    return float(np.sum(WQ * (b - a) * 0.5 * np.exp(mu * (a + (b - a) * XI))))


def source_rule_grad(a, b, mu):
    """(d/da, d/db) of source_rule."""
    e = 0.5 * np.exp(mu * (a + (b - a) * XI))
    da = float(np.sum(WQ * (-e + (b - a) * e * mu * (1.0 - XI))))
    db = float(np.sum(WQ * (e + (b - a) * e * mu * XI)))
    return da, db


def model(z, phi, eps, mu):
    """Residual (2,) and Jacobian (2 x 2) in the unknowns z = (w, tau)."""
    w, t = z
    x1 = 0.5 + eps * t
    u1, u2 = phi[0] * w, phi[1] * w
    assert u1 > 0 and u2 > 0 and 0.0 < x1 < 1.0, (u1, u2, x1)
    R = np.array([u1 * u1 / 2 - 0.5 - source_rule(0.0, x1, mu),
                  u2 * u2 / 2 - u1 * u1 / 2 - source_rule(x1, 1.0, mu)])
    _, db1 = source_rule_grad(0.0, x1, mu)
    da2, _ = source_rule_grad(x1, 1.0, mu)
    Jw = np.array([u1 * phi[0], u2 * phi[1] - u1 * phi[0]])
    Jt = -eps * np.array([db1, da2])
    return R, np.stack([Jw, Jt], axis=1)


def lm(z0, phi, eps, mu, tol, damp="tau", schedule="reading", max_iters=100):
    """The LM iteration with this build's readings of the open constants:
    lambda_0 = 1e-4; lambda/10 (>= 1e-12) after a full step, 10 lambda (<= 1e8)
    after a shortened one; Armijo backtracking with c1 = 1e-4 plus 16 ulp of |J|,
    alpha in {1, 1/2, ...}, at most 30 halvings; stop when |g| <= tol max(1, |g_0|).

    damp = "tau" puts lambda on the second unknown (Eq. levmarq-step), "w" on the
    first; schedule = "inverted" swaps the two lambda updates. The two wrong
    variants exist so that the tests can show the comparison tells them apart.
    Returns rows [lambda used, alpha, w, tau] per accepted step."""
    z = np.array(z0, dtype=np.float64)
    lam = 1e-4
    rows = []
    R, Jm = model(z, phi, eps, mu)
    J = 0.5 * R @ R
    g = Jm.T @ R
    thresh = tol * max(1.0, float(np.linalg.norm(g)))
    D = np.diag([0.0, 1.0]) if damp == "tau" else np.diag([1.0, 0.0])
    while np.linalg.norm(g) > thresh and len(rows) < max_iters:
        d = np.linalg.solve(Jm.T @ Jm + lam * D, -g)
        slope = g @ d
        alpha = 1.0
        for h in range(31):
            zt = z + alpha * d
            Rt, _ = model(zt, phi, eps, mu)
            if 0.5 * Rt @ Rt <= J + 1e-4 * alpha * slope + 16 * EPS * abs(J):
                break
            alpha *= 0.5
        else:
            raise RuntimeError("line search failed")
        rows.append([lam, alpha, zt[0], zt[1]])
        full = (h == 0) if schedule == "reading" else (h != 0)
        lam = max(lam / 10, 1e-12) if full else min(lam * 10, 1e8)
        z = zt
        R, Jm = model(z, phi, eps, mu)
        J = 0.5 * R @ R
        g = Jm.T @ R
    return np.array(rows)
