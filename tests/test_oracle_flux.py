"""Pins of the oracle's physical flux and Roe numerical flux.

The Euler flux is Eq. euler (Sec. 4.2). The paper names no numerical flux; the
reading here is the Roe flux with Roe averages weighted by sqrt(rho), waves
v_n - c, v_n, v_n + c, and Harten's entropy fix |lam| -> (lam^2 + delta^2) /
(2 delta) below delta = 0.1 c~ (Burgers: upwinding on a = (u+ + u-)/2 with
delta = 0.05 (|u+| + |u-|) |n|). Pins: closed-form values,
consistency H(U, U, n) = f(U).n, the Roe property through exact upwinding
(supersonic normal flow, isolated contact and shear waves), conservation,
rotational invariance and homogeneity in the scaled normal.
"""

import math

import numpy as np
import pytest

import oracle as orc

GAMMA = 1.4


def prim_to_cons(rho, u, v, P, gamma=GAMMA):
    return np.array([rho, rho * u, rho * v, P / (gamma - 1) + 0.5 * rho * (u * u + v * v)])


def flux_closed_form(rho, u, v, P, gamma=GAMMA):
    E = P / (gamma - 1) + 0.5 * rho * (u * u + v * v)
    fx = [rho * u, rho * u * u + P, rho * u * v, u * (E + P)]
    fy = [rho * v, rho * u * v, rho * v * v + P, v * (E + P)]
    return np.stack([fx, fy], axis=1)


def test_euler_flux_closed_form():
    for (rho, u, v, P) in [(1.0, 2.0, 0.3, 1.0), (0.7, -0.4, 1.1, 2.5), (1.3, 0.0, 0.0, 0.8)]:
        f, Pc = orc.euler_flux(GAMMA, prim_to_cons(rho, u, v, P))
        np.testing.assert_allclose(f, flux_closed_form(rho, u, v, P), rtol=1e-14, atol=1e-14)
        assert abs(Pc - P) < 1e-13


def test_freestream_state():
    U = orc.freestream(GAMMA, np.array([2.0, 0.1]))
    c = math.sqrt(GAMMA)
    np.testing.assert_allclose(U, prim_to_cons(1.0, 2 * c * math.cos(0.1), 2 * c * math.sin(0.1), 1.0), rtol=1e-15)


def _fn(U, n):
    f, _ = orc.euler_flux(GAMMA, U)
    return f @ n


def test_roe_consistency_and_homogeneity():
    rng = np.random.default_rng(1)
    for _ in range(20):
        U = prim_to_cons(rng.uniform(0.5, 2), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.5, 2))
        n = rng.normal(size=2)
        np.testing.assert_allclose(orc.euler_roe(GAMMA, U, U, n), _fn(U, n), rtol=1e-13, atol=1e-13)
        U2 = prim_to_cons(rng.uniform(0.5, 2), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.5, 2))
        H1 = orc.euler_roe(GAMMA, U, U2, n)
        np.testing.assert_allclose(orc.euler_roe(GAMMA, U, U2, 3.7 * n), 3.7 * H1, rtol=1e-13, atol=1e-13)


def test_roe_supersonic_upwinding():
    # normal velocity above the sound speed on both sides: every wave moves outward,
    # so the Roe flux equals the interior normal flux exactly (and the exterior one
    # for flow entering through the face)
    rng = np.random.default_rng(2)
    for _ in range(20):
        th = rng.uniform(0, 2 * math.pi)
        n = np.array([math.cos(th), math.sin(th)]) * rng.uniform(0.2, 3)
        nh = n / np.linalg.norm(n)
        t = np.array([-nh[1], nh[0]])
        rho1, rho2 = rng.uniform(0.5, 1.5, 2)
        P1, P2 = rng.uniform(0.5, 1.5, 2)
        vn1, vn2 = rng.uniform(3.0, 4.0, 2)
        vt1, vt2 = rng.uniform(-1, 1, 2)
        v1 = vn1 * nh + vt1 * t
        v2 = vn2 * nh + vt2 * t
        Up = prim_to_cons(rho1, *v1, P1)
        Um = prim_to_cons(rho2, *v2, P2)
        np.testing.assert_allclose(orc.euler_roe(GAMMA, Up, Um, n), _fn(Up, n), rtol=1e-12, atol=1e-12)
        Up2 = prim_to_cons(rho1, *(-v1), P1)
        Um2 = prim_to_cons(rho2, *(-v2), P2)
        np.testing.assert_allclose(orc.euler_roe(GAMMA, Up2, Um2, n), _fn(Um2, n), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_roe_resolves_contact_and_shear_waves(sign):
    # a jump in density only (contact) or in tangential velocity only (shear) is an
    # eigenvector of the Roe matrix with eigenvalue v_n, so the flux is the upwind one
    n = np.array([0.6, 0.8]) * 1.7
    nh = n / np.linalg.norm(n)
    t = np.array([-nh[1], nh[0]])
    vn = sign * 0.4  # subsonic
    v = vn * nh + 0.3 * t
    Up = prim_to_cons(1.0, *v, 1.0)
    Um = prim_to_cons(1.6, *v, 1.0)
    up = Up if sign > 0 else Um
    np.testing.assert_allclose(orc.euler_roe(GAMMA, Up, Um, n), _fn(up, n), rtol=1e-12, atol=1e-12)
    v2 = vn * nh - 0.5 * t
    Um = prim_to_cons(1.0, *v2, 1.0)
    up = Up if sign > 0 else Um
    np.testing.assert_allclose(orc.euler_roe(GAMMA, Up, Um, n), _fn(up, n), rtol=1e-12, atol=1e-12)


def test_roe_conservation_and_rotation():
    rng = np.random.default_rng(3)
    for _ in range(20):
        Up = prim_to_cons(rng.uniform(0.5, 2), *rng.uniform(-2, 2, 2), rng.uniform(0.5, 2))
        Um = prim_to_cons(rng.uniform(0.5, 2), *rng.uniform(-2, 2, 2), rng.uniform(0.5, 2))
        n = rng.normal(size=2)
        H = orc.euler_roe(GAMMA, Up, Um, n)
        np.testing.assert_allclose(orc.euler_roe(GAMMA, Um, Up, -n), -H, rtol=1e-12, atol=1e-12)
        th = rng.uniform(0, 2 * math.pi)
        Rm = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])

        def rot(U):
            return np.array([U[0], *(Rm @ U[1:3]), U[3]])

        Hr = orc.euler_roe(GAMMA, rot(Up), rot(Um), Rm @ n)
        np.testing.assert_allclose(Hr, rot(H), rtol=1e-12, atol=1e-12)


def test_roe_subsonic_not_central():
    # for a subsonic acoustic jump the dissipation is non-zero: |A| differs from A
    n = np.array([1.0, 0.0])
    Up = prim_to_cons(1.0, 0.2, 0.0, 1.0)
    Um = prim_to_cons(1.0, 0.2, 0.0, 1.3)
    H = orc.euler_roe(GAMMA, Up, Um, n)
    central = 0.5 * (_fn(Up, n) + _fn(Um, n))
    assert np.linalg.norm(H - central) > 1e-3


def test_burgers_roe_upwind():
    f = lambda u: 0.5 * u * u
    for up, um in [(1.0, 2.0), (0.3, 1.7), (2.0, 0.5)]:
        assert abs(orc.burgers_roe(up, um, 1.0) - f(up)) < 1e-15      # flow to +x leaves through n=+1
        assert abs(orc.burgers_roe(up, um, -1.0) + f(um)) < 1e-15     # and enters through n=-1
        assert abs(orc.burgers_roe(-up, -um, 1.0) - f(um)) < 1e-15    # reversed flow takes the exterior state
    # consistency and conservation
    assert abs(orc.burgers_roe(0.7, 0.7, 1.0) - f(0.7)) < 1e-15
    assert abs(orc.burgers_roe(0.7, -0.2, 1.0) + orc.burgers_roe(-0.2, 0.7, -1.0)) < 1e-15


def _one_sided_slopes(fun, s0, h=1e-6):
    left = (fun(s0) - fun(s0 - h)) / h
    right = (fun(s0 + h) - fun(s0)) / h
    return left, right


def test_roe_entropy_fix_makes_flux_c1_at_sonic_faces():
    # the acoustic wave speed v_n - c of the Roe state passes through the fix threshold
    # along this path; without a fix the flux has a kink where the speed changes sign
    n = np.array([1.0, 0.0])
    Um = prim_to_cons(1.1, 1.2, 0.1, 1.05)

    def roe_speed_minus(s):
        Up = prim_to_cons(1.0, s, 0.0, 1.0)
        rl, rr = math.sqrt(1.0), math.sqrt(1.1)
        u = (rl * s + rr * 1.2) / (rl + rr)
        v = (rr * 0.1) / (rl + rr)
        hl = (1.0 / 0.4 + 0.5 * s * s + 1.0) / 1.0
        hr = (1.05 / 0.4 + 0.5 * 1.1 * (1.44 + 0.01) + 1.05) / 1.1
        hh = (rl * hl + rr * hr) / (rl + rr)
        c = math.sqrt(0.4 * (hh - 0.5 * (u * u + v * v)))
        return u - c, c

    # locate the two switch points |v_n - c| = 0.1 c by bisection on s, and a zero crossing
    import scipy.optimize as so
    f_plus = lambda s: roe_speed_minus(s)[0] - 0.1 * roe_speed_minus(s)[1]
    f_minus = lambda s: roe_speed_minus(s)[0] + 0.1 * roe_speed_minus(s)[1]
    f_zero = lambda s: roe_speed_minus(s)[0]
    for f in (f_plus, f_minus, f_zero):
        s0 = so.brentq(f, 0.0, 3.0, xtol=1e-14)
        for comp in range(4):
            H = lambda s: orc.euler_roe(GAMMA, prim_to_cons(1.0, s, 0.0, 1.0), Um, n)[comp]
            left, right = _one_sided_slopes(H, s0)
            assert abs(left - right) <= 1e-4 * max(1.0, abs(left)), (comp, left, right)


def test_burgers_entropy_fix_c1():
    # Roe speed a = (u+ + u-)/2 crosses zero along u+ -> path with u- = -0.8
    for s0 in (0.8, 0.8 * 1.1 / 0.9, 0.8 * 0.9 / 1.1):  # a = 0 and the two switch points |a| = delta
        left, right = _one_sided_slopes(lambda s: orc.burgers_roe(s, -0.8, 1.0), s0)
        assert abs(left - right) <= 1e-4, (s0, left, right)
    # away from the switch the flux is the unmodified Roe flux (exact upwinding)
    assert abs(orc.burgers_roe(1.0, 2.0, 1.0) - 0.5) < 1e-15
