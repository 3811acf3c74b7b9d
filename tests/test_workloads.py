"""Seeded input generators: determinism and the shapes and structure the workloads promise."""

import numpy as np

from paper_2305_15661_gb300 import workloads as W


def test_splitmix64_known_values():
    # splitmix64 from state 0: the first output of the reference generator is 0xE220A8397B1DCDAF
    z = W._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))[0]
    assert int(z) == 0xE220A8397B1DCDAF


def test_generators_are_deterministic_and_seeded():
    a = W.normal(3, 1, 1000)
    b = W.normal(3, 1, 1000)
    c = W.normal(4, 1, 1000)
    np.testing.assert_array_equal(a, b)
    assert np.abs(a - c).max() > 0.1
    assert abs(a.mean()) < 0.1 and abs(a.std() - 1.0) < 0.1
    u = W.uniform(3, 2, 10000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.02


def test_burgers_workload_shapes():
    wl = W.burgers_workload()
    assert wl.Phi.shape == (600, 5) and wl.Psi.shape == (201, 2)
    np.testing.assert_allclose(wl.Phi.T @ wl.Phi, np.eye(5), atol=1e-13)
    assert abs(wl.Psi[0]).max() < 1e-15 and abs(wl.Psi[-1]).max() < 1e-12
    assert 1.0 <= wl.mus[0, 0] <= 2.0
    assert np.all(np.abs(wl.tau_eval) <= 0.1 / 200)


def test_euler_workload_structure():
    wl = W.euler_workload(n=10, p=2, k_u=6, k_x=4)
    assert wl.ev.shape == (200, 3) and wl.X.shape == (121, 2)
    assert np.all(W.triangle_areas(wl.X, wl.ev) > 0)
    np.testing.assert_allclose(wl.Phi.T @ wl.Phi, np.eye(6), atol=1e-12)
    np.testing.assert_allclose(wl.Psi.T @ wl.Psi, np.eye(4), atol=1e-12)
    # first state column is the perturbed free stream, with positive sign
    assert np.all(wl.Phi[0::4, 0] > 0)
    # mesh modes vanish on the boundary
    bnd = np.any((wl.X < 1e-12) | (wl.X > 1 - 1e-12), axis=1)
    assert np.abs(wl.Psi.reshape(-1, 2, 4)[bnd]).max() < 1e-12
    xd = wl.X + (wl.Psi @ wl.tau_eval).reshape(-1, 2)
    assert np.min(W.triangle_areas(xd, wl.ev) / W.triangle_areas(wl.X, wl.ev)) > 0.5


def test_weight_sets():
    wl = W.euler_workload(n=20, p=1, k_u=3, k_x=2)
    sets = W.eq_weight_sets(wl, 16, seed=3, lo=50, hi=400)
    bnd = W.boundary_elements(wl.X, wl.ev)
    for elems, rho in sets:
        assert 50 <= len(elems) <= 400
        assert np.all(np.diff(elems) > 0)
        assert np.all((rho >= 0.5) & (rho <= 50))
        for side in bnd:
            assert np.intersect1d(side, elems).size >= 1
