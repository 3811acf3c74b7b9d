"""The greedy-search indicator (Eq. greedy0): the full HDM residual norm at many
(mu, w, tau) points through the C ABI, against the oracle's globally assembled
residual."""

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _oracle_norm(O, wl, mu, w, tau):
    U = wl.Phi @ w
    x = (wl.X.reshape(-1) + wl.Psi @ tau) if wl.kx else wl.X.reshape(-1)
    R, _, bad = O.residual(U, x, mu)
    return np.inf if bad else float(np.linalg.norm(R))


def _points(wl, n, seed):
    rng = np.random.default_rng(seed)
    ys = np.stack([wl.w_eval * (1 + 1e-3 * rng.normal(size=wl.ku)) for _ in range(n)])
    zs = np.stack([wl.tau_eval * rng.uniform(0.2, 1.2) for _ in range(n)])
    return ys, zs


@pytest.mark.parametrize("p,kappa", [(1, 0.0), (2, 0.1), (3, 0.0)])
def test_euler_norms_match_oracle(p, kappa):
    # 2 * 11^2 = 242 elements: several 64-element chunks and a ragged last one;
    # kappa != 0 checks that the distortion term stays out of the HDM residual
    wl = W.euler_workload(n=11, p=p, k_u=9, k_x=4, seed=31, n_mu=5, mu_box=True)
    ys, zs = _points(wl, 5, 1)
    ctx = ift.Context.from_workload(wl, kappa=kappa)
    g = ctx.hdm_residual_norms(wl.mus, ys, zs)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    for q in range(5):
        r = _oracle_norm(O, wl, wl.mus[q], ys[q], zs[q])
        assert abs(g[q] - r) <= 1e-12 * r, (q, g[q], r)


def test_burgers_norms_match_oracle():
    wl = W.burgers_workload(n_elems=200, p=2, k_u=5, seed=1, n_mu=3)
    ys = np.stack([wl.w_eval * s for s in (1.0, 0.9, 1.1)])
    zs = np.stack([wl.tau_eval * s for s in (1.0, 0.5, -0.5)])
    ctx = ift.Context.from_workload(wl)
    g = ctx.hdm_residual_norms(wl.mus.reshape(-1, 1), ys, zs)
    O = orc.Oracle.from_workload(wl)
    for q in range(3):
        r = _oracle_norm(O, wl, wl.mus[q], ys[q], zs[q])
        assert abs(g[q] - r) <= 1e-12 * r


def test_fp32_norms():
    wl = W.euler_workload(n=16, p=2, k_u=12, k_x=4, seed=32, n_mu=4, mu_box=True)
    ys, zs = _points(wl, 4, 2)
    g = ift.Context.from_workload(wl, precision=ift.FP32).hdm_residual_norms(wl.mus, ys, zs)
    O = orc.Oracle.from_workload(wl)
    for q in range(4):
        r = _oracle_norm(O, wl, wl.mus[q], ys[q], zs[q])
        # FP32 residual entries (unit roundoff 6e-8) from sums of a few dozen terms whose
        # size is that of the fluxes, compared with a residual far smaller than them
        assert abs(g[q] - r) <= 1e-3 * r


def test_nonphysical_point_is_infinite():
    wl = W.euler_workload(n=8, p=1, k_u=6, k_x=2, seed=33, n_mu=2, mu_box=True)
    ys = np.stack([wl.w_eval, -wl.w_eval])  # negative density everywhere in the second
    zs = np.stack([wl.tau_eval, wl.tau_eval])
    g = ift.Context.from_workload(wl).hdm_residual_norms(wl.mus, ys, zs)
    assert np.isfinite(g[0]) and np.isinf(g[1])


def test_greedy_search_picks_the_oracle_argmax():
    # candidates solved by the batched hyperreduced LM with one shared weight set,
    # then the indicator at each solution; the oracle evaluates the same points
    wl = W.euler_workload(n=12, p=2, k_u=8, k_x=2, seed=34)
    mus = W.mu_box_samples(35, 1, 12)
    rho = W.eq_weight_sets(wl, 1, seed=36, lo=110, hi=111)[0]
    ctx = ift.Context.from_workload(wl, tol=1e-8)
    ctx.set_eq_weights_batched([rho] * len(mus))
    best, norms, res = ctx.greedy_search(mus)
    O = orc.Oracle.from_workload(wl)
    ref = np.array([_oracle_norm(O, wl, mus[q], res["w"][q], res["tau"][q]) for q in range(len(mus))])
    np.testing.assert_allclose(norms, ref, rtol=1e-12)
    assert best == int(np.argmax(ref))
    assert all(i["status"] == 0 for i in res["info"])


def test_errors():
    wl = W.euler_workload(n=6, p=1, k_u=4, k_x=2, seed=3, n_mu=2, mu_box=True)
    ctx = ift.Context(ift.EULER2D, 1)
    with pytest.raises(ift.IFTError) as ei:
        ctx.hdm_residual_norms(wl.mus, np.zeros((2, 4)), np.zeros((2, 2)))
    assert ei.value.status == -2
