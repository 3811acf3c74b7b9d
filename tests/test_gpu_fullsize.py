"""Solves at the full sizes the benchmark numbers are quoted on, against the FP64 oracle.

* The 20,000-element Euler configuration (p = 2, k_u = 20, k_x = 4, rho = 1): the
  FP64 solve (the benchmark's step) takes the oracle's trajectory, with equal
  initialisation and joint iteration counts and (w, tau) to 1e-10 (Sec. 3.2.3,
  Remark rem:solver); the mixed-precision solve of the same workload reaches the
  oracle's optimum (the oracle's own optimality residual at the GPU's point within
  1.5x the threshold, the point within 1e-6).
* The 80,000-element p = 3 configuration (k_u = 40, k_x = 8) with 1,024
  hyperreduced queries solved in one batch in the mixed form with BF16 tensor-core
  H: three queries (the smallest, a median and the largest weight set among those
  that converge) are solved by the oracle and certified: the oracle's optimality
  residual at the GPU's point within 1.5x the threshold, and the distance between
  the two converged points within what the stopping test allows,
  2 (|g(z)| + |g(z_ref)|) / lambda_min(H) (near an optimum z - z* = H^{-1} g to
  first order), with J~ within the matching second-order change. On the smallest
  sets (100 elements for k = 48 unknowns) H is ill-conditioned enough (lambda_min
  2.8e-9 against lambda_max 1.1e-5 on one query) that a fixed 1e-6 relative
  distance is tighter than the tolerance fixes.

The oracle solves run on every host core (OpenMP); the 20,000-element one takes a
few seconds.
"""

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W
from test_gpu_parity import check_solve_against_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def config2():
    wl = W.euler_workload(n=100, p=2, k_u=20, k_x=4, seed=2)
    O = orc.Oracle.from_workload(wl)
    mu = wl.mus[0]
    wg = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess)
    ref = O.solve(wl.Phi, wl.Psi, mu, wg, tol=1e-8)
    assert ref["status"] == 0
    return wl, O, mu, ref


def test_config2_fp64_solve_follows_the_oracle(config2):
    wl, O, mu, ref = config2
    ctx = ift.Context.from_workload(wl, tol=1e-8)
    g = ctx.solve_rom(mu)
    assert check_solve_against_oracle(g, ref, O, wl, mu, None, 1e-8) == "same"
    ctx.close()


def test_config2_mixed_solve_reaches_the_oracle_optimum(config2):
    wl, O, mu, ref = config2
    ctx = ift.Context.from_workload(wl, precision=ift.MIXED, tol=1e-8)
    g = ctx.solve_rom(mu)
    assert g["status"] == 0 and g["fp32_iters"] > 0
    rr = O.reduced(wl.Phi, wl.Psi, g["w"], g["tau"], mu)
    gn = np.linalg.norm(np.concatenate([rr["S"], rr["T"]]))
    assert gn <= 1.5 * 1e-8 * max(1.0, ref["g0"]), (gn, ref["g0"])
    z = np.concatenate([g["w"], g["tau"]])
    zr = np.concatenate([ref["w"], ref["tau"]])
    assert np.linalg.norm(z - zr) <= 1e-6 * np.linalg.norm(zr)
    assert abs(g["J"] - ref["J"]) <= 1e-8 * ref["J"]
    ctx.close()


def test_config4_mixed_bf16_batch_against_the_oracle():
    B = 1024
    wl = W.euler_workload(n=200, p=3, k_u=40, k_x=8, seed=4, n_mu=B, mu_box=True)
    sets = W.eq_weight_sets(wl, B, seed=5)
    ctx = ift.Context.from_workload(wl, precision=ift.MIXED, contraction=ift.CONTRACT_BF16, tol=1e-8)
    ctx.set_eq_weights_batched(sets)
    res = ctx.solve_rom_batched(wl.mus)
    ctx.close()
    st = np.array([i["status"] for i in res["info"]])
    assert (st == 0).sum() >= 0.95 * B
    sizes = np.array([len(s[0]) for s in sets])
    ok = np.nonzero(st == 0)[0]
    order = ok[np.argsort(sizes[ok], kind="stable")]
    picks = [order[0], order[len(order) // 2], order[-1]]
    O = orc.Oracle.from_workload(wl)
    for q in picks:
        mu = wl.mus[q]
        wg = wl.Phi.T @ W.replicate_guess(wl, W.freestream_state(wl.gamma, mu[0], mu[1]))
        ref = O.solve(wl.Phi, wl.Psi, mu, wg, rho_set=sets[q], tol=1e-8)
        assert ref["status"] == 0, (q, ref["status"])
        w, tau = res["w"][q], res["tau"][q]
        rr = O.reduced(wl.Phi, wl.Psi, w, tau, mu, rho_set=sets[q])
        gn = np.linalg.norm(np.concatenate([rr["S"], rr["T"]]))
        assert gn <= 1.5 * 1e-8 * max(1.0, ref["g0"]), (q, sizes[q], gn, ref["g0"])
        r0 = O.reduced(wl.Phi, wl.Psi, ref["w"], ref["tau"], mu, rho_set=sets[q])
        g_ref = np.linalg.norm(np.concatenate([r0["S"], r0["T"]]))
        ev = np.linalg.eigvalsh(r0["H"])
        assert ev[0] > 0.0
        z = np.concatenate([w, tau])
        zr = np.concatenate([ref["w"], ref["tau"]])
        dz = np.linalg.norm(z - zr)
        assert dz <= 2.0 * (gn + g_ref) / ev[0], (q, sizes[q], dz, gn, g_ref, ev[0])
        # and J~ to second order along that distance
        dJ_max = 2.0 * (g_ref * dz + 0.5 * ev[-1] * dz * dz) + 1e-12 * ref["J"]
        assert abs(rr["J"] - ref["J"]) <= dJ_max, (q, rr["J"], ref["J"], dJ_max)
