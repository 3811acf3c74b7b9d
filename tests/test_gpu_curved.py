"""Curved (q = 2) elements on the GPU against the FP64 oracle: the six-node
quadratic element map with the cofactor g G^{-T} and the scaled face normals at
every quadrature point (Eq. p2r-flux), the distortion of Eq. dist_elem1 by
quadrature, and the reduced quantities, gradient pass and solves built on them.
Tolerances as for straight-sided elements: FP64 element blocks rel 1e-12 of the
Jacobian scale, reduced quantities 1e-10, FP32 H 1e-5.
"""

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def fro(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def shifted(X, n, seed, amp=0.1):
    rng = np.random.default_rng(seed)
    interior = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    d = rng.uniform(-1, 1, size=X.shape) * amp / n
    d[~interior] = 0.0
    return X + d


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kappa", [0.0, 0.1])
def test_curved_element_parity(p, kappa):
    n = 4
    X, ev = W.square_tri_mesh_q2(n, curve=0.4)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA, kappa=kappa, q=2)
    ctx = ift.Context(ift.EULER2D, p, kappa=kappa, q=2)
    ctx.set_mesh(X, ev)
    assert ctx.nxe == 12
    mu = np.array([2.0, 0.03])
    rng = np.random.default_rng(p)
    U = np.tile(orc.freestream(GAMMA, mu), O.Nu // 4) * (1 + 0.05 * rng.normal(size=O.Nu))
    x = shifted(X, n, seed=p).ravel()
    elems = np.arange(O.n_elems, dtype=np.int32)
    g = ctx.element_eval(mu, U, x, elems)
    for e in elems:
        Ue, Up, xe = O.gather(U, x, e)
        r = O.element(e, Ue, Up, xe, mu)
        assert rel(g["R"][e], r["R"]) < 1e-12
        scale = max(np.abs(r["JU"]).max(), np.abs(r["JUp"]).max(), np.abs(r["Jx"]).max())
        for key in ("JU", "JUp", "Jx"):
            assert np.abs(g[key][e] - r[key]).max() <= 1e-12 * scale, key
        assert abs(g["N"][e] - r["N"]) <= 1e-12 * max(abs(r["N"]), 1e-12)
        if kappa:
            assert np.abs(g["dN"][e] - r["dN"]).max() <= 1e-10 * max(np.abs(r["dN"]).max(), 1e-12)


@pytest.mark.parametrize("p,ku,kx,kappa", [(2, 10, 4, 0.0), (3, 12, 8, 0.1), (1, 7, 3, 0.1)])
def test_curved_reduced_fp64_and_fp32(p, ku, kx, kappa):
    wl = W.euler_workload(n=8, p=p, k_u=ku, k_x=kx, seed=61, q=2, curve=0.4)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, wl.mus[0])
    g = ift.Context.from_workload(wl, kappa=kappa).reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    for key in ("S", "T", "H"):
        assert fro(g[key], r[key]) < 1e-10, key
    assert abs(g["J"] - r["J"]) <= 1e-10 * r["J"]
    f = ift.Context.from_workload(wl, kappa=kappa, precision=ift.FP32).reduced_residual_jacobian(
        wl.mus[0], wl.w_eval, wl.tau_eval)
    assert fro(f["H"], r["H"]) < 1e-5
    assert abs(f["J"] - r["J"]) <= 1e-5 * r["J"]
    # the split-precision evaluation: S~, T~, J~ from the FP64 gradient pass (two elements per warp)
    s = ift.Context.from_workload(wl, kappa=kappa, precision=ift.FP32_JACOBIAN).reduced_residual_jacobian(
        wl.mus[0], wl.w_eval, wl.tau_eval)
    assert fro(np.concatenate([s["S"], s["T"]]), np.concatenate([r["S"], r["T"]])) < 1e-10
    assert abs(s["J"] - r["J"]) <= 1e-10 * r["J"]


def test_curved_sparse_and_batched():
    wl = W.euler_workload(n=10, p=2, k_u=9, k_x=4, seed=62, n_mu=3, mu_box=True, q=2, curve=0.4)
    sets = W.eq_weight_sets(wl, 3, seed=63, lo=30, hi=80)
    O = orc.Oracle.from_workload(wl)
    ctx = ift.Context.from_workload(wl)
    ctx.set_eq_weights(sets[0])
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, wl.mus[0], rho_set=sets[0])
    for key in ("S", "T", "H"):
        assert fro(g[key], r[key]) < 1e-10, key
    ctx.set_eq_weights_batched(sets)
    ys, zs = np.stack([wl.w_eval] * 3), np.stack([wl.tau_eval] * 3)
    gb = ctx.reduced_residual_jacobian_batched(wl.mus, ys, zs)
    for q in range(3):
        r = O.reduced(wl.Phi, wl.Psi, ys[q], zs[q], wl.mus[q], rho_set=sets[q])
        for key in ("S", "T", "H"):
            assert fro(gb[key][q], r[key]) < 1e-10, (q, key)


def test_curved_solves_match_the_oracle():
    wl = W.euler_workload(n=6, p=2, k_u=8, k_x=3, seed=64, q=2, curve=0.4)
    mu = wl.mus[0]
    O = orc.Oracle.from_workload(wl)
    ref = O.solve(wl.Phi, wl.Psi, mu, wl.Phi.T @ W.replicate_guess(wl, wl.U_guess), tol=1e-8)
    assert ref["status"] == 0
    g = ift.Context.from_workload(wl, tol=1e-8).solve_rom(mu)
    assert g["status"] == 0
    assert abs(g["iters"] + g["init_iters"] - ref["iters"] - ref["init_iters"]) <= 2
    z, zr = np.concatenate([g["w"], g["tau"]]), np.concatenate([ref["w"], ref["tau"]])
    assert np.linalg.norm(z - zr) <= 1e-8 * np.linalg.norm(zr)
    m = ift.Context.from_workload(wl, tol=1e-8, precision=ift.MIXED).solve_rom(mu)
    assert m["status"] == 0
    zm = np.concatenate([m["w"], m["tau"]])
    rr = O.reduced(wl.Phi, wl.Psi, m["w"], m["tau"], mu)
    assert np.linalg.norm(np.concatenate([rr["S"], rr["T"]])) <= 1.5e-8 * max(1.0, ref["g0"])
    assert np.linalg.norm(zm - zr) <= 1e-6 * np.linalg.norm(zr)


def test_q2_config_errors():
    with pytest.raises(ift.IFTError):
        ift.Context(ift.BURGERS1D, 2, q=2)
    with pytest.raises(ift.IFTError):
        ift.Context(ift.EULER2D, 2, q=3)
