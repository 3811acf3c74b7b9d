"""Mixed precision (FP32 element kernels and contraction for most LM iterations,
FP64 assemblies to finish) and the larger reduced sizes (p = 3, k_u = 40, k_x = 8).

A mixed solve follows a different trajectory than the FP64 oracle's, so it is
judged by what the paper's stopping test fixes: the oracle itself must find the
GPU's final point optimal to the tolerance (its own |[S;T]| there), and the two
converged points must agree to the accuracy that tolerance allows.
"""

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fro(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _certify(O, wl, mu, rho_set, w, tau, ref, tol):
    rr = O.reduced(wl.Phi, wl.Psi, w, tau, mu, rho_set=rho_set)
    gn = np.linalg.norm(np.concatenate([rr["S"], rr["T"]]))
    assert gn <= 1.5 * tol * max(1.0, ref["g0"]), (gn, ref["g0"])
    z = np.concatenate([w, tau])
    zr = np.concatenate([ref["w"], ref["tau"]])
    assert np.linalg.norm(z - zr) <= 1e-6 * np.linalg.norm(zr)


def test_mixed_solve_dense_matches_fp64_oracle():
    wl = W.euler_workload(n=10, p=2, k_u=10, k_x=4, seed=21)
    mu = wl.mus[0]
    O = orc.Oracle.from_workload(wl)
    ref = O.solve(wl.Phi, wl.Psi, mu, wl.Phi.T @ W.replicate_guess(wl, wl.U_guess), tol=1e-8)
    ctx = ift.Context.from_workload(wl, precision=ift.MIXED, tol=1e-8)
    g = ctx.solve_rom(mu)
    assert g["status"] == 0 and ref["status"] == 0
    # part of the joint iteration runs in FP32 and the FP64 stage is shorter than an FP64 solve
    assert g["fp32_iters"] > 0 and g["iters"] < ref["iters"]
    # the FP64 stage recomputes H after shortened steps only, and at its first point
    # only if the FP32 stage's last result was not evaluated there
    assert 0 <= g["h_evals"] <= g["trials"] + 1
    _certify(O, wl, mu, None, g["w"], g["tau"], ref, 1e-8)


def test_mixed_finishing_stage_keeps_h():
    # A finishing stage of several full steps: H is recomputed after a shortened step
    # only (at its first point it is the FP32 stage's last H when that was evaluated
    # there), the point still certified by the oracle.
    wl = W.euler_workload(n=12, p=2, k_u=12, k_x=4, seed=31, n_mu=3, mu_box=True)
    sets = W.eq_weight_sets(wl, 3, seed=32, lo=150, hi=250)
    ctx = ift.Context.from_workload(wl, precision=ift.MIXED, tol=1e-9)
    ctx.set_eq_weights_batched(sets)
    res = ctx.solve_rom_batched(wl.mus)
    O = orc.Oracle.from_workload(wl)
    kept = 0
    for q in range(3):
        i = res["info"][q]
        assert i["status"] == 0
        evals = i["trials"] + 1  # the restart point, then every trial point (new steps and halvings)
        assert 0 <= i["h_evals"] <= evals
        kept += evals - i["h_evals"]
        mu = wl.mus[q]
        wg = wl.Phi.T @ W.replicate_guess(wl, W.freestream_state(wl.gamma, mu[0], mu[1]))
        ref = O.solve(wl.Phi, wl.Psi, mu, wg, rho_set=sets[q], tol=1e-9)
        _certify(O, wl, mu, sets[q], res["w"][q], res["tau"][q], ref, 1e-9)
    assert kept > 0
    # the FP32-Jacobian mode recomputes H at every evaluation
    f = ift.Context.from_workload(wl, precision=ift.FP32_JACOBIAN, tol=1e-9)
    f.set_eq_weights_batched(sets)
    assert all(i["h_evals"] == 0 for i in f.solve_rom_batched(wl.mus)["info"])


def test_mixed_batched_matches_fp64_oracle():
    wl = W.euler_workload(n=12, p=2, k_u=8, k_x=2, seed=6, n_mu=4, mu_box=True)
    sets = W.eq_weight_sets(wl, 4, seed=7, lo=96, hi=200)
    ctx = ift.Context.from_workload(wl, precision=ift.MIXED, tol=1e-8)
    ctx.set_eq_weights_batched(sets)
    res = ctx.solve_rom_batched(wl.mus)
    O = orc.Oracle.from_workload(wl)
    for q in range(4):
        mu = wl.mus[q]
        wg = wl.Phi.T @ W.replicate_guess(wl, W.freestream_state(wl.gamma, mu[0], mu[1]))
        ref = O.solve(wl.Phi, wl.Psi, mu, wg, rho_set=sets[q], tol=1e-8)
        assert res["info"][q]["status"] == ref["status"] == 0
        _certify(O, wl, mu, sets[q], res["w"][q], res["tau"][q], ref, 1e-8)


@pytest.mark.parametrize("precision", [ift.FP64, ift.FP32])
def test_p3_k48_assembly(precision):
    # the reduced sizes of the mixed-precision configuration: p = 3, k_u = 40, k_x = 8
    wl = W.euler_workload(n=8, p=3, k_u=40, k_x=8, seed=22)
    O = orc.Oracle.from_workload(wl)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, wl.mus[0])
    ctx = ift.Context.from_workload(wl, precision=precision)
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    if precision == ift.FP64:
        for key in ("S", "T", "H"):
            assert _fro(g[key], r[key]) < 1e-10, key
        assert abs(g["J"] - r["J"]) <= 1e-10 * r["J"]
    else:
        assert _fro(g["H"], r["H"]) < 1e-5
        assert _fro(np.concatenate([g["S"], g["T"]]), np.concatenate([r["S"], r["T"]])) < 1e-3
        assert abs(g["J"] - r["J"]) <= 1e-5 * r["J"]


def test_p3_k48_batched_sampled_queries_full_mesh():
    # 200 x 200 x 2 = 80,000 elements: the oracle checks sampled hyperreduced queries
    wl = W.euler_workload(n=200, p=3, k_u=40, k_x=8, seed=4, n_mu=3, mu_box=True)
    sets = W.eq_weight_sets(wl, 3, seed=5, lo=100, hi=300)
    ctx = ift.Context.from_workload(wl, precision=ift.FP32)
    ctx.set_eq_weights_batched(sets)
    ys = np.stack([wl.w_eval] * 3)
    zs = np.stack([wl.tau_eval] * 3)
    g = ctx.reduced_residual_jacobian_batched(wl.mus, ys, zs)
    O = orc.Oracle.from_workload(wl)
    for q in range(3):
        r = O.reduced(wl.Phi, wl.Psi, ys[q], zs[q], wl.mus[q], rho_set=sets[q])
        assert _fro(g["H"][q], r["H"]) < 1e-5
        assert _fro(np.concatenate([g["S"][q], g["T"][q]]), np.concatenate([r["S"], r["T"]])) < 1e-3
        assert abs(g["J"][q] - r["J"]) <= 1e-5 * r["J"]


@pytest.mark.parametrize("contraction,tol", [(ift.CONTRACT_TF32, 5e-3), (ift.CONTRACT_3XTF32, 1e-5),
                                             (ift.CONTRACT_BF16, 3e-2)])
@pytest.mark.parametrize("p,ku,kx,kappa", [(2, 20, 4, 0.0), (3, 40, 8, 0.1), (1, 7, 3, 0.1)])
def test_tensor_core_contraction(contraction, tol, p, ku, kx, kappa):
    # H on the tensor cores: TF32 to its 10-bit mantissa, 3xTF32 to FP32 accuracy,
    # BF16 to its 7-bit mantissa; S~, T~, J~ do not go through the tensor cores and
    # equal the FP32 context's bit for bit. p = 1 has n_u = 12 rows (a ragged last
    # k-step: 8-row TF32 steps, 16-row BF16 steps) and k = 10 (partial tiles).
    wl = W.euler_workload(n=8, p=p, k_u=ku, k_x=kx, seed=23)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, wl.mus[0])
    f32 = ift.Context.from_workload(wl, precision=ift.FP32, kappa=kappa)
    tc = ift.Context.from_workload(wl, precision=ift.FP32, kappa=kappa, contraction=contraction)
    a = f32.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    b = tc.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    assert _fro(b["H"], r["H"]) < tol
    assert np.array_equal(b["H"], b["H"].T)
    for key in ("S", "T"):
        assert np.array_equal(a[key], b[key]), key
    assert a["J"] == b["J"]


def test_tensor_core_contraction_sparse_and_batched():
    wl = W.euler_workload(n=12, p=2, k_u=16, k_x=4, seed=24, n_mu=3, mu_box=True)
    sets = W.eq_weight_sets(wl, 3, seed=25, lo=40, hi=120)
    O = orc.Oracle.from_workload(wl)
    ctx = ift.Context.from_workload(wl, precision=ift.FP32, contraction=ift.CONTRACT_3XTF32)
    ctx.set_eq_weights(sets[0])
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, wl.mus[0], rho_set=sets[0])
    assert _fro(g["H"], r["H"]) < 1e-5
    ctx.set_eq_weights_batched(sets)
    ys, zs = np.stack([wl.w_eval] * 3), np.stack([wl.tau_eval] * 3)
    gb = ctx.reduced_residual_jacobian_batched(wl.mus, ys, zs)
    for q in range(3):
        r = O.reduced(wl.Phi, wl.Psi, ys[q], zs[q], wl.mus[q], rho_set=sets[q])
        assert _fro(gb["H"][q], r["H"]) < 1e-5


@pytest.mark.parametrize("contraction", [ift.CONTRACT_TF32, ift.CONTRACT_BF16])
def test_mixed_solve_with_tensor_core_contraction(contraction):
    # H only steers the step: a mixed solve whose FP32 stage takes H from TF32 or
    # BF16 tensor cores converges to the FP64 oracle's optimum
    wl = W.euler_workload(n=10, p=2, k_u=10, k_x=4, seed=21)
    mu = wl.mus[0]
    O = orc.Oracle.from_workload(wl)
    ref = O.solve(wl.Phi, wl.Psi, mu, wl.Phi.T @ W.replicate_guess(wl, wl.U_guess), tol=1e-8)
    ctx = ift.Context.from_workload(wl, precision=ift.MIXED, tol=1e-8, contraction=contraction)
    g = ctx.solve_rom(mu)
    assert g["status"] == 0 and g["fp32_iters"] > 0
    _certify(O, wl, mu, None, g["w"], g["tau"], ref, 1e-8)


def test_contraction_option_errors():
    with pytest.raises(ift.IFTError):
        ift.Context(ift.EULER2D, 2, precision=ift.FP64, contraction=ift.CONTRACT_TF32)
    with pytest.raises(ift.IFTError):
        ift.Context(ift.EULER2D, 2, precision=ift.FP32, contraction=7)


@pytest.mark.parametrize("p,kappa,contraction", [(2, 0.0, ift.CONTRACT_FP), (3, 0.1, ift.CONTRACT_TF32),
                                                 (1, 0.0, ift.CONTRACT_3XTF32), (2, 0.1, ift.CONTRACT_BF16)])
def test_fp32_jacobian_mode_gradient_is_fp64(p, kappa, contraction):
    # H from the FP32 element Jacobians; S~, T~, J~ from the FP64 residual-and-adjoint pass
    wl = W.euler_workload(n=8, p=p, k_u=9, k_x=3, seed=81)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, wl.mus[0])
    ctx = ift.Context.from_workload(wl, precision=ift.FP32_JACOBIAN, kappa=kappa, contraction=contraction)
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    assert _fro(g["S"], r["S"]) < 1e-10 and _fro(g["T"], r["T"]) < 1e-10
    assert abs(g["J"] - r["J"]) <= 1e-10 * r["J"]
    assert _fro(g["H"], r["H"]) < {ift.CONTRACT_TF32: 5e-3, ift.CONTRACT_BF16: 3e-2}.get(contraction, 1e-5)


def test_fp32_jacobian_mode_sparse_weights_and_burgers():
    wl = W.euler_workload(n=10, p=2, k_u=8, k_x=2, seed=82)
    rho = W.eq_weight_sets(wl, 1, seed=83, lo=40, hi=41)[0]
    O = orc.Oracle.from_workload(wl)
    ctx = ift.Context.from_workload(wl, precision=ift.FP32_JACOBIAN)
    ctx.set_eq_weights(rho)
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, wl.mus[0], rho_set=rho)
    assert _fro(np.concatenate([g["S"], g["T"]]), np.concatenate([r["S"], r["T"]])) < 1e-10
    wb = W.burgers_workload(n_elems=40, p=2, k_u=4, seed=3)
    Ob = orc.Oracle.from_workload(wb)
    rb = Ob.reduced(wb.Phi, wb.Psi, wb.w_eval, wb.tau_eval, wb.mus[0])
    gb = ift.Context.from_workload(wb, precision=ift.FP32_JACOBIAN).reduced_residual_jacobian(
        wb.mus[0], wb.w_eval, wb.tau_eval)
    assert _fro(np.concatenate([gb["S"], gb["T"]]), np.concatenate([rb["S"], rb["T"]])) < 1e-10
    assert abs(gb["J"] - rb["J"]) <= 1e-10 * rb["J"]


@pytest.mark.parametrize("p,count,kappa", [(2, 37, 0.0), (3, 11, 0.1), (1, 5, 0.0)])
def test_gradient_pass_odd_element_counts(p, count, kappa):
    # The FP64 gradient pass evaluates two elements per warp (one per half-warp); with
    # an odd number of sampled elements a half re-evaluates its partner's element
    # with weight 0. S~, T~, J~ must still be the oracle's to 1e-10, the non-physical
    # count must stay 0, and a chunked batch with odd chunk tails must agree too.
    wl = W.euler_workload(n=8, p=p, k_u=9, k_x=3, seed=91, n_mu=3, mu_box=True)
    sets = W.eq_weight_sets(wl, 3, seed=92, lo=count, hi=count + 1)
    assert all(len(e) % 2 == 1 for e, _ in sets)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    ctx = ift.Context.from_workload(wl, precision=ift.FP32_JACOBIAN, kappa=kappa)
    ctx.set_eq_weights(sets[0])
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, wl.mus[0], rho_set=sets[0])
    assert _fro(np.concatenate([g["S"], g["T"]]), np.concatenate([r["S"], r["T"]])) < 1e-10
    assert abs(g["J"] - r["J"]) <= 1e-10 * r["J"]
    ctx.set_eq_weights_batched(sets)
    ctx.set_launch_shapes(2, 2, 4)  # chunks of 4: odd tails in every query
    ys, zs = np.stack([wl.w_eval] * 3), np.stack([wl.tau_eval] * 3)
    gb = ctx.reduced_residual_jacobian_batched(wl.mus, ys, zs)
    for q in range(3):
        r = O.reduced(wl.Phi, wl.Psi, ys[q], zs[q], wl.mus[q], rho_set=sets[q])
        assert _fro(np.concatenate([gb["S"][q], gb["T"][q]]), np.concatenate([r["S"], r["T"]])) < 1e-10
        assert abs(gb["J"][q] - r["J"]) <= 1e-10 * r["J"]


def test_fp32_jacobian_mode_solves_reach_the_fp64_optimum():
    wl = W.euler_workload(n=10, p=2, k_u=10, k_x=4, seed=21)
    mu = wl.mus[0]
    O = orc.Oracle.from_workload(wl)
    ref = O.solve(wl.Phi, wl.Psi, mu, wl.Phi.T @ W.replicate_guess(wl, wl.U_guess), tol=1e-8)
    for contraction in (ift.CONTRACT_FP, ift.CONTRACT_TF32, ift.CONTRACT_BF16):
        ctx = ift.Context.from_workload(wl, precision=ift.FP32_JACOBIAN, tol=1e-8, contraction=contraction)
        g = ctx.solve_rom(mu)
        assert g["status"] == 0
        # the iteration is the FP64 one up to the rounding of H: the same number of steps, give or
        # take (BF16's H, about 8 times coarser than TF32's, may cost a few more)
        allow = 6 if contraction == ift.CONTRACT_BF16 else 2
        assert abs(g["iters"] + g["init_iters"] - ref["iters"] - ref["init_iters"]) <= allow
        _certify(O, wl, mu, None, g["w"], g["tau"], ref, 1e-8)


def test_fp32_jacobian_mode_batched():
    wl = W.euler_workload(n=12, p=2, k_u=8, k_x=2, seed=6, n_mu=4, mu_box=True)
    sets = W.eq_weight_sets(wl, 4, seed=7, lo=96, hi=200)
    ctx = ift.Context.from_workload(wl, precision=ift.FP32_JACOBIAN, tol=1e-8)
    ctx.set_eq_weights_batched(sets)
    ys, zs = np.stack([wl.w_eval] * 4), np.stack([wl.tau_eval] * 4)
    gb = ctx.reduced_residual_jacobian_batched(wl.mus, ys, zs)
    O = orc.Oracle.from_workload(wl)
    for q in range(4):
        r = O.reduced(wl.Phi, wl.Psi, ys[q], zs[q], wl.mus[q], rho_set=sets[q])
        assert _fro(np.concatenate([gb["S"][q], gb["T"][q]]), np.concatenate([r["S"], r["T"]])) < 1e-10
        assert abs(gb["J"][q] - r["J"]) <= 1e-10 * r["J"]
    res = ctx.solve_rom_batched(wl.mus)
    for q in range(4):
        mu = wl.mus[q]
        wg = wl.Phi.T @ W.replicate_guess(wl, W.freestream_state(wl.gamma, mu[0], mu[1]))
        ref = O.solve(wl.Phi, wl.Psi, mu, wg, rho_set=sets[q], tol=1e-8)
        assert res["info"][q]["status"] == ref["status"] == 0
        _certify(O, wl, mu, sets[q], res["w"][q], res["tau"][q], ref, 1e-8)
