"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

Tolerances (FP64): element residuals and Jacobians rel 1e-12, reduced H, g, J
rel 1e-10 (Frobenius / max-norm), LM iterates rel 1e-10 at the same iteration
count. FP32 element kernels: the tolerances below follow from FP32 rounding
(unit roundoff 6e-8) amplified by sums of a few hundred terms and by the
cancellation in g = sum_e A_e^T R_e.
"""

import dataclasses

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def jac_scale(r):
    return max(np.abs(r["JU"]).max(), np.abs(r["JUp"]).max(), np.abs(r["Jx"]).max())


def deformed(X, ev, n, seed, amp=0.3):
    rng = np.random.default_rng(seed)
    interior = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    d = rng.uniform(-1, 1, size=X.shape) * amp / n
    d[~interior] = 0.0
    return X + d


# ---------------------------------------------------------------------------
# element level
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kappa", [0.0, 0.1])
def test_euler_element_parity(p, kappa):
    n = 4
    X, ev = W.square_tri_mesh(n)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA, kappa=kappa)
    ctx = ift.Context(ift.EULER2D, p, kappa=kappa)
    ctx.set_mesh(X, ev)
    mu = np.array([2.0, 0.03])
    rng = np.random.default_rng(p)
    U = np.tile(orc.freestream(GAMMA, mu), O.Nu // 4) * (1 + 0.05 * rng.normal(size=O.Nu))
    x = deformed(X, ev, n, seed=p).ravel()
    elems = np.arange(O.n_elems, dtype=np.int32)
    g = ctx.element_eval(mu, U, x, elems)
    for e in elems:
        Ue, Up, xe = O.gather(U, x, e)
        r = O.element(e, Ue, Up, xe, mu)
        assert rel(g["R"][e], r["R"]) < 1e-12
        # Jacobian blocks against the element's Jacobian scale: a block can be pure
        # rounding noise (a supersonic outflow face does not depend on the exterior state)
        scale = jac_scale(r)
        for key in ("JU", "JUp", "Jx"):
            assert np.abs(g[key][e] - r[key]).max() <= 1e-12 * scale, key
        assert abs(g["N"][e] - r["N"]) <= 1e-12 * max(abs(r["N"]), 1e-12)
        if kappa:
            assert rel(g["dN"][e], r["dN"]) < 1e-10


@pytest.mark.parametrize("p", [1, 2, 3])
def test_burgers_element_parity(p):
    X, ev = W.interval_mesh(7)
    O = orc.Oracle(orc.PROB_BURGERS1D, p, X, ev)
    ctx = ift.Context(ift.BURGERS1D, p)
    ctx.set_mesh(X, ev)
    rng = np.random.default_rng(p)
    U = 1.0 + 0.3 * rng.normal(size=O.Nu)
    x = X + np.concatenate([[0], 0.03 * rng.uniform(-1, 1, 6), [0]])
    mu = np.array([1.3])
    g = ctx.element_eval(mu, U, x, np.arange(7, dtype=np.int32))
    for e in range(7):
        Ue, Up, xe = O.gather(U, x, e)
        r = O.element(e, Ue, Up, xe, mu)
        assert rel(g["R"][e], r["R"]) < 1e-12
        for key in ("JU", "JUp", "Jx"):
            assert np.abs(g[key][e] - r[key]).max() <= 1e-12 * jac_scale(r), key


def test_fp32_element_accuracy():
    n, p = 4, 2
    X, ev = W.square_tri_mesh(n)
    O = orc.Oracle(orc.PROB_EULER2D, p, X, ev, gamma=GAMMA)
    ctx = ift.Context(ift.EULER2D, p, precision=ift.FP32)
    ctx.set_mesh(X, ev)
    mu = np.array([2.0, 0.0])
    rng = np.random.default_rng(3)
    U = np.tile(orc.freestream(GAMMA, mu), O.Nu // 4) * (1 + 0.05 * rng.normal(size=O.Nu))
    x = deformed(X, ev, n, seed=3).ravel()
    g = ctx.element_eval(mu, U, x, np.arange(O.n_elems, dtype=np.int32))
    worst = {"R": 0.0, "JU": 0.0, "JUp": 0.0, "Jx": 0.0}
    for e in range(O.n_elems):
        Ue, Up, xe = O.gather(U, x, e)
        r = O.element(e, Ue, Up, xe, mu)
        for key in worst:
            # residuals are differences of O(1) fluxes: measure against the flux scale;
            # Jacobian blocks against the element's Jacobian scale
            scale = np.abs(r["JU"]).max() * np.abs(Ue).max() if key == "R" else jac_scale(r)
            worst[key] = max(worst[key], np.abs(g[key][e] - r[key]).max() / scale)
    assert all(v < 1e-5 for v in worst.values()), worst


# ---------------------------------------------------------------------------
# reduced assembly
# ---------------------------------------------------------------------------

def _assembly_pair(wl, rho_set=None, precision=ift.FP64, kappa=None):
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    ctx = ift.Context.from_workload(wl, precision=precision, **({"kappa": kappa} if kappa is not None else {}))
    ctx.set_eq_weights(rho_set)
    mu = wl.mus[0]
    g = ctx.reduced_residual_jacobian(mu, wl.w_eval, wl.tau_eval)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, mu, rho_set=rho_set)
    return g, r, ctx


def _fro(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("kappa", [0.0, 0.1])
def test_euler_reduced_fp64_dense(kappa):
    wl = W.euler_workload(n=8, p=2, k_u=8, k_x=4, seed=5)
    g, r, _ = _assembly_pair(wl, kappa=kappa)
    assert g["status"] == 0
    for key in ("S", "T", "H"):
        assert _fro(g[key], r[key]) < 1e-10, key
    assert abs(g["J"] - r["J"]) <= 1e-10 * r["J"]


@pytest.mark.parametrize("p", [1, 3])
def test_euler_reduced_fp64_sparse_rho(p):
    wl = W.euler_workload(n=10, p=p, k_u=7, k_x=3, seed=6)
    sets = W.eq_weight_sets(wl, 2, seed=7, lo=20, hi=60)
    for rs in sets:
        g, r, _ = _assembly_pair(wl, rho_set=rs)
        for key in ("S", "T", "H"):
            assert _fro(g[key], r[key]) < 1e-10, key
        assert abs(g["J"] - r["J"]) <= 1e-10 * r["J"]


def test_burgers_reduced_fp64_full_size():
    wl = W.burgers_workload()
    wl.w_eval = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess) + 0.05 * wl.w_eval
    g, r, _ = _assembly_pair(wl)
    for key in ("S", "T", "H"):
        assert _fro(g[key], r[key]) < 1e-10, key
    assert abs(g["J"] - r["J"]) <= 1e-10 * r["J"]


def test_euler_config2_full_size_fp64_and_fp32():
    # 100 x 100 x 2 triangles, p = 2, k_u = 20, k_x = 4: the full assembly of the benchmark
    wl = W.euler_workload(n=100, p=2, k_u=20, k_x=4, seed=2)
    g, r, _ = _assembly_pair(wl)
    for key in ("S", "T", "H"):
        assert _fro(g[key], r[key]) < 1e-10, key
    assert abs(g["J"] - r["J"]) <= 1e-10 * r["J"]
    ctx32 = ift.Context.from_workload(wl, precision=ift.FP32)
    g32 = ctx32.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    assert _fro(g32["H"], r["H"]) < 1e-5
    assert _fro(np.concatenate([g32["S"], g32["T"]]), np.concatenate([r["S"], r["T"]])) < 1e-3
    assert abs(g32["J"] - r["J"]) <= 1e-5 * r["J"]


def test_fp32_small_assembly_tolerances():
    wl = W.euler_workload(n=8, p=2, k_u=8, k_x=4, seed=5)
    g, r, _ = _assembly_pair(wl, precision=ift.FP32)
    assert _fro(g["H"], r["H"]) < 1e-5
    assert _fro(np.concatenate([g["S"], g["T"]]), np.concatenate([r["S"], r["T"]])) < 1e-3
    assert abs(g["J"] - r["J"]) <= 1e-5 * r["J"]


@pytest.mark.parametrize("p,ku,kx", [(2, 16, 4), (2, 20, 4), (2, 4, 4), (2, 10, 3), (2, 13, 3), (3, 12, 4),
                                     (3, 9, 2), (1, 8, 4)])
def test_fp32_reduced_assembly_shapes(p, ku, kx):
    # the FP32 state columns of p = 2 take eight- and four-column blocks when k_u and
    # k are multiples of four and single columns otherwise; p = 3 and p = 1 take the
    # per-column products
    wl = W.euler_workload(n=6, p=p, k_u=ku, k_x=kx, seed=40 + ku)
    g, r, _ = _assembly_pair(wl, precision=ift.FP32)
    assert _fro(g["H"], r["H"]) < 1e-5
    assert _fro(np.concatenate([g["S"], g["T"]]), np.concatenate([r["S"], r["T"]])) < 1e-3
    assert abs(g["J"] - r["J"]) <= 1e-5 * r["J"]


@pytest.mark.parametrize("p", [2, 3])
def test_fp32_assembly_on_a_translated_mesh(p):
    # the same mesh moved to x, y ~ 1000: FP32 vertex coordinates there are only good
    # to ~6e-5 absolute, 5e-4 of an element's edge, while the FP32 element pass takes
    # its edges from differences formed in FP64 and rounded once (the edge table), so
    # the FP32 tolerances still hold
    wl = W.euler_workload(n=8, p=p, k_u=12, k_x=4, seed=61)
    wl.X = wl.X + 1000.0
    g, r, _ = _assembly_pair(wl, precision=ift.FP32)
    assert _fro(g["H"], r["H"]) < 1e-5
    assert _fro(np.concatenate([g["S"], g["T"]]), np.concatenate([r["S"], r["T"]])) < 1e-3
    assert abs(g["J"] - r["J"]) <= 1e-5 * r["J"]


def test_assembly_is_deterministic():
    wl = W.euler_workload(n=20, p=2, k_u=10, k_x=4, seed=8)
    ctx = ift.Context.from_workload(wl)
    a = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    b = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    for key in ("S", "T", "H"):
        np.testing.assert_array_equal(a[key], b[key])
    assert a["J"] == b["J"]


def test_device_pointer_variant_matches_host():
    import torch

    wl = W.euler_workload(n=10, p=2, k_u=8, k_x=4, seed=9)
    ctx = ift.Context.from_workload(wl)
    h = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=dev)
    k = wl.ku + wl.kx
    S, T, H, J = (torch.zeros(n, dtype=torch.float64, device=dev) for n in (wl.ku, wl.kx, k * k, 1))
    stream = torch.cuda.current_stream().cuda_stream
    ctx.reduced_residual_jacobian_dev(t(wl.mus[0]), t(wl.w_eval), t(wl.tau_eval), S, T, H, J, stream=stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(S.cpu().numpy(), h["S"])
    np.testing.assert_array_equal(T.cpu().numpy(), h["T"])
    np.testing.assert_array_equal(H.cpu().numpy().reshape(k, k), h["H"])
    assert J.item() == h["J"]


# ---------------------------------------------------------------------------
# LM solve
# ---------------------------------------------------------------------------

def _solve_pair(wl, tol, rho_set=None):
    O = orc.Oracle.from_workload(wl)
    ctx = ift.Context.from_workload(wl, tol=tol)
    ctx.set_eq_weights(rho_set)
    mu = wl.mus[0]
    g = ctx.solve_rom(mu)
    wg = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess)
    r = O.solve(wl.Phi, wl.Psi, mu, wg, rho_set=rho_set, tol=tol)
    return g, r, O, wl, mu, rho_set, tol


def check_solve_against_oracle(g, r, O, wl, mu, rho_set, tol):
    """Same iteration count: the same trajectory, so (w, tau) agree to 1e-10.
    With linear convergence the last iterations can sit at the rounding floor of J
    (J changing by ~1e-16 relative per step), where the sufficient-decrease test and
    hence the damping updates are decided by rounding; two FP64 implementations that
    sum in different orders can then stop one or two steps apart. In that case the
    oracle itself must find the GPU's point converged (its own |[S;T]| there within
    1.5x the threshold) and the two points agree to the stopping tolerance.
    Returns the branch taken: "same" (equal counts, 1e-10) or "certified"."""
    assert g["status"] == 0 and r["status"] == 0, (g, r["status"])
    z = np.concatenate([g["w"], g["tau"]])
    zr = np.concatenate([r["w"], r["tau"]])
    if g["init_iters"] == r["init_iters"] and g["iters"] == r["iters"]:
        # a trial within rounding of the sufficient-decrease threshold may be halved once more
        assert abs(g["trials"] - r["trials"]) <= 2, (g["trials"], r["trials"])
        assert np.linalg.norm(z - zr) <= 1e-10 * np.linalg.norm(zr), np.linalg.norm(z - zr) / np.linalg.norm(zr)
        assert abs(g["J"] - r["J"]) <= 1e-12 * r["J"]
        return "same"
    else:
        assert abs((g["init_iters"] + g["iters"]) - (r["init_iters"] + r["iters"])) <= 2, (g, r)
        rr = O.reduced(wl.Phi, wl.Psi, g["w"], g["tau"], mu, rho_set=rho_set)
        gn = np.linalg.norm(np.concatenate([rr["S"], rr["T"]]))
        assert gn <= 1.5 * tol * max(1.0, r["g0"]), (gn, r["g0"])
        assert np.linalg.norm(z - zr) <= 1e-6 * np.linalg.norm(zr)
        return "certified"


def _check_solve(*pair):
    return check_solve_against_oracle(*pair)


def test_burgers_config1_solve():
    # the 200-element Burgers configuration: the oracle's trajectory step for step
    assert _check_solve(*_solve_pair(W.burgers_workload(), tol=1e-10)) == "same"


def test_euler_small_solve_dense():
    assert _check_solve(*_solve_pair(W.euler_workload(n=8, p=2, k_u=8, k_x=4, seed=6), tol=1e-8)) == "same"


def test_singular_w_block_solve_takes_the_shifted_factorisation():
    # a zero column of Phi: H has a zero row and column, so each LM step's Cholesky
    # meets a zero pivot on both sides and is retried with the diagonal shift
    # 1e-14 tr(M)/k; the same steps, the same number of shifts, and the zero
    # column's coefficient exactly 0
    wl = W.euler_workload(n=8, p=2, k_u=8, k_x=4, seed=6)
    Phi = wl.Phi.copy()
    Phi[:, -1] = 0.0
    pair = _solve_pair(dataclasses.replace(wl, Phi=Phi), tol=1e-8)
    g, r = pair[0], pair[1]
    assert _check_solve(*pair) == "same"
    assert r["shifts"] == r["init_iters"] + r["iters"] > 0
    assert g["shifts"] == r["shifts"]
    assert g["w"][-1] == 0.0


def test_euler_small_solve_sparse_rho(record_property):
    # the one solve of this file that stops a step or two away from the oracle's count
    # (its last steps sit at the rounding floor of J), so the oracle certifies the point
    wl = W.euler_workload(n=12, p=2, k_u=8, k_x=2, seed=6)
    rs = W.eq_weight_sets(wl, 1, seed=7, lo=96, hi=150)[0]
    branch = _check_solve(*_solve_pair(wl, tol=1e-8, rho_set=rs))
    record_property("solve_branches", branch)
    assert branch in ("same", "certified")


def test_given_start_and_repeat_solves():
    wl = W.burgers_workload()
    ctx = ift.Context.from_workload(wl, tol=1e-10)
    mu = wl.mus[0]
    a = ctx.solve_rom(mu)
    assert a["status"] == 0
    b = ctx.solve_rom(mu)
    np.testing.assert_array_equal(a["w"], b["w"])
    warm = ift.Context.from_workload(wl, tol=1e-10, lm_init=ift.INIT_GIVEN)
    c = warm.solve_rom(mu, a["w"], a["tau"])
    assert c["status"] == 0 and c["init_iters"] == 0 and c["iters"] <= 1


# ---------------------------------------------------------------------------
# edge cases and errors
# ---------------------------------------------------------------------------

def test_errors_and_call_order():
    ctx = ift.Context(ift.EULER2D, 2)
    with pytest.raises(ift.IFTError) as ei:
        ctx.reduced_residual_jacobian(np.array([2.0, 0.0]), np.zeros(3), np.zeros(1))
    assert ei.value.status == -2
    X, ev = W.square_tri_mesh(2)
    with pytest.raises(ift.IFTError) as ei:
        ctx.set_mesh(X, ev[:, [0, 2, 1]])  # clockwise: inverted
    assert ei.value.status == -1
    ctx.set_mesh(X, ev)
    with pytest.raises(ift.IFTError):
        ctx.set_bases(np.zeros((10, 2)), np.zeros((18, 1)))  # wrong N_u
    with pytest.raises(ift.IFTError):
        ctx.set_eq_weights((np.array([0, 0]), np.array([1.0, 1.0])))  # duplicate element
    with pytest.raises(ift.IFTError):
        ctx.set_eq_weights((np.array([0, 1]), np.array([1.0, -1.0])))  # negative weight
    with pytest.raises(ift.IFTError):
        ift.Context(ift.EULER2D, 7)


def test_nonphysical_point_reported():
    wl = W.euler_workload(n=6, p=1, k_u=4, k_x=2, seed=3)
    ctx = ift.Context.from_workload(wl)
    w = -wl.w_eval  # negative density everywhere
    g = ctx.reduced_residual_jacobian(wl.mus[0], w, wl.tau_eval)
    assert g["status"] == -5 and np.isinf(g["J"])


def test_no_mesh_motion_basis():
    wl = W.euler_workload(n=6, p=2, k_u=5, k_x=2, seed=3)
    wl.Psi = np.zeros((wl.Psi.shape[0], 0))
    wl.tau_eval = np.zeros(0)
    g, r, _ = _assembly_pair(wl)
    for key in ("S", "H"):
        assert _fro(g[key], r[key]) < 1e-10, key
    assert g["T"].shape == (0,)


@pytest.mark.parametrize("contraction,htol", [(ift.CONTRACT_FP, 1e-5), (ift.CONTRACT_BF16, 3e-2)])
def test_no_mesh_motion_basis_fp32(contraction, htol):
    # k_x = 0 in FP32: the edge table holds only the reference edges, the state
    # columns take the 8-column blocks (k = 8), and with BF16 the tcgen05 product
    # forms H from the stack
    wl = W.euler_workload(n=6, p=2, k_u=8, k_x=2, seed=3)
    wl.Psi = np.zeros((wl.Psi.shape[0], 0))
    wl.tau_eval = np.zeros(0)
    O = orc.Oracle.from_workload(wl)
    r = O.reduced(wl.Phi, wl.Psi, wl.w_eval, wl.tau_eval, wl.mus[0])
    ctx = ift.Context.from_workload(wl, precision=ift.FP32, contraction=contraction)
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    assert _fro(g["H"], r["H"]) < htol
    assert _fro(g["S"], r["S"]) < 1e-3
    assert abs(g["J"] - r["J"]) <= 1e-5 * r["J"]
    assert g["T"].shape == (0,)
    ctx.close()


def test_single_element_and_ragged_weight_list():
    wl = W.euler_workload(n=5, p=2, k_u=6, k_x=2, seed=2)
    for elems in ([7], [0, 1, 2], list(range(0, 50, 3))):
        rs = (np.array(elems), np.linspace(0.5, 3.0, len(elems)))
        g, r, _ = _assembly_pair(wl, rho_set=rs)
        for key in ("S", "T", "H"):
            assert _fro(g[key], r[key]) < 1e-10, key


# ---------------------------------------------------------------------------
# the largest reduced size a context takes (k_u + k_x = 64)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [2, 3])
def test_largest_reduced_size_assembly_and_solve(p, record_property):
    # 64 unknowns: H is 64 x 64 and the LM step's Cholesky runs on the full warp buffer
    wl = W.euler_workload(n=8, p=p, k_u=56, k_x=8, seed=17)
    g, r, _ = _assembly_pair(wl)
    for key in ("S", "T", "H"):
        assert _fro(g[key], r[key]) < 1e-10, key
    assert abs(g["J"] - r["J"]) <= 1e-10 * r["J"]
    branch = _check_solve(*_solve_pair(wl, tol=1e-8))
    record_property("solve_branches", branch)


def test_reduced_size_above_the_maximum_is_rejected():
    wl = W.euler_workload(n=4, p=2, k_u=57, k_x=8, seed=17)
    ctx = ift.Context(wl.problem, wl.p, gamma=wl.gamma)
    ctx.set_mesh(wl.X, wl.ev)
    with pytest.raises(ift.IFTError) as ei:
        ctx.set_bases(wl.Phi, wl.Psi)
    assert ei.value.status == -1
