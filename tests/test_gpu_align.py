"""Snapshot alignment (Eq. align0) on the GPU against the FP64 oracle: the
full-space residual F = [R; N], the products J v and J^T v that the conjugate-
gradient solve applies element by element (against the oracle's dense global
Jacobians), and the aligned (w, x) of the Levenberg-Marquardt iteration."""

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def interior_mask(X, dim=2):
    if dim == 1:
        inner = (X[:, 0] > 1e-12) & (X[:, 0] < 1 - 1e-12)
        return inner
    inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    return np.repeat(inner, 2)


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


CASES = [
    ("euler p1", dict(n=3, p=1, k_u=5, k_x=2, seed=4), 0.1),
    ("euler p2", dict(n=3, p=2, k_u=6, k_x=3, seed=5), 0.0),
    ("curved p2", dict(n=3, p=2, k_u=6, k_x=3, seed=6, q=2, curve=0.4), 0.1),
]


@pytest.mark.parametrize("name,kw,kappa", CASES)
def test_residual_and_products_match_dense_jacobians(name, kw, kappa):
    wl = W.euler_workload(**kw)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    ctx = ift.Context.from_workload(wl, kappa=kappa)
    mu = wl.mus[0]
    w = wl.w_eval
    x = wl.X.ravel() + wl.Psi @ wl.tau_eval
    U = wl.Phi @ w
    R, N, bad = O.residual(U, x, mu)
    assert bad == 0
    F = ctx.align_residual(mu, w, x)
    assert rel(F[:O.Nu], R) < 1e-12
    assert np.abs(F[O.Nu:] - N).max() <= 1e-12 * max(np.abs(N).max(), 1e-12)
    dRdU, dRdx, dNdx = O.jacobian_dense(U, x, mu)
    rng = np.random.default_rng(7)
    dU, dx = rng.normal(size=O.Nu), rng.normal(size=O.Nx)
    dF = ctx.align_jvp(mu, w, x, dU, dx)
    ref = np.concatenate([dRdU @ dU + dRdx @ dx, dNdx @ dx])
    assert rel(dF, ref) < 1e-12
    v = rng.normal(size=O.Nu + O.n_elems)
    gU, gx = ctx.align_vjp(mu, w, x, v)
    assert rel(gU, dRdU.T @ v[:O.Nu]) < 1e-12
    assert rel(gx, dRdx.T @ v[:O.Nu] + dNdx.T @ v[O.Nu:]) < 1e-12


# k_u + n_xe = 34 > 32: the element gradients span two 32-column chunks per warp
WIDE = ("euler p1 wide", dict(n=3, p=1, k_u=28, k_x=2, seed=8), 0.1)
# p = 3: n_u = 40 rows per element block
P3 = ("euler p3", dict(n=3, p=3, k_u=8, k_x=2, seed=9), 0.1)


@pytest.mark.parametrize("name,kw,kappa", [CASES[0], CASES[2], WIDE, P3])
def test_alignment_gradient_and_first_step(name, kw, kappa):
    # |J^T F| at the start over the unknowns, and the point after one step, as the oracle
    wl = W.euler_workload(**kw)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    ctx = ift.Context.from_workload(wl, kappa=kappa)
    mu = np.array([2.1, 0.01])
    mask = interior_mask(wl.X)
    r0 = O.align(wl.Phi, mu, wl.w_eval, wl.X.ravel(), mask, tol=0.0, max_iters=0)
    g0 = ctx.align(mu, wl.w_eval, wl.X.ravel(), mask, tol=0.0, max_iters=0)
    assert abs(g0["g0"] - r0["g0"]) <= 1e-10 * r0["g0"]
    assert abs(g0["J"] - r0["J"]) <= 1e-12 * r0["J"]
    r1 = O.align(wl.Phi, mu, wl.w_eval, wl.X.ravel(), mask, tol=0.0, max_iters=1)
    g1 = ctx.align(mu, wl.w_eval, wl.X.ravel(), mask, tol=0.0, max_iters=1)
    assert g1["iters"] == r1["iters"] == 1
    assert np.linalg.norm(g1["w"] - r1["w"]) <= 1e-8 * np.linalg.norm(r1["w"])
    assert np.abs(g1["x"] - r1["x"]).max() <= 1e-8


@pytest.mark.parametrize("name,kw,kappa", [CASES[0], CASES[2]])
def test_alignment_matches_the_oracle(name, kw, kappa):
    wl = W.euler_workload(**kw)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    ctx = ift.Context.from_workload(wl, kappa=kappa)
    mu = np.array([2.1, 0.01])
    mask = interior_mask(wl.X)
    # J^T F of this non-zero-residual problem is a cancellation whose rounding floor
    # lies near 1e-9 of its starting norm; 1e-7 is reached by both implementations
    tol = 1e-7
    ref = O.align(wl.Phi, mu, wl.w_eval, wl.X.ravel(), mask, tol=tol, max_iters=300)
    assert ref["status"] == 0
    g = ctx.align(mu, wl.w_eval, wl.X.ravel(), mask, tol=tol, max_iters=300)
    assert g["status"] == 0 and g["cg_iters"] > 0
    assert np.array_equal(g["x"][~mask], wl.X.ravel()[~mask])
    # the same Gauss-Newton steps up to the accuracy of the inner solves
    assert abs(g["iters"] - ref["iters"]) <= max(2, ref["iters"] // 10)
    assert abs(g["J"] - ref["J"]) <= 1e-6 * ref["J"]
    assert np.linalg.norm(g["w"] - ref["w"]) <= 1e-5 * np.linalg.norm(ref["w"])
    assert np.abs(g["x"] - ref["x"]).max() <= 1e-5
    # and the oracle finds the GPU's point stationary: its own gradient there
    U, x = wl.Phi @ g["w"], g["x"]
    R, N, _ = O.residual(U, x, mu)
    dRdU, dRdx, dNdx = O.jacobian_dense(U, x, mu)
    free = np.nonzero(mask)[0]
    gr = np.concatenate([wl.Phi.T @ (dRdU.T @ R), (dRdx.T @ R + dNdx.T @ N)[free]])
    assert np.linalg.norm(gr) <= 1.5 * tol * max(1.0, ref["g0"])


def test_known_minimum_free_stream_on_the_gpu():
    n = 3
    X, ev = W.square_tri_mesh(n)
    O = orc.Oracle(orc.PROB_EULER2D, 1, X, ev, gamma=GAMMA, kappa=0.1)
    mu = np.array([2.0, 0.02])
    Uinf = np.tile(orc.freestream(GAMMA, mu), O.Nu // 4)
    rng = np.random.default_rng(1)
    Phi, _ = np.linalg.qr(np.concatenate([Uinf[:, None], rng.normal(size=(O.Nu, 3))], axis=1))
    w_inf = Phi.T @ Uinf
    ctx = ift.Context(ift.EULER2D, 1, kappa=0.1)
    ctx.set_mesh(X, ev)
    ctx.set_bases(Phi, np.zeros((X.size, 0)))
    mask = interior_mask(X)
    x0 = X.ravel() + mask * rng.uniform(-0.05, 0.05, size=X.size) / n
    w0 = w_inf + 1e-3 * np.linalg.norm(w_inf) * rng.normal(size=4)
    g = ctx.align(mu, w0, x0, mask, tol=1e-12, max_iters=60)
    assert g["status"] == 0
    np.testing.assert_allclose(g["w"], w_inf, rtol=0, atol=1e-12 * np.linalg.norm(w_inf))
    R, _, bad = O.residual(Phi @ g["w"], g["x"], mu)
    assert bad == 0 and np.abs(R).max() <= 1e-12


def test_alignment_errors():
    wl = W.euler_workload(n=3, p=1, k_u=5, k_x=2, seed=4)
    ctx = ift.Context.from_workload(wl)
    with pytest.raises(ift.IFTError):
        ctx.align(wl.mus[0], wl.w_eval, wl.X.ravel(), interior_mask(wl.X), tol=-1.0)


@pytest.mark.parametrize("n_elems", [12, 37])
def test_alignment_burgers_first_step(n_elems):
    # 1-D: two coordinates per element, sixteen elements per warp group of the product
    # (12: one partial group; 37: 16 + 16 + 5)
    wl = W.burgers_workload(n_elems=n_elems, p=2, k_u=4, seed=3)
    O = orc.Oracle.from_workload(wl, kappa=0.1)
    ctx = ift.Context.from_workload(wl, kappa=0.1)
    mu = wl.mus[0]
    X = wl.X.ravel()
    mask = (X > 1e-12) & (X < 1 - 1e-12)
    r0 = O.align(wl.Phi, mu, wl.w_eval, X, mask, tol=0.0, max_iters=0)
    g0 = ctx.align(mu, wl.w_eval, X, mask, tol=0.0, max_iters=0)
    assert abs(g0["g0"] - r0["g0"]) <= 1e-10 * r0["g0"]
    assert abs(g0["J"] - r0["J"]) <= 1e-12 * r0["J"]
    r1 = O.align(wl.Phi, mu, wl.w_eval, X, mask, tol=0.0, max_iters=1)
    g1 = ctx.align(mu, wl.w_eval, X, mask, tol=0.0, max_iters=1)
    assert g1["iters"] == r1["iters"] == 1
    assert np.linalg.norm(g1["w"] - r1["w"]) <= 1e-8 * np.linalg.norm(r1["w"])
    assert np.abs(g1["x"] - r1["x"]).max() <= 1e-8


def test_alignment_burgers_converges_as_the_oracle():
    wl = W.burgers_workload(n_elems=12, p=2, k_u=4, seed=3)
    O = orc.Oracle.from_workload(wl, kappa=0.1)
    ctx = ift.Context.from_workload(wl, kappa=0.1)
    mu = wl.mus[0]
    X = wl.X.ravel()
    mask = (X > 1e-12) & (X < 1 - 1e-12)
    ref = O.align(wl.Phi, mu, wl.w_eval, X, mask, tol=1e-7, max_iters=300)
    assert ref["status"] == 0
    g = ctx.align(mu, wl.w_eval, X, mask, tol=1e-7, max_iters=300)
    assert g["status"] == 0
    assert abs(g["J"] - ref["J"]) <= 1e-6 * ref["J"]
    assert np.abs(g["x"] - ref["x"]).max() <= 1e-5
    assert np.linalg.norm(g["w"] - ref["w"]) <= 1e-5 * np.linalg.norm(ref["w"])


def test_alignment_state_only():
    # no free mesh coordinate: Levenberg-Marquardt on w alone, the mesh unchanged
    wl = W.euler_workload(n=3, p=1, k_u=5, k_x=2, seed=4)
    O = orc.Oracle.from_workload(wl, kappa=0.1)
    ctx = ift.Context.from_workload(wl, kappa=0.1)
    mu = np.array([2.1, 0.01])
    mask = np.zeros(wl.X.size, dtype=bool)
    ref = O.align(wl.Phi, mu, wl.w_eval, wl.X.ravel(), mask, tol=1e-9, max_iters=100)
    g = ctx.align(mu, wl.w_eval, wl.X.ravel(), mask, tol=1e-9, max_iters=100)
    assert ref["status"] == 0 and g["status"] == 0
    # near 1e-9 the stopping test sits at the rounding floor of J^T F: two FP64
    # implementations summing in different orders may stop one step apart
    assert abs(g["iters"] - ref["iters"]) <= 1
    assert np.array_equal(g["x"], wl.X.ravel())
    assert np.linalg.norm(g["w"] - ref["w"]) <= 1e-8 * np.linalg.norm(ref["w"])


def test_alignment_full_size_objective():
    # the bench's alignment (100 x 100 x 2 triangles, p = 2, k_u = 20, interior nodes free):
    # the objective at the start and after one step equals the oracle's (1/2)|F|^2 at the
    # GPU's points, the step descends, and the fixed coordinates do not move
    wl = W.euler_workload(n=100, p=2, k_u=20, k_x=4, seed=2)
    O = orc.Oracle.from_workload(wl, kappa=0.1)
    ctx = ift.Context.from_workload(wl, kappa=0.1)
    mu = wl.mus[0]
    mask = interior_mask(wl.X)
    x0 = wl.X.ravel()

    def objective(w, x):
        R, N, bad = O.residual(wl.Phi @ w, x, mu)
        assert bad == 0
        return 0.5 * (R @ R + N @ N)

    g0 = ctx.align(mu, wl.w_eval, x0, mask, tol=0.0, max_iters=0)
    J0 = objective(wl.w_eval, x0)
    assert abs(g0["J"] - J0) <= 1e-12 * J0
    g1 = ctx.align(mu, wl.w_eval, x0, mask, tol=0.0, max_iters=1)
    assert g1["iters"] == 1 and g1["cg_iters"] > 0
    J1 = objective(g1["w"], g1["x"])
    assert abs(g1["J"] - J1) <= 1e-12 * J1
    assert J1 < J0
    assert np.array_equal(g1["x"][~mask], x0[~mask])


def test_alignment_device_pointer_variant_matches_host():
    import torch

    wl = W.euler_workload(n=3, p=1, k_u=5, k_x=2, seed=4)
    ctx = ift.Context.from_workload(wl, kappa=0.1)
    mu = np.array([2.1, 0.01])
    mask = interior_mask(wl.X)
    h = ctx.align(mu, wl.w_eval, wl.X.ravel(), mask, tol=1e-9, max_iters=20)
    dev = torch.device("cuda", 0)
    t = lambda a, dt=torch.float64: torch.as_tensor(np.asarray(a), dtype=dt, device=dev).clone()
    # inputs produced on a stream of their own, which the call is given
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        w, x = t(wl.w_eval), t(wl.X.ravel())
        d = ctx.align_dev(t(mu), w, x, t(mask, torch.uint8), tol=1e-9, max_iters=20, stream=side.cuda_stream)
    torch.cuda.synchronize()
    assert d["status"] == h["status"] and d["iters"] == h["iters"] and d["cg_iters"] == h["cg_iters"]
    np.testing.assert_array_equal(w.cpu().numpy(), h["w"])
    np.testing.assert_array_equal(x.cpu().numpy(), h["x"])
    assert d["J"] == h["J"]


def test_inexact_cg_steps_reach_the_same_point():
    # align_cg_tol = 1e-2: inexact Levenberg-Marquardt steps, the same stopping test on
    # |J^T F|, so the aligned point is the oracle's (exact-step) one
    name, kw, kappa = CASES[0]
    wl = W.euler_workload(**kw)
    O = orc.Oracle.from_workload(wl, kappa=kappa)
    mu = np.array([2.1, 0.01])
    mask = interior_mask(wl.X)
    ref = O.align(wl.Phi, mu, wl.w_eval, wl.X.ravel(), mask, tol=1e-7, max_iters=300)
    exact = ift.Context.from_workload(wl, kappa=kappa).align(mu, wl.w_eval, wl.X.ravel(), mask, tol=1e-7,
                                                              max_iters=300)
    loose = ift.Context.from_workload(wl, kappa=kappa, align_cg_tol=1e-2).align(mu, wl.w_eval, wl.X.ravel(), mask,
                                                                                 tol=1e-7, max_iters=300)
    assert ref["status"] == 0 and exact["status"] == 0 and loose["status"] == 0
    assert loose["cg_iters"] < exact["cg_iters"]
    assert abs(loose["J"] - ref["J"]) <= 1e-6 * ref["J"]
    assert np.abs(loose["x"] - ref["x"]).max() <= 1e-5
    assert np.linalg.norm(loose["w"] - ref["w"]) <= 1e-5 * np.linalg.norm(ref["w"])


def test_align_cg_tol_is_validated():
    with pytest.raises(ift.IFTError):
        ift.Context(ift.EULER2D, 1, align_cg_tol=1.0)
    with pytest.raises(ift.IFTError):
        ift.Context(ift.EULER2D, 1, align_cg_tol=-1e-3)
