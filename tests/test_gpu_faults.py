"""Failure handling with injected bad inputs (made on the host; nothing here faults,
traps or hangs the GPU): every bad input comes back as a status, and the context
stays usable for the next good call."""

import ctypes

import numpy as np
import pytest

from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(**kw):
    wl = W.euler_workload(n=6, p=1, k_u=5, k_x=2, seed=61, n_mu=4, mu_box=True)
    return wl, ift.Context.from_workload(wl, **kw)


def test_nan_parameter_is_nonphysical_and_context_recovers():
    wl, ctx = _ctx()
    bad = np.array([np.nan, 0.0])
    g = ctx.reduced_residual_jacobian(bad, wl.w_eval, wl.tau_eval)
    assert g["status"] == -5 and np.isinf(g["J"])
    r = ctx.solve_rom(bad)
    assert r["status"] == -5
    # the next good calls are unaffected
    good = ctx.solve_rom(wl.mus[0])
    assert good["status"] == 0


def test_non_finite_point_is_nonphysical():
    wl, ctx = _ctx()
    w = wl.w_eval.copy()
    w[1] = np.inf
    g = ctx.reduced_residual_jacobian(wl.mus[0], w, wl.tau_eval)
    assert g["status"] == -5 and np.isinf(g["J"])
    z = wl.tau_eval.copy()
    z[0] = np.nan
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, z)
    assert g["status"] == -5
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    assert g["status"] == 0 and np.isfinite(g["J"])


def test_inverting_mesh_motion_is_nonphysical():
    # a mesh-motion amplitude that folds triangles: g <= 0 is reported, not used
    wl, ctx = _ctx()
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, 1e3 * wl.tau_eval)
    assert g["status"] == -5


def test_bad_weights_rejected():
    wl, ctx = _ctx()
    for elems, rho in (([0, 1], [1.0, np.nan]), ([0, 1], [1.0, 0.0]), ([0, wl.n_elems], [1.0, 1.0]),
                       ([-1], [1.0])):
        with pytest.raises(ift.IFTError) as ei:
            ctx.set_eq_weights((np.array(elems), np.array(rho)))
        assert ei.value.status == -1
    # rejected weights leave the previous ones in place
    g = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    assert g["status"] == 0


def test_batched_query_with_nan_parameter_does_not_stop_the_others():
    wl, ctx = _ctx(tol=1e-8)
    sets = W.eq_weight_sets(wl, 4, seed=62, lo=40, hi=60)
    ctx.set_eq_weights_batched(sets)
    mus = wl.mus.copy()
    mus[2, 0] = np.nan
    res = ctx.solve_rom_batched(mus)
    st = [i["status"] for i in res["info"]]
    assert st[2] == -5
    assert res["status"] == -5
    assert all(s in (0, 1, 2) for q, s in enumerate(st) if q != 2)
    # and the same context solves the good batch afterwards
    res2 = ctx.solve_rom_batched(wl.mus)
    assert all(i["status"] in (0, 1, 2) for i in res2["info"])


def test_zero_iterations_reports_not_converged():
    wl, ctx = _ctx(max_iters=0, tol=1e-14)
    r = ctx.solve_rom(wl.mus[0])
    assert r["status"] == 1 and r["iters"] == 0


def test_bad_sizes_rejected():
    wl, ctx = _ctx()
    with pytest.raises(ift.IFTError):
        ctx.set_bases(wl.Phi[:-1], wl.Psi)
    with pytest.raises(ift.IFTError):
        ctx.set_bases(np.zeros((wl.Phi.shape[0], 65)), wl.Psi)  # k_u + k_x > 64
    with pytest.raises(ift.IFTError):
        ift.MLP(2, 8, 17, 3)


def test_loop_body_bound_ends_solve_with_timeout_and_context_recovers():
    # The device loop of a solve is bounded by a count of loop bodies kept by the LM
    # step kernel (no wait or spin on the device). A bound of 3 bodies ends the solve
    # long before it converges; the status is IFT_ERR_TIMEOUT and the same context
    # then evaluates exactly as a fresh one.
    wl = W.euler_workload(n=6, p=1, k_u=5, k_x=2, seed=61)
    ctx = ift.Context.from_workload(wl, max_loop_bodies=3)
    with pytest.raises(ift.IFTError) as ei:
        ctx.solve_rom(wl.mus[0])
    assert ei.value.status == -6
    fresh = ift.Context.from_workload(wl)
    a = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    b = fresh.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    assert a["status"] == 0
    np.testing.assert_array_equal(a["H"], b["H"])
    assert a["J"] == b["J"]
    full = fresh.solve_rom(wl.mus[0])
    assert full["status"] == 0 and full["init_iters"] + full["iters"] > 3
    # a batched solve under the same bound: every query ends with the same status
    sets = W.eq_weight_sets(wl, 3, seed=62, lo=20, hi=40)
    ctx.set_eq_weights_batched(sets)
    mus = np.ascontiguousarray(np.stack([wl.mus[0]] * 3))
    y, z = np.zeros(3 * wl.ku), np.zeros(3 * wl.kx)
    info = (ift.SolveInfo * 3)()
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = ift.load().ift_solve_rom_batched(ctx._h, P(mus), P(y), P(z), info)
    assert st == -6 and all(i.status == -6 for i in info)
    assert ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)["status"] == 0


def test_negative_loop_body_bound_is_rejected():
    with pytest.raises(ift.IFTError) as ei:
        _ctx(max_loop_bodies=-1)
    assert ei.value.status == -1
