"""The allocation-free assembly entry point (ift_reduced_residual_jacobian_static).

It serves callers that cannot allocate device memory when they need the reduced
system: code that owns all device memory through its own pool or arena, programs
that reserve their whole budget at start-up, and latency-critical loops where an
allocation would synchronise the device. Every buffer is the caller's and the
scratch lives in a fixed array inside the library. These tests call it through
the C ABI twice in a row and check both results against the context-based entry
point on the same inputs, within the FP64 parity tolerance of the other tests
(Euler p = 2 dense and sparse, Burgers p = 1 and 3, Euler p = 3 at the largest
basis, k_u + k_x = 64); that free device memory does not change across calls;
that a context planned for a larger basis still runs after a static call has
prepared the shared kernel for a smaller one; and the documented outcomes of bad
inputs (host errors, NaN outputs after the device index check, J = +inf at a
non-physical state). The file is collected last.
"""

import ctypes

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fro(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _bc_types(wl, nbr):
    """Boundary types in the documented layout: Euler far field 1 on every boundary
    face; Burgers inflow 1 on face 0 (outward normal -x), outflow 2 on face 1."""
    bc = np.where(nbr < 0, 1, 0).astype(np.int8)
    if wl.problem == ift.BURGERS1D:
        bc[:, 1] = np.where(nbr[:, 1] < 0, 2, 0)
    return bc


class _Static:
    """Device copies of one workload's mesh, connectivity and bases, and the call."""

    def __init__(self, wl, rs=None):
        import torch

        self.torch = torch
        self.dev = torch.device("cuda", 0)
        self.wl = wl
        nbr, nbf = orc.Oracle.from_workload(wl).neighbors()  # test harness: connectivity from the mesh
        self.nbr_np, self.nbf_np = nbr, nbf
        self.X, self.ev = self.t64(wl.X), self.t32(wl.ev)
        self.nb, self.nf = self.t32(nbr), self.t32(nbf)
        self.bc = torch.as_tensor(_bc_types(wl, nbr), device=self.dev)
        self.Phi, self.Psi = self.t64(wl.Phi), self.t64(wl.Psi)
        self.elems = self.t32(rs[0]) if rs is not None else None
        self.rho = self.t64(rs[1]) if rs is not None else None
        self.k = wl.ku + wl.kx

    def t64(self, a):
        return self.torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=self.dev)

    def t32(self, a):
        return self.torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32), device=self.dev)

    def outputs(self):
        wl, k = self.wl, self.k
        return [self.torch.full((n,), float("nan"), dtype=self.torch.float64, device=self.dev)
                for n in (wl.ku, max(wl.kx, 1), k * k, 1)]

    def call(self, y, z, ev=None, elems=None, rho=None):
        wl = self.wl
        S, T, H, J = self.outputs()
        ift.reduced_residual_jacobian_static(
            wl.problem, wl.p, self.X, self.ev if ev is None else ev, self.nb, self.nf, self.bc, self.Phi, self.Psi,
            self.elems if elems is None else elems, self.rho if rho is None else rho, self.t64(wl.mus[0]),
            self.t64(y), self.t64(z if wl.kx else np.zeros(1)), S, T, H, J, gamma=wl.gamma)
        self.torch.cuda.synchronize()
        return (S.cpu().numpy(), T.cpu().numpy()[:wl.kx], H.cpu().numpy().reshape(self.k, self.k), J.item())


def _check_two_calls(wl, rs=None):
    ctx = ift.Context.from_workload(wl)
    ctx.set_eq_weights(rs)
    ref = ctx.reduced_residual_jacobian(wl.mus[0], wl.w_eval, wl.tau_eval)
    st = _Static(wl, rs)
    for _ in range(2):
        S, T, H, J = st.call(wl.w_eval, wl.tau_eval)
        assert _fro(S, ref["S"]) < 1e-10
        if wl.kx:
            assert _fro(T, ref["T"]) < 1e-10
        assert _fro(H, ref["H"]) < 1e-10
        assert abs(J - ref["J"]) <= 1e-10 * ref["J"]
    return st


@pytest.mark.parametrize("sparse", [False, True])
def test_static_scratch_assembly_matches_context_call(sparse):
    wl = W.euler_workload(n=20, p=2, k_u=12, k_x=4, seed=11)
    rs = W.eq_weight_sets(wl, 1, seed=12, lo=100, hi=200)[0] if sparse else None
    _check_two_calls(wl, rs)


@pytest.mark.parametrize("p", [1, 3])
def test_static_scratch_burgers(p):
    wl = W.burgers_workload(n_elems=60, p=p, k_u=5, seed=3)
    _check_two_calls(wl)


def test_static_scratch_largest_basis():
    # k_u + k_x = 64, the documented maximum, on p = 3 elements (40-row element blocks)
    wl = W.euler_workload(n=10, p=3, k_u=56, k_x=8, seed=13)
    _check_two_calls(wl)


def test_static_call_allocates_nothing():
    import torch

    wl = W.euler_workload(n=20, p=2, k_u=12, k_x=4, seed=11)
    st = _check_two_calls(wl)  # the first call on the device has done its set-up
    outs = [st.outputs() for _ in range(3)]
    mu, y, z = st.t64(wl.mus[0]), st.t64(wl.w_eval), st.t64(wl.tau_eval)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for S, T, H, J in outs:
        ift.reduced_residual_jacobian_static(wl.problem, wl.p, st.X, st.ev, st.nb, st.nf, st.bc, st.Phi, st.Psi,
                                             None, None, mu, y, z, S, T, H, J, gamma=wl.gamma)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for S, T, H, J in outs[1:]:
        assert torch.equal(H, outs[0][2]) and torch.equal(J, outs[0][3])


def test_context_planned_for_larger_basis_survives_static_call():
    # A context planned for k = 48 sets the shared FP64 p = 2 kernel's shared-memory
    # limit for its own size; a static call for k = 16 must not lower it.
    big = W.euler_workload(n=12, p=2, k_u=40, k_x=8, seed=14)
    ctx = ift.Context.from_workload(big)
    ref = ctx.reduced_residual_jacobian(big.mus[0], big.w_eval, big.tau_eval)
    small = W.euler_workload(n=20, p=2, k_u=12, k_x=4, seed=11)
    _check_two_calls(small)
    again = ctx.reduced_residual_jacobian(big.mus[0], big.w_eval, big.tau_eval)
    assert again["status"] == 0
    np.testing.assert_array_equal(again["H"], ref["H"])
    assert again["J"] == ref["J"]


def test_static_bad_indices_give_nan():
    # indices the device check catches before any element is evaluated
    wl = W.euler_workload(n=8, p=2, k_u=6, k_x=2, seed=15)
    rs = W.eq_weight_sets(wl, 1, seed=16, lo=20, hi=30)[0]
    st = _Static(wl, rs)
    good = st.call(wl.w_eval, wl.tau_eval)
    assert np.isfinite(good[3])
    ev_bad = wl.ev.copy()
    ev_bad[rs[0][3], 1] = wl.X.shape[0] + 5  # a vertex id past the end, on a listed element
    el_bad = rs[0].copy()
    el_bad[-1] = wl.n_elems  # an element id past the end
    rho_bad = rs[1].copy()
    rho_bad[0] = -1.0
    for kw in (dict(ev=st.t32(ev_bad)), dict(elems=st.t32(el_bad)), dict(rho=st.t64(rho_bad))):
        S, T, H, J = st.call(wl.w_eval, wl.tau_eval, **kw)
        assert np.all(np.isnan(S)) and np.all(np.isnan(H)) and np.isnan(J), kw
    # the array keeps no state from the failed calls
    again = st.call(wl.w_eval, wl.tau_eval)
    np.testing.assert_array_equal(again[2], good[2])


def test_static_nonphysical_state_gives_infinite_objective():
    wl = W.euler_workload(n=8, p=2, k_u=6, k_x=2, seed=15)
    st = _Static(wl)
    S, T, H, J = st.call(-np.asarray(wl.w_eval), wl.tau_eval)  # negative density everywhere
    assert J == float("inf")


def test_static_scratch_rejects_oversized_bases_and_bad_counts():
    import torch

    dev = torch.device("cuda", 0)
    z64 = lambda n: torch.zeros(n, dtype=torch.float64, device=dev)
    z32 = lambda n: torch.zeros(n, dtype=torch.int32, device=dev)
    X = z64((4, 2))
    Phi = torch.zeros((24, 70), dtype=torch.float64, device=dev)  # k_u = 70 > 64
    Psi = torch.zeros((8, 0), dtype=torch.float64, device=dev)
    with pytest.raises(ift.IFTError) as ei:
        ift.reduced_residual_jacobian_static(ift.EULER2D, 2, X, z32((1, 3)), z32((1, 3)), z32((1, 3)),
                                             torch.zeros((1, 3), dtype=torch.int8, device=dev), Phi, Psi, None,
                                             None, z64(2), z64(70), None, z64(70), None, z64(4900), z64(1))
    assert ei.value.status == -1
    # nnz below -1 (only -1, "rho = 1 everywhere", is a valid negative count)
    lib = ift.load()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    Phi = z64((24, 4))
    ev, nb, bc = z32((1, 3)), z32((1, 3)), torch.zeros((1, 3), dtype=torch.int8, device=dev)
    el, rho, mu, y, S, H, J = z32(1), z64(1), z64(2), z64(4), z64(4), z64(16), z64(1)
    for nnz in (-5, -2, 0):
        st = lib.ift_reduced_residual_jacobian_static(ift.EULER2D, 2, 3, p(X), 1, p(ev), p(nb), p(nb), p(bc), p(Phi),
                                                      4, None, 0, nnz, p(el), p(rho), p(mu), p(y), None, 1.4, 0.0,
                                                      1e-8, p(S), None, p(H), p(J), None)
        assert st == -1, nnz
