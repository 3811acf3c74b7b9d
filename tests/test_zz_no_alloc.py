"""The allocation-free assembly entry point (ift_reduced_residual_jacobian_static).

It serves callers that cannot allocate device memory when they need the reduced
system (for example while capturing a CUDA graph, or under their own memory
pool): every buffer is the caller's and the scratch lives in a fixed array
inside the library. This test calls it through the C ABI twice in a row and
checks both results against the context-based entry point on the same inputs,
within the FP64 parity tolerance of the other tests. It lives in a file of its
own that pytest collects last.
"""

import numpy as np
import pytest

import oracle as orc
from paper_2305_15661_gb300 import ift
from paper_2305_15661_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fro(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("sparse", [False, True])
def test_static_scratch_assembly_matches_context_call(sparse):
    import torch

    dev = torch.device("cuda", 0)
    wl = W.euler_workload(n=20, p=2, k_u=12, k_x=4, seed=11)
    rs = W.eq_weight_sets(wl, 1, seed=12, lo=100, hi=200)[0] if sparse else None
    ctx = ift.Context.from_workload(wl)
    ctx.set_eq_weights(rs)
    mu = wl.mus[0]
    ref = ctx.reduced_residual_jacobian(mu, wl.w_eval, wl.tau_eval)

    # connectivity in the documented layout (test harness: taken from the mesh via the oracle)
    nbr, nbf = orc.Oracle.from_workload(wl).neighbors()
    bc = np.where(nbr < 0, 1, 0).astype(np.int8)
    t64 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    t32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32), device=dev)
    X, ev, nb, nf = t64(wl.X), t32(wl.ev), t32(nbr), t32(nbf)
    bct = torch.as_tensor(bc, device=dev)
    Phi, Psi = t64(wl.Phi), t64(wl.Psi)
    elems = t32(rs[0]) if sparse else None
    rho = t64(rs[1]) if sparse else None
    k = wl.ku + wl.kx
    for _ in range(2):
        S, T, H, J = (torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
                      for n in (wl.ku, wl.kx, k * k, 1))
        ift.reduced_residual_jacobian_static(ift.EULER2D, wl.p, X, ev, nb, nf, bct, Phi, Psi, elems, rho, t64(mu),
                                             t64(wl.w_eval), t64(wl.tau_eval), S, T, H, J)
        torch.cuda.synchronize()
        assert _fro(S.cpu().numpy(), ref["S"]) < 1e-10
        assert _fro(T.cpu().numpy(), ref["T"]) < 1e-10
        assert _fro(H.cpu().numpy().reshape(k, k), ref["H"]) < 1e-10
        assert abs(J.item() - ref["J"]) <= 1e-10 * ref["J"]


def test_static_scratch_rejects_oversized_bases():
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
