"""Algorithmic work per element of the hot path, for roofline accounting.

One fused multiply-add counts as 2 FLOPs; +, -, *, /, sqrt and exp count 1.

The nonlinear pointwise routines are counted, not estimated: their values and
one forward-mode derivative direction each were counted on an
operation-counting instantiation of the independent FP64 implementation
(``python -m oracle.workcount`` writes the constants below; a CPU test checks
them). Everything else is linear algebra on the reference element, counted in
closed form from its sizes (n_b nodes, n_q volume points, n_f faces of n_fq
points, n_t trace nodes per face, m variables, d dimensions, n_u = n_b m,
n_u' = n_f n_t m neighbour trace values, n_x = (d + 1) d mesh coordinates).

Per element of the fused assembly (Eqs. hdm_elem, levmarq-elem, ift-eqp-res0):

* reconstruction U_e = Phi_e w, U_e' = Phi_e' w, x_e = X_e + Psi_e tau:
  2 (n_u + n_u') k_u + 2 n_x k_x;
* the residual R_e: per volume point the interpolation 2 n_b m, the flux and
  its contravariant form g f G^{-T} (2 d^2 m), the test sums 2 n_q d n_b m;
  per face point the two traces 4 n_t m, the Roe flux, the lifting 2 n_t m;
* the pointwise Jacobians, once per point: m derivative directions of the flux
  at every volume point, m along U+ and m along U- of the Roe flux at every
  face point;
* the state columns of A_e = [dR_e/dU_e Phi_e + dR_e/dU_e' Phi_e' | ...], the
  volume part and the face part each by the cheaper of two standard forms:
  - volume, explicit: the block dR_e/dU_e formed through the flux Jacobians,
    per point n_q (2 d n_b m^2 + 2 n_b^2 m^2) (the test against D first, then the
    basis B), then the product with Phi_e, 2 n_u^2 k_u;
  - volume, directional: per column the interpolation, the pointwise Jacobians
    applied (2 d m^2 per point), the contravariant form and the test sums;
  - faces, explicit: per face point the two trace blocks (4 n_t^2 m^2, the
    interior one added into dR_e/dU_e before its product), and per face the
    neighbour block's product with the neighbour's trace rows, 2 (n_t m)^2 k_u;
  - faces, directional: per column and face point the traces, the two Roe
    Jacobians applied (4 m^2) and the lifting;
  - faces, mixed: the interior trace's block (2 n_t^2 m^2 per face point) added
    into dR_e/dU_e before its product, and per column and face point only the
    neighbour's trace, dH/dU- applied (2 m^2) and the lifting;
* the mesh columns dR_e/dx_e Psi_e by the cheaper of: per direction the
  contravariant change of the volume flux (2 d^2 m per point) with the test
  sums and the scaled-normal change of the face flux (2 d m per face point) with
  the lifting, along the k_x columns; or the quadrature sum taken once,
  E = 2 n_q n_b m d^2, then per column 2 n_u d^2 for the volume and the face
  terms as before;
* the weighted contraction: the symmetric A_e^T A_e (n_u k (k + 1): k (k + 1) / 2
  dot products of length n_u), A_e^T R_e (2 n_u k) and |R_e|^2 (2 n_u).

The geometry (a few dozen operations per element), the distortion term (kappa
= 0 in the benchmark) and the weight multiplies are not counted, so the count
is a lower bound on the work any implementation of the assembly does.

Bytes per element of the full assembly (unique data): the element's Phi rows
n_u k_u words, the Psi rows of its vertices n_x k_x, X_e and the connectivity;
neighbour trace rows are counted once overall because every element's rows
are read by its neighbours too (they hit in L2). The hyperreduced gather of a
sampled element reads its own Phi rows and its neighbours' trace rows:
(n_u + n_u') k_u words.
"""

from __future__ import annotations

# Counted by oracle/workcount.py (value, derivative along one direction):
EULER_FLUX = (19, 41)  # f(U)
EULER_ROE = (203, 262, 262)  # H(U+, U-; n): value, along U+, along U-
BURGERS_ROE = (17, 15)  # H(u+, u-; n): value, along u+
# Burgers flux u^2/2 (2 value operations, 1 per derivative direction) and source
# g 0.5 exp(mu x(xi)) with x(xi) = x_0 + h xi (5 value operations): closed forms.
BURGERS_FLUX = (2, 1)
BURGERS_SOURCE = 5


def sizes(problem: int, p: int):
    if problem == 1:
        m, d, nb, nq, nf, nt, nfq, nv = 1, 1, p + 1, p + 2, 2, 1, 1, 2
    else:
        m, d, nb, nq, nf, nt, nfq, nv = 4, 2, (p + 1) * (p + 2) // 2, (p + 2) ** 2, 3, p + 1, p + 2, 3
    return dict(m=m, d=d, nb=nb, nq=nq, nf=nf, nt=nt, nfq=nfq, nv=nv, nu=nb * m, nup=nf * nt * m, nx=nv * d)


def flops_per_element(problem: int, p: int, ku: int, kx: int, jac: bool = True) -> dict:
    """Algorithmic FLOPs of one element of the fused assembly (jac=True) or of the
    residual-only pass (jac=False), with the breakdown by part."""
    s = sizes(problem, p)
    m, d, nb, nq, nf, nt, nfq = s["m"], s["d"], s["nb"], s["nq"], s["nf"], s["nt"], s["nfq"]
    nu, nup, nx = s["nu"], s["nup"], s["nx"]
    k = ku + kx
    nfp = nf * nfq  # face points
    if problem == 1:
        fval, ftan = BURGERS_FLUX
        hval, htan_p = BURGERS_ROE
        htan_m = htan_p
        src = BURGERS_SOURCE + 2 * nb * m  # the source and its test sum, per volume point
    else:
        fval, ftan = EULER_FLUX
        hval, htan_p, htan_m = EULER_ROE
        src = 0
    test = 2 * nq * d * nb * m
    out = {"reconstruction": 2 * (nu + nup) * ku + 2 * nx * kx}
    out["residual"] = (nq * (2 * nb * m + fval + 2 * d * d * m + src) + test
                       + nfp * (4 * nt * m + hval + 2 * nt * m))
    out["objective"] = 2 * nu
    if jac:
        out["pointwise_jacobians"] = nq * m * ftan + nfp * m * (htan_p + htan_m)
        vol_explicit = nq * (2 * d * nb * m * m + 2 * nb * nb * m * m) + 2 * nu * nu * ku
        vol_directional = ku * (nq * (2 * nb * m + 2 * d * m * m + 2 * d * d * m) + test)
        face_explicit = nfp * 4 * nt * nt * m * m + nf * 2 * (nt * m) ** 2 * ku
        face_directional = ku * nfp * (4 * nt * m + 4 * m * m + 2 * nt * m)
        face_mixed = nfp * 2 * nt * nt * m * m + ku * nfp * (2 * nt * m + 2 * m * m + 2 * nt * m)
        faces = {"explicit": face_explicit, "directional": face_directional, "mixed": face_mixed}
        face_form = min(faces, key=faces.get)
        out["state_columns"] = min(vol_explicit, vol_directional) + faces[face_form]
        out["state_columns_form"] = ("volume " + ("explicit" if vol_explicit <= vol_directional else "directional")
                                     + ", faces " + face_form)
        face_dir = nfp * (2 * d * m + 2 * nt * m)
        per_dir = nq * 2 * d * d * m + test + face_dir
        via_e = 2 * nq * nb * m * d * d + kx * (2 * nu * d * d + face_dir)
        out["mesh_columns"] = min(kx * per_dir, via_e) if kx > 0 else 0
        out["contraction"] = nu * k * (k + 1) + 2 * nu * k
    parts = [v for key, v in out.items() if key != "state_columns_form"]
    out["total"] = sum(parts)
    # the two halves the benchmark reports: the element evaluation (residual and
    # pointwise Jacobians) and the reduction to the k x k system
    out["element"] = out["residual"] + out.get("pointwise_jacobians", 0)
    out["reduction"] = out["total"] - out["element"]
    return out


def bytes_per_element(problem: int, p: int, ku: int, kx: int, word: int = 8) -> int:
    s = sizes(problem, p)
    return s["nu"] * ku * word + s["nv"] * s["d"] * (kx * 8 + 8) + s["nv"] * 4 + s["nf"] * 9


def gather_bytes_per_element(problem: int, p: int, ku: int, word: int = 8) -> int:
    """Basis rows a hyperreduced evaluation of one sampled element reads: its own
    Phi rows and its neighbours' trace rows."""
    s = sizes(problem, p)
    return (s["nu"] + s["nup"]) * ku * word
