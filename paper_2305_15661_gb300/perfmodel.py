"""Algorithmic work per element of the hot path, for roofline accounting.

The count follows the explicit formulation of the method (Eqs. hdm_elem,
levmarq-elem, ift-eqp-res0): form R_e, the element Jacobian blocks
dR_e/dU_e, dR_e/dU_e', dR_e/dx_e, the reduced Jacobian A_e = [dR_e/dU_e Phi_e +
dR_e/dU_e' Phi_e' | dR_e/dx_e Psi_e] and the weighted contraction
A_e^T A_e, A_e^T R_e, |R_e|^2. One fused multiply-add counts as 2 FLOPs.

(a) element residual and Jacobians, per element:
    volume, per quadrature point: interpolation 2 n_b m, flux C_f, flux
    Jacobian C_A, contravariant flux 2 d^2 m and Jacobian 2 d^2 m^2;
    volume test 2 n_q d n_b m; volume Jacobian block 2 n_q d n_b^2 m^2;
    faces, per face point: two traces 4 n_t m, Roe flux C_roe and its 8 state
    derivatives 8 C_roe, test 2 n_t m, face Jacobian blocks 4 n_t^2 m^2.
(b) reduction (the contraction count of Eq. levmarq-elem plus g and J):
    2 n_u k_u (n_u + n_u') + 2 n_u k_x n_x + n_u k (k + 1) + 2 n_u k + 2 n_u,
    where n_u k (k + 1) is the symmetric product A_e^T A_e (its k (k + 1) / 2
    distinct entries, each a length-n_u dot product).
C_f = 20, C_A = 40, C_roe = 200 for Euler (operation counts of the pointwise
routines); Burgers: C_f = 1, C_A = 0, C_roe = 12, plus the source
(exp and 4 flops per point).

Bytes per element of the full assembly (unique data): the element's Phi rows
n_u k_u words, the Psi rows of its vertices n_x k_x, X_e and the connectivity;
neighbour trace rows are counted once overall because every element's rows
are read by its neighbours too (they hit in L2).
"""

from __future__ import annotations


def sizes(problem: int, p: int):
    if problem == 1:
        m, d, nb, nq, nf, nt, nfq, nv = 1, 1, p + 1, p + 2, 2, 1, 1, 2
    else:
        m, d, nb, nq, nf, nt, nfq, nv = 4, 2, (p + 1) * (p + 2) // 2, (p + 2) ** 2, 3, p + 1, p + 2, 3
    return dict(m=m, d=d, nb=nb, nq=nq, nf=nf, nt=nt, nfq=nfq, nv=nv, nu=nb * m, nup=nf * nt * m, nx=nv * d)


def flops_per_element(problem: int, p: int, ku: int, kx: int, jac: bool = True) -> dict:
    s = sizes(problem, p)
    m, d, nb, nq, nf, nt, nfq = s["m"], s["d"], s["nb"], s["nq"], s["nf"], s["nt"], s["nfq"]
    nu, nup, nx = s["nu"], s["nup"], s["nx"]
    k = ku + kx
    if problem == 1:
        cf, ca, croe, csrc = 1, 0, 12, 5
    else:
        cf, ca, croe, csrc = 20, 40, 200, 0
    recon = 2 * (nu + nup) * ku + 2 * nx * kx
    vol_res = nq * (2 * nb * m + cf + 2 * d * d * m + csrc) + 2 * nq * d * nb * m
    face_res = nf * nfq * (4 * nt * m + croe + 2 * nt * m)
    a = recon + vol_res + face_res
    b = 2 * nu  # |R|^2
    if jac:
        a += nq * (ca + 2 * d * d * m * m) + 2 * nq * d * nb * nb * m * m
        a += nf * nfq * (8 * croe + 4 * nt * nt * m * m)
        b += 2 * nu * ku * (nu + nup) + 2 * nu * kx * nx + nu * k * (k + 1) + 2 * nu * k
    return {"element": a, "reduction": b, "total": a + b}


def bytes_per_element(problem: int, p: int, ku: int, kx: int, word: int = 8) -> int:
    s = sizes(problem, p)
    return s["nu"] * ku * word + s["nv"] * s["d"] * (kx * 8 + 8) + s["nv"] * 4 + s["nf"] * 9
