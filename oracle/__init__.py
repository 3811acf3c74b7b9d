"""FP64 CPU oracle for the EQP-IFT hot path (arXiv 2305.15661).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers. The CUDA library never
imports, links or runs anything here, and this package never touches the CUDA
library. The arithmetic lives in ``ift_oracle.cpp``; this module only marshals
arguments through ctypes and adds the global-assembly helpers the pins need.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ift_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

PROB_BURGERS1D = 1
PROB_EULER2D = 2
BC_DEFAULT = 0
BC_SHEAR_TEST = 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (g++, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        cmd = ["g++", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c++17", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
        pd, pi, pl = P(d), P(i), P(l)
        vp = ctypes.c_void_p
        sig = {
            "orc_create": (vp, [i, i, l, pd, l, pi, d, d, d, i, i]),
            "orc_destroy": (None, [vp]),
            "orc_sizes": (None, [vp, pl]),
            "orc_neighbors": (None, [vp, pi, pi]),
            "orc_ref_nodes": (None, [vp, pd, pi]),
            "orc_ref_quadrature": (None, [vp, pd, pd, pd, pd]),
            "orc_ref_basis": (None, [vp, i, pd, pd, pd]),
            "orc_gauss_legendre": (None, [i, pd, pd]),
            "orc_euler_flux": (None, [d, pd, pd, pd]),
            "orc_euler_roe": (None, [d, pd, pd, pd, pd]),
            "orc_burgers_roe": (d, [d, d, d]),
            "orc_freestream": (None, [d, pd, pd]),
            "orc_element": (i, [vp, l, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd]),
            "orc_element_physical": (None, [vp, l, pd, pd, pd, pd, pd]),
            "orc_gather": (None, [vp, pd, pd, l, pd, pd, pd]),
            "orc_gather_rows": (None, [vp, i, pd, i, pd, l, pd, pd, pd]),
            "orc_global_residual": (i, [vp, pd, pd, pd, pd, pd]),
            "orc_global_jacobian": (i, [vp, pd, pd, pd, pd, pd, pd]),
            "orc_reduced": (i, [vp, i, pd, i, pd, l, pi, pd, pd, pd, pd, pd, pd, pd, pd, i]),
            "orc_objective": (i, [vp, i, pd, i, pd, l, pi, pd, pd, pd, pd, pd, i]),
            "orc_solve": (i, [vp, i, pd, i, pd, l, pi, pd, pd, pd, pd, i, d, i, pd, pd, pd, pd, pi, i, pd, pi]),
            "orc_num_threads": (i, []),
            "orc_count_element": (i, [vp, l, pd, pd, pd, pd, pd, pd, pd, ctypes.POINTER(ctypes.c_longlong)]),
            "orc_count_pointwise": (None, [vp, i, pd, pd, pd, pd, ctypes.POINTER(ctypes.c_longlong)]),
            "orc_shear_state": (None, [d, d, d, pd]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _pd(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def gauss_legendre(n: int):
    lib = _load()
    x = np.zeros(n)
    w = np.zeros(n)
    lib.orc_gauss_legendre(n, _pd(x), _pd(w))
    return x, w


def euler_flux(gamma, U):
    lib = _load()
    U = _f64(U)
    f = np.zeros(8)
    P = np.zeros(1)
    lib.orc_euler_flux(gamma, _pd(U), _pd(f), _pd(P))
    return f.reshape(4, 2), float(P[0])


def euler_roe(gamma, Up, Um, n):
    lib = _load()
    H = np.zeros(4)
    lib.orc_euler_roe(gamma, _pd(_f64(Up)), _pd(_f64(Um)), _pd(_f64(n)), _pd(H))
    return H


def burgers_roe(up, um, n):
    return float(_load().orc_burgers_roe(up, um, n))


def shear_state(gamma, x, y):
    U = np.zeros(4)
    _load().orc_shear_state(gamma, x, y, _pd(U))
    return U


def freestream(gamma, mu):
    U = np.zeros(4)
    _load().orc_freestream(gamma, _pd(_f64(mu)), _pd(U))
    return U


class Oracle:
    """One problem instance: mesh, reference element and connectivity."""

    def __init__(self, problem, p, X, ev, gamma=1.4, kappa=0.0, eps=1e-8, bc_mode=BC_DEFAULT, q=1):
        """q: geometry degree, 1 (straight-sided, ev = vertices) or 2 (2-D curved, ev = the
        three vertices then the midpoint nodes of edges 0-1, 1-2, 2-0)."""
        lib = _load()
        self.problem = problem
        self.p = p
        self.q = q
        self.X = _f64(X)
        self.ev = np.ascontiguousarray(ev, dtype=np.int32)
        self.dim = 1 if problem == PROB_BURGERS1D else 2
        self.m = 1 if problem == PROB_BURGERS1D else 4
        n_verts = self.X.shape[0]
        n_elems = self.ev.shape[0]
        self._h = lib.orc_create(problem, p, n_verts, _pd(self.X), n_elems, _pi(self.ev), gamma, kappa, eps,
                                 bc_mode, q)
        if not self._h:
            raise ValueError("oracle: bad problem, degree or mesh")
        s = np.zeros(10, dtype=np.int64)
        lib.orc_sizes(self._h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_long)))
        (self.nb, self.nu, self.nup, self.nxe, self.nq, self.nfq, self.ntrace, self.nface, self.Nu,
         self.Nx) = [int(v) for v in s]
        self.n_elems = n_elems
        self.n_verts = n_verts

    @classmethod
    def from_workload(cls, wl, kappa=None, bc_mode=BC_DEFAULT):
        return cls(wl.problem, wl.p, wl.X, wl.ev, gamma=wl.gamma, kappa=wl.kappa if kappa is None else kappa,
                   bc_mode=bc_mode, q=getattr(wl, "q", 1))

    def __del__(self):
        if getattr(self, "_h", None):
            _load().orc_destroy(self._h)
            self._h = None

    # -- reference element -------------------------------------------------
    def neighbors(self):
        nbr = np.zeros(self.n_elems * self.nface, dtype=np.int32)
        nf = np.zeros_like(nbr)
        _load().orc_neighbors(self._h, _pi(nbr), _pi(nf))
        return nbr.reshape(-1, self.nface), nf.reshape(-1, self.nface)

    def ref_nodes(self):
        nodes = np.zeros(self.nb * self.dim)
        fn = np.zeros(self.nface * self.ntrace, dtype=np.int32)
        _load().orc_ref_nodes(self._h, _pd(nodes), _pi(fn))
        return nodes.reshape(self.nb, self.dim), fn.reshape(self.nface, self.ntrace)

    def ref_quadrature(self):
        vq = np.zeros(self.nq * self.dim)
        vw = np.zeros(self.nq)
        ft = np.zeros(self.nfq)
        fw = np.zeros(self.nfq)
        _load().orc_ref_quadrature(self._h, _pd(vq), _pd(vw), _pd(ft), _pd(fw))
        return vq.reshape(self.nq, self.dim), vw, ft, fw

    def ref_basis(self, xi):
        xi = _f64(np.atleast_2d(xi))
        n = xi.shape[0]
        phi = np.zeros(n * self.nb)
        dphi = np.zeros(n * self.nb * self.dim)
        _load().orc_ref_basis(self._h, n, _pd(xi), _pd(phi), _pd(dphi))
        return phi.reshape(n, self.nb), dphi.reshape(n, self.nb, self.dim)

    # -- element level -----------------------------------------------------
    def element(self, e, Ue, Up, xe, mu, jac=True):
        """R_e and (optionally) dR_e/dU_e, dR_e/dU_e', dR_e/dx_e, N_e, dN_e/dx_e."""
        Re = np.zeros(self.nu)
        Ne = np.zeros(1)
        if jac:
            JU = np.zeros(self.nu * self.nu)
            JUp = np.zeros(self.nu * self.nup)
            Jx = np.zeros(self.nu * self.nxe)
            dN = np.zeros(self.nxe)
        else:
            JU = JUp = Jx = dN = None
        bad = _load().orc_element(self._h, e, _pd(_f64(Ue)), _pd(_f64(Up)), _pd(_f64(xe)), _pd(_f64(mu)),
                                  _pd(Re), _pd(JU), _pd(JUp), _pd(Jx), _pd(Ne), _pd(dN))
        out = {"R": Re, "N": float(Ne[0]), "nonphysical": bool(bad)}
        if jac:
            out.update(JU=JU.reshape(self.nu, self.nu), JUp=JUp.reshape(self.nu, self.nup),
                       Jx=Jx.reshape(self.nu, self.nxe), dN=dN)
        return out

    def element_physical(self, e, Ue, Up, xe, mu):
        Re = np.zeros(self.nu)
        _load().orc_element_physical(self._h, e, _pd(_f64(Ue)), _pd(_f64(Up)), _pd(_f64(xe)), _pd(_f64(mu)),
                                     _pd(Re))
        return Re

    def gather(self, U, x, e):
        Ue = np.zeros(self.nu)
        Up = np.zeros(self.nup)
        xe = np.zeros(self.nxe)
        _load().orc_gather(self._h, _pd(_f64(U)), _pd(_f64(x)), e, _pd(Ue), _pd(Up), _pd(xe))
        return Ue, Up, xe

    def gather_rows(self, Phi, Psi, e):
        Phi = _f64(Phi)
        Psi = _f64(Psi)
        ku, kx = Phi.shape[1], Psi.shape[1]
        Pe = np.zeros(self.nu * ku)
        Pp = np.zeros(self.nup * ku)
        Se = np.zeros(self.nxe * max(kx, 1))
        _load().orc_gather_rows(self._h, ku, _pd(Phi), kx, _pd(Psi), e, _pd(Pe), _pd(Pp), _pd(Se))
        return Pe.reshape(self.nu, ku), Pp.reshape(self.nup, ku), Se[: self.nxe * kx].reshape(self.nxe, kx)

    # -- global level ------------------------------------------------------
    def residual(self, U, x, mu):
        R = np.zeros(self.Nu)
        N = np.zeros(self.n_elems)
        bad = _load().orc_global_residual(self._h, _pd(_f64(U)), _pd(_f64(x)), _pd(_f64(mu)), _pd(R), _pd(N))
        return R, N, int(bad)

    def jacobian_dense(self, U, x, mu):
        dRdU = np.zeros((self.Nu, self.Nu))
        dRdx = np.zeros((self.Nu, self.Nx))
        dNdx = np.zeros((self.n_elems, self.Nx))
        _load().orc_global_jacobian(self._h, _pd(_f64(U)), _pd(_f64(x)), _pd(_f64(mu)), _pd(dRdU), _pd(dRdx),
                                    _pd(dNdx))
        return dRdU, dRdx, dNdx

    def jacobian_sparse(self, U, x, mu):
        """dR/dU as a scipy CSR matrix, scattered from the element Jacobians."""
        import scipy.sparse as sp

        nbr, nbf = self.neighbors()
        _, fn = self.ref_nodes()
        rows, cols, vals = [], [], []
        ii = np.arange(self.nu)
        for e in range(self.n_elems):
            Ue, Up, xe = self.gather(U, x, e)
            out = self.element(e, Ue, Up, xe, mu, jac=True)
            r0 = e * self.nu
            rows.append(np.repeat(r0 + ii, self.nu))
            cols.append(np.tile(r0 + ii, self.nu))
            vals.append(out["JU"].ravel())
            for k in range(self.nface):
                e2 = nbr[e, k]
                if e2 < 0:
                    continue
                k2 = nbf[e, k]
                for j in range(self.ntrace):
                    node = fn[k2, self.ntrace - 1 - j]
                    for a in range(self.m):
                        col = e2 * self.nu + node * self.m + a
                        rows.append(r0 + ii)
                        cols.append(np.full(self.nu, col))
                        vals.append(out["JUp"][:, (k * self.ntrace + j) * self.m + a])
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        vals = np.concatenate(vals)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.Nu, self.Nu))

    # -- operation counts (work accounting) ------------------------------------
    def count_element(self, e, Ue, Up, xe, mu, dUe=None, dUp=None, dxe=None):
        """Floating-point operations of the oracle's element residual at (Ue, Up, xe):
        (value operations of R_e, derivative operations of one forward-mode sweep along
        the seeded direction; an input without a seed has a structurally zero
        derivative and costs nothing)."""
        out = np.zeros(2, dtype=np.int64)
        opt = lambda a: None if a is None else _pd(_f64(a))
        _load().orc_count_element(self._h, e, _pd(_f64(Ue)), _pd(_f64(Up)), _pd(_f64(xe)), _pd(_f64(mu)),
                                  opt(dUe), opt(dUp), opt(dxe),
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
        return int(out[0]), int(out[1])

    def count_pointwise(self, which, Up, Um, n, d):
        """Operations of one pointwise routine: which = 0 Euler flux f(U+), 1 Euler Roe
        flux (U+ seeded), 2 Burgers Roe flux (u+ seeded). Returns (value, derivative)."""
        out = np.zeros(2, dtype=np.int64)
        _load().orc_count_pointwise(self._h, which, _pd(_f64(Up)), _pd(_f64(Um)), _pd(_f64(n)), _pd(_f64(d)),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
        return int(out[0]), int(out[1])

    # -- snapshot alignment (Eq. align0) --------------------------------------
    def align(self, Phi, mu, w0, x0, free_mask, tol=1e-8, max_iters=100, trace=False):
        """min over (w, x_free) of (1/2)|F|^2, F = [R(Phi w, x; mu); N(x)], every element
        weight 1, by Levenberg-Marquardt on the dense global Jacobians (small meshes
        only). The step solves (J^T J + lambda D) d = -J^T F exactly (D = 1 on the mesh
        coordinates, 0 on w), with the damping and line-search rules of the reduced
        solve (lambda_0 = 1e-4, /10 after a full step, x10 after a shortened one,
        Armijo 1e-4 with 16 ulp of |J|, at most 30 halvings); stops when
        |J^T F| <= tol max(1, |J^T F| at the start). With trace=True the result carries
        "trace": one row per accepted step, [lambda used, alpha, w..., x_free...]."""
        Phi = np.asarray(Phi, dtype=np.float64)
        free = np.nonzero(np.asarray(free_mask).ravel())[0]
        w = np.array(w0, dtype=np.float64)
        x = np.array(x0, dtype=np.float64).ravel()
        ku, nf = Phi.shape[1], len(free)

        def F_of(w, x):
            R, N, bad = self.residual(Phi @ w, x, mu)
            return np.concatenate([R, N]), bad

        def jac(w, x):
            dRdU, dRdx, dNdx = self.jacobian_dense(Phi @ w, x, mu)
            top = np.concatenate([dRdU @ Phi, dRdx[:, free]], axis=1)
            bot = np.concatenate([np.zeros((self.n_elems, ku)), dNdx[:, free]], axis=1)
            return np.concatenate([top, bot], axis=0)

        F, bad = F_of(w, x)
        J = 0.5 * F @ F
        Jm = jac(w, x)
        g = Jm.T @ F
        g0 = np.linalg.norm(g)
        thresh = tol * max(1.0, g0)
        lam, iters, trials, status = 1e-4, 0, 0, 1
        rows = []
        D = np.concatenate([np.zeros(ku), np.ones(nf)])
        while True:
            if np.linalg.norm(g) <= thresh:
                status = 0
                break
            if iters >= max_iters:
                break
            d = np.linalg.solve(Jm.T @ Jm + lam * np.diag(D), -g)
            slope = g @ d
            alpha, h, accepted = 1.0, 0, False
            while True:
                wt = w + alpha * d[:ku]
                xt = x.copy()
                xt[free] += alpha * d[ku:]
                Ft, bad = F_of(wt, xt)
                Jt = 0.5 * Ft @ Ft
                trials += 1
                if bad == 0 and np.isfinite(Jt) and Jt <= J + 1e-4 * alpha * slope + 16 * 2.220446049250313e-16 * abs(J):
                    accepted = True
                    break
                h += 1
                if h > 30:
                    break
                alpha *= 0.5
            if not accepted:
                status = 2
                break
            rows.append(np.concatenate([[lam, alpha], wt, xt[free]]))
            lam = max(lam / 10, 1e-12) if h == 0 else min(lam * 10, 1e8)
            w, x, F, J = wt, xt, Ft, Jt
            iters += 1
            Jm = jac(w, x)
            g = Jm.T @ F
        out = {"status": status, "w": w, "x": x, "J": J, "gnorm": float(np.linalg.norm(g)), "g0": float(g0),
               "iters": iters, "trials": trials}
        if trace:
            out["trace"] = np.array(rows).reshape(-1, 2 + ku + nf)
        return out

    # -- reduced level -----------------------------------------------------
    @staticmethod
    def _rho_args(rho_set):
        if rho_set is None:
            return -1, None, None
        elems, rho = rho_set
        elems = np.ascontiguousarray(elems, dtype=np.int32)
        rho = _f64(rho)
        return len(elems), elems, rho

    def reduced(self, Phi, Psi, w, tau, mu, rho_set=None, nthreads=0):
        """S~, T~, H (k x k), J~ at (w, tau); rho_set = (elems, rho) or None for rho = 1."""
        Phi = _f64(Phi)
        Psi = _f64(Psi)
        ku, kx = Phi.shape[1], Psi.shape[1]
        nnz, el, rh = self._rho_args(rho_set)
        S = np.zeros(ku)
        T = np.zeros(max(kx, 1))
        H = np.zeros((ku + kx) ** 2)
        J = np.zeros(1)
        bad = _load().orc_reduced(self._h, ku, _pd(Phi), kx, _pd(Psi), nnz, _pi(el), _pd(rh), _pd(_f64(w)),
                                  _pd(_f64(tau) if kx else np.zeros(1)), _pd(_f64(mu)), _pd(S), _pd(T), _pd(H),
                                  _pd(J), nthreads)
        return {"S": S, "T": T[:kx], "H": H.reshape(ku + kx, ku + kx), "J": float(J[0]), "nonphysical": int(bad)}

    def objective(self, Phi, Psi, w, tau, mu, rho_set=None, nthreads=0):
        Phi = _f64(Phi)
        Psi = _f64(Psi)
        ku, kx = Phi.shape[1], Psi.shape[1]
        nnz, el, rh = self._rho_args(rho_set)
        J = np.zeros(1)
        bad = _load().orc_objective(self._h, ku, _pd(Phi), kx, _pd(Psi), nnz, _pi(el), _pd(rh), _pd(_f64(w)),
                                    _pd(_f64(tau) if kx else np.zeros(1)), _pd(_f64(mu)), _pd(J), nthreads)
        return float(J[0]), int(bad)

    def solve(self, Phi, Psi, mu, w_guess, tau0=None, rho_set=None, do_init=True, tol=1e-8, max_iters=200,
              nthreads=0, trace=False):
        """Levenberg-Marquardt solve (Sec. 3.2.3, Remark rem:solver). With trace=True the
        result carries "trace": one row per accepted step, [phase (0 init, 1 joint),
        lambda used in the step, step length alpha, w..., tau...]."""
        Phi = _f64(Phi)
        Psi = _f64(Psi)
        ku, kx = Phi.shape[1], Psi.shape[1]
        nnz, el, rh = self._rho_args(rho_set)
        w = np.zeros(ku)
        tau = np.zeros(max(kx, 1))
        info = np.zeros(16)
        hist = np.zeros(2 * (max_iters + 2))
        nh = np.zeros(1, dtype=np.int32)
        t0 = None if tau0 is None else _f64(tau0)
        tr = np.zeros(2 * (max_iters + 1) * (ku + kx + 3)) if trace else None
        ntr = np.zeros(1, dtype=np.int32)
        st = _load().orc_solve(self._h, ku, _pd(Phi), kx, _pd(Psi), nnz, _pi(el), _pd(rh), _pd(_f64(mu)),
                               _pd(_f64(w_guess)), _pd(t0), int(do_init), tol, max_iters, _pd(w), _pd(tau),
                               _pd(info), _pd(hist), _pi(nh), nthreads, _pd(tr), _pi(ntr) if trace else None)
        out = {"status": int(st), "w": w, "tau": tau[:kx], "init_iters": int(info[1]),
               "iters": int(info[2]), "trials": int(info[3]), "shifts": int(info[4]), "J": info[5],
               "normS": info[6], "normT": info[7], "g0": info[8], "init_status": int(info[9]),
               "hist": hist[: int(nh[0])]}
        if trace:
            out["trace"] = tr[: int(ntr[0]) * (ku + kx + 3)].reshape(-1, ku + kx + 3)
        return out
