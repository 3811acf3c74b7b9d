"""Python binding of the C-ABI library libift.so (include/ift.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels. There is no CPU fallback; if the library cannot be loaded the
calls raise. PyTorch is used only for device memory and streams in the
``*_dev`` variants (tensors' data pointers and the current stream).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libift.so")

IFT_OK = 0
IFT_NOT_CONVERGED = 1
IFT_LINESEARCH_FAILED = 2
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", 2: "LINESEARCH_FAILED", -1: "ERR_ARG", -2: "ERR_STATE",
                -3: "ERR_CUDA", -4: "ERR_OOM", -5: "ERR_NONPHYSICAL", -6: "ERR_TIMEOUT", -7: "ERR_NOTIMPL"}
BURGERS1D = 1
EULER2D = 2
FP64 = 0
FP32 = 1
MIXED = 2
FP32_JACOBIAN = 3
INIT_PAPER = 0
INIT_GIVEN = 1
CONTRACT_FP = 0
CONTRACT_TF32 = 1
CONTRACT_3XTF32 = 2
CONTRACT_BF16 = 3


class IFTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("problem", ctypes.c_int), ("p", ctypes.c_int), ("precision", ctypes.c_int),
                ("gamma", ctypes.c_double), ("kappa", ctypes.c_double), ("eps_g", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iters", ctypes.c_int), ("lm_init", ctypes.c_int),
                ("contraction", ctypes.c_int), ("q", ctypes.c_int), ("align_cg_tol", ctypes.c_double),
                ("max_loop_bodies", ctypes.c_int)]


class AlignInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("cg_iters", ctypes.c_int),
                ("trials", ctypes.c_int), ("J", ctypes.c_double), ("gnorm", ctypes.c_double),
                ("g0", ctypes.c_double), ("ms_form", ctypes.c_double), ("ms_cg", ctypes.c_double),
                ("ms_search", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("init_iters", ctypes.c_int), ("iters", ctypes.c_int),
                ("trials", ctypes.c_int), ("shifts", ctypes.c_int), ("J", ctypes.c_double),
                ("normS", ctypes.c_double), ("normT", ctypes.c_double), ("g0", ctypes.c_double),
                ("fp32_iters", ctypes.c_int), ("fp32_trials", ctypes.c_int), ("h_evals", ctypes.c_int)]


_lib = None

EXPORTS = ["ift_config_default", "ift_create", "ift_destroy", "ift_last_error", "ift_create_error",
           "ift_reference_nodes", "ift_sizes", "ift_set_mesh", "ift_set_bases", "ift_set_eq_weights",
           "ift_reduced_residual_jacobian", "ift_reduced_residual_jacobian_dev", "ift_element_eval",
           "ift_solve_rom", "ift_solve_rom_dev", "ift_reduced_residual_jacobian_static",
           "ift_set_eq_weights_batched", "ift_reduced_residual_jacobian_batched", "ift_solve_rom_batched",
           "ift_solve_rom_batched_dev", "ift_autotune", "ift_set_launch_shapes", "ift_hdm_residual_norms", "ift_element_gradients", "ift_mlp_create", "ift_mlp_destroy",
           "ift_mlp_num_params", "ift_mlp_get_params", "ift_mlp_set_params", "ift_mlp_get_scaling", "ift_mlp_set_scaling", "ift_mlp_loss_grad", "ift_mlp_train",
           "ift_mlp_predict", "ift_mlp_predict_bf16", "ift_nearest_start", "ift_align_residual", "ift_align_jvp", "ift_align_vjp",
           "ift_align", "ift_align_dev"]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libift.so; raises OSError if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libift.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    pd = ctypes.POINTER(ctypes.c_double)
    pi = ctypes.POINTER(ctypes.c_int32)
    pl = ctypes.POINTER(ctypes.c_int64)
    P = ctypes.POINTER
    sigs = {
        "ift_config_default": (None, [P(Config)]),
        "ift_create": (i32, [P(Config), vp, P(vp)]),
        "ift_destroy": (i32, [vp]),
        "ift_last_error": (ctypes.c_char_p, [vp]),
        "ift_create_error": (ctypes.c_char_p, []),
        "ift_reference_nodes": (i32, [vp, pd, pi]),
        "ift_sizes": (i32, [vp, pl]),
        "ift_set_mesh": (i32, [vp, i64, pd, i64, pi]),
        "ift_set_bases": (i32, [vp, i64, i32, pd, i64, i32, pd]),
        "ift_set_eq_weights": (i32, [vp, i64, pi, pd]),
        "ift_reduced_residual_jacobian": (i32, [vp, pd, pd, pd, pd, pd, pd, pd]),
        "ift_reduced_residual_jacobian_dev": (i32, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "ift_element_eval": (i32, [vp, pd, pd, pd, i64, pi, pd, pd, pd, pd, pd, pd]),
        "ift_solve_rom": (i32, [vp, pd, pd, pd, P(SolveInfo)]),
        "ift_solve_rom_dev": (i32, [vp, vp, vp, vp, P(SolveInfo), vp]),
        "ift_set_eq_weights_batched": (i32, [vp, i32, pl, pi, pd]),
        "ift_autotune": (i32, [vp, pd, pd, pd, pi]),
        "ift_set_launch_shapes": (i32, [vp, i32, i32, i32]),
        "ift_hdm_residual_norms": (i32, [vp, i32, pd, pd, pd, pd]),
        "ift_element_gradients": (i32, [vp, pd, pd, pd, i64, pi, pd]),
        "ift_reduced_residual_jacobian_batched": (i32, [vp, pd, pd, pd, pd, pd, pd, pd]),
        "ift_solve_rom_batched": (i32, [vp, pd, pd, pd, P(SolveInfo)]),
        "ift_solve_rom_batched_dev": (i32, [vp, vp, vp, vp, vp, vp]),
        "ift_reduced_residual_jacobian_static": (i32, [i32, i32, i64, vp, i64, vp, vp, vp, vp, vp, i32, vp, i32,
                                                       i64, vp, vp, vp, vp, vp, dbl, dbl, dbl, vp, vp, vp, vp,
                                                       vp]),
        "ift_mlp_create": (i32, [i32, i32, i32, i32, ctypes.c_uint64, vp, P(vp)]),
        "ift_mlp_destroy": (i32, [vp]),
        "ift_mlp_num_params": (i32, [vp, pl]),
        "ift_mlp_get_params": (i32, [vp, pd]),
        "ift_mlp_set_params": (i32, [vp, pd]),
        "ift_mlp_get_scaling": (i32, [vp, pd, pd, pd, pd]),
        "ift_mlp_set_scaling": (i32, [vp, pd, pd, pd, pd]),
        "ift_mlp_loss_grad": (i32, [vp, i64, pd, pd, pd, pd]),
        "ift_mlp_train": (i32, [vp, i64, pd, pd, i32, i32, dbl, ctypes.c_uint64, pd]),
        "ift_mlp_predict": (i32, [vp, i64, pd, pd]),
        "ift_mlp_predict_bf16": (i32, [vp, i64, pd, pd]),
        "ift_nearest_start": (i32, [i64, i32, pd, i32, pd, i64, pd, pd, pd]),
        "ift_align_residual": (i32, [vp, pd, pd, pd, pd]),
        "ift_align_jvp": (i32, [vp, pd, pd, pd, pd, pd, pd]),
        "ift_align_vjp": (i32, [vp, pd, pd, pd, pd, pd, pd]),
        "ift_align": (i32, [vp, pd, pd, pd, ctypes.POINTER(ctypes.c_uint8), dbl, i32, P(AlignInfo)]),
        "ift_align_dev": (i32, [vp, vp, vp, vp, vp, dbl, i32, P(AlignInfo), vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _pd(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _tptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def reduced_residual_jacobian_static(problem, p, X, ev, nbr, nbr_face, bc, Phi, Psi, elems, rho, mu, y, z, S, T,
                                     H, J, gamma=1.4, kappa=0.0, eps_g=1e-8, stream=None):
    """The allocation-free assembly: every array argument is a caller-owned CUDA tensor
    (X, Phi, Psi, rho, mu, y, z, S, T, H, J float64; ev, nbr, nbr_face, elems int32; bc int8).
    elems = rho = None means rho = 1 on every element."""
    lib = load()
    nnz = -1 if elems is None else int(elems.numel())
    st = lib.ift_reduced_residual_jacobian_static(
        problem, p, int(X.shape[0]), _tptr(X), int(ev.shape[0]), _tptr(ev), _tptr(nbr), _tptr(nbr_face), _tptr(bc),
        _tptr(Phi), int(Phi.shape[1]), _tptr(Psi) if Psi.shape[1] else None, int(Psi.shape[1]), nnz, _tptr(elems),
        _tptr(rho), _tptr(mu), _tptr(y), _tptr(z) if Psi.shape[1] else None, gamma, kappa, eps_g, _tptr(S),
        _tptr(T), _tptr(H), _tptr(J), ctypes.c_void_p(stream) if stream else None)
    if st != IFT_OK:
        raise IFTError(st, "ift_reduced_residual_jacobian_static failed")


class Context:
    """One problem instance on the current CUDA device."""

    def __init__(self, problem: int, p: int, precision: int = FP64, gamma: float = 1.4, kappa: float = 0.0,
                 eps_g: float = 1e-8, tol: float = 1e-8, max_iters: int = 200, lm_init: int = INIT_PAPER,
                 contraction: int = CONTRACT_FP, stream=None, q: int = 1, align_cg_tol: float = 1e-12,
                 max_loop_bodies: int = 0):
        lib = load()
        cfg = Config()
        lib.ift_config_default(ctypes.byref(cfg))
        cfg.problem, cfg.p, cfg.precision, cfg.q = problem, p, precision, q
        cfg.gamma, cfg.kappa, cfg.eps_g, cfg.tol = gamma, kappa, eps_g, tol
        cfg.max_iters, cfg.lm_init, cfg.contraction = max_iters, lm_init, contraction
        cfg.align_cg_tol = align_cg_tol
        cfg.max_loop_bodies = max_loop_bodies
        h = ctypes.c_void_p()
        st = lib.ift_create(ctypes.byref(cfg), ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
        if st != IFT_OK:
            raise IFTError(st, lib.ift_create_error().decode())
        self._h = h
        self.cfg = cfg
        s = np.zeros(8, dtype=np.int64)
        lib.ift_sizes(h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        self.nb, self.nu, self.nup, self.nxe, self.nface, self.ntrace, self.nq, self.nfq = (int(v) for v in s)
        self.dim = 1 if problem == BURGERS1D else 2
        self.n_mu = 1 if problem == BURGERS1D else 2
        self.ku = self.kx = 0
        self.B = 0

    def close(self):
        if getattr(self, "_h", None):
            load().ift_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow_positive=False):
        if st < 0 or (st > 0 and not allow_positive):
            raise IFTError(st, load().ift_last_error(self._h).decode())
        return st

    # -- set-up ------------------------------------------------------------
    def reference_nodes(self):
        nodes = np.zeros(self.nb * self.dim)
        fn = np.zeros(self.nface * self.ntrace, dtype=np.int32)
        self._check(load().ift_reference_nodes(self._h, _pd(nodes), _pi(fn)))
        return nodes.reshape(self.nb, self.dim), fn.reshape(self.nface, self.ntrace)

    def set_mesh(self, X, ev):
        X = _f64(X)
        ev = np.ascontiguousarray(ev, dtype=np.int32)
        self.n_verts = X.shape[0]
        self.n_elems = ev.shape[0]
        self._check(load().ift_set_mesh(self._h, self.n_verts, _pd(X), self.n_elems, _pi(ev)))

    def set_bases(self, Phi, Psi):
        Phi = _f64(Phi)
        Psi = _f64(Psi)
        self.ku, self.kx = Phi.shape[1], Psi.shape[1]
        self._check(load().ift_set_bases(self._h, Phi.shape[0], self.ku, _pd(Phi), Psi.shape[0], self.kx,
                                         _pd(Psi) if self.kx else None))

    def set_eq_weights(self, rho_set):
        """rho_set = (elems, rho) or None for rho = 1 on every element."""
        if rho_set is None:
            self._check(load().ift_set_eq_weights(self._h, -1, None, None))
            return
        elems = np.ascontiguousarray(rho_set[0], dtype=np.int32)
        rho = _f64(rho_set[1])
        self._check(load().ift_set_eq_weights(self._h, len(elems), _pi(elems), _pd(rho)))

    @classmethod
    def from_workload(cls, wl, precision=FP64, **kw):
        kw.setdefault("q", getattr(wl, "q", 1))
        ctx = cls(wl.problem, wl.p, precision=precision, gamma=wl.gamma, kappa=kw.pop("kappa", wl.kappa), **kw)
        ctx.set_mesh(wl.X, wl.ev)
        ctx.set_bases(wl.Phi, wl.Psi)
        return ctx

    # -- evaluation --------------------------------------------------------
    def reduced_residual_jacobian(self, mu, y, z):
        k = self.ku + self.kx
        S = np.zeros(self.ku)
        T = np.zeros(max(self.kx, 1))
        H = np.zeros(k * k)
        J = np.zeros(1)
        zz = _f64(z) if self.kx else np.zeros(1)
        st = load().ift_reduced_residual_jacobian(self._h, _pd(_f64(mu)), _pd(_f64(y)), _pd(zz), _pd(S), _pd(T),
                                                  _pd(H), _pd(J))
        if st not in (IFT_OK, -5):
            self._check(st)
        return {"S": S, "T": T[:self.kx], "H": H.reshape(k, k), "J": float(J[0]), "status": int(st)}

    def reduced_residual_jacobian_dev(self, mu, y, z, S, T, H, J, stream=None):
        """Device-pointer variant; all arguments are CUDA tensors (float64)."""
        self._check(load().ift_reduced_residual_jacobian_dev(self._h, _tptr(mu), _tptr(y), _tptr(z), _tptr(S),
                                                             _tptr(T), _tptr(H), _tptr(J),
                                                             ctypes.c_void_p(stream) if stream else None))

    def element_eval(self, mu, U, x, elems):
        elems = np.ascontiguousarray(elems, dtype=np.int32)
        n = len(elems)
        R = np.zeros(n * self.nu)
        JU = np.zeros(n * self.nu * self.nu)
        JUp = np.zeros(n * self.nu * self.nup)
        Jx = np.zeros(n * self.nu * self.nxe)
        N = np.zeros(n)
        dN = np.zeros(n * self.nxe)
        self._check(load().ift_element_eval(self._h, _pd(_f64(mu)), _pd(_f64(U)), _pd(_f64(x)), n, _pi(elems),
                                            _pd(R), _pd(JU), _pd(JUp), _pd(Jx), _pd(N), _pd(dN)))
        return {"R": R.reshape(n, self.nu), "JU": JU.reshape(n, self.nu, self.nu),
                "JUp": JUp.reshape(n, self.nu, self.nup), "Jx": Jx.reshape(n, self.nu, self.nxe), "N": N,
                "dN": dN.reshape(n, self.nxe)}

    # -- snapshot alignment (Eq. align0) ------------------------------------
    def _align_sizes(self):
        return self.n_elems * self.nu, self.n_elems, self.n_verts * self.dim

    def align_residual(self, mu, w, x):
        """F = [R; N] at (w, x) over every element (x: all mesh coordinates)."""
        Nu, Ne, _ = self._align_sizes()
        F = np.zeros(Nu + Ne)
        self._check(load().ift_align_residual(self._h, _pd(_f64(mu)), _pd(_f64(w)), _pd(_f64(x)), _pd(F)))
        return F

    def align_jvp(self, mu, w, x, dU, dx):
        Nu, Ne, _ = self._align_sizes()
        dF = np.zeros(Nu + Ne)
        self._check(load().ift_align_jvp(self._h, _pd(_f64(mu)), _pd(_f64(w)), _pd(_f64(x)), _pd(_f64(dU)),
                                         _pd(_f64(dx)), _pd(dF)))
        return dF

    def align_vjp(self, mu, w, x, v):
        Nu, _, Nx = self._align_sizes()
        gU, gx = np.zeros(Nu), np.zeros(Nx)
        self._check(load().ift_align_vjp(self._h, _pd(_f64(mu)), _pd(_f64(w)), _pd(_f64(x)), _pd(_f64(v)),
                                         _pd(gU), _pd(gx)))
        return gU, gx

    def align(self, mu, w0, x0, free_mask, tol=1e-8, max_iters=100):
        """Levenberg-Marquardt on (w, free mesh coordinates) for Eq. align0; returns
        the aligned (w, x) and the solver's counts."""
        w = _f64(w0).copy()
        x = _f64(x0).copy()
        mask = np.ascontiguousarray(free_mask, dtype=np.uint8)
        info = AlignInfo()
        st = load().ift_align(self._h, _pd(_f64(mu)), _pd(w), _pd(x),
                              mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), tol, max_iters,
                              ctypes.byref(info))
        self._check(st, allow_positive=True)
        return {"status": int(st), "w": w, "x": x, "iters": info.iters, "cg_iters": info.cg_iters,
                "trials": info.trials, "J": info.J, "gnorm": info.gnorm, "g0": info.g0,
                "ms_form": info.ms_form, "ms_cg": info.ms_cg, "ms_search": info.ms_search}

    def align_dev(self, mu, w, x, free_mask, tol=1e-8, max_iters=100, stream=None):
        """Device-pointer variant of align: mu, w, x (float64, w and x updated in place)
        and free_mask (uint8) are CUDA tensors; synchronises the stream."""
        info = AlignInfo()
        st = load().ift_align_dev(self._h, _tptr(mu), _tptr(w), _tptr(x), _tptr(free_mask), tol, max_iters,
                                  ctypes.byref(info), ctypes.c_void_p(stream) if stream else None)
        self._check(st, allow_positive=True)
        return {"status": int(st), "iters": info.iters, "cg_iters": info.cg_iters, "trials": info.trials,
                "J": info.J, "gnorm": info.gnorm, "g0": info.g0, "ms_form": info.ms_form, "ms_cg": info.ms_cg,
                "ms_search": info.ms_search}

    def solve_rom(self, mu, y0=None, z0=None):
        y = np.zeros(self.ku) if y0 is None else _f64(y0).copy()
        z = np.zeros(max(self.kx, 1)) if z0 is None else np.concatenate([_f64(z0), np.zeros(1)])
        info = SolveInfo()
        st = load().ift_solve_rom(self._h, _pd(_f64(mu)), _pd(y), _pd(z), ctypes.byref(info))
        if st != -5:  # a non-physical start is a result of the solve, reported in status
            self._check(st, allow_positive=True)
        return {"status": int(st), "w": y, "tau": z[:self.kx], "init_iters": info.init_iters, "iters": info.iters,
                "trials": info.trials, "shifts": info.shifts, "J": info.J, "normS": info.normS,
                "normT": info.normT, "g0": info.g0, "fp32_iters": info.fp32_iters, "fp32_trials": info.fp32_trials,
                "h_evals": info.h_evals}

    def autotune(self, mu, y, z):
        """Pick the launch shapes by timing this workload; returns (warps, batched warps, chunk)."""
        out = np.zeros(3, dtype=np.int32)
        zz = _f64(z) if self.kx else np.zeros(1)
        self._check(load().ift_autotune(self._h, _pd(_f64(mu)), _pd(_f64(y)), _pd(zz), _pi(out)))
        return tuple(int(v) for v in out)

    def set_launch_shapes(self, warps, batched_warps, chunk):
        self._check(load().ift_set_launch_shapes(self._h, warps, batched_warps, chunk))

    def hdm_residual_norms(self, mus, ys, zs):
        """|R(Phi y_q, X + Psi z_q; mu_q)|_2 over every element, for each row q."""
        mus = _f64(mus).reshape(len(ys), -1)
        ys = _f64(ys)
        zz = _f64(zs) if self.kx else np.zeros(1)
        out = np.zeros(len(ys))
        self._check(load().ift_hdm_residual_norms(self._h, len(ys), _pd(mus), _pd(ys), _pd(zz), _pd(out)))
        return out

    def element_gradients(self, mu, y, z, elems=None):
        """Rows [S^(e) | T^(e) | J^(e)] per element (every element if elems is None)."""
        n = -1 if elems is None else len(elems)
        rows = self.n_elems if elems is None else len(elems)
        out = np.zeros((rows, self.ku + self.kx + 1))
        el = None if elems is None else np.ascontiguousarray(elems, dtype=np.int32)
        zz = _f64(z) if self.kx else np.zeros(1)
        st = load().ift_element_gradients(self._h, _pd(_f64(mu)), _pd(_f64(y)), _pd(zz), n, _pi(el), _pd(out))
        if st not in (IFT_OK, -5):
            self._check(st)
        return out

    def greedy_search(self, mus):
        """Eq. greedy0 over candidate parameters mus with the batched weight sets
        already set (one per candidate): solve every candidate, evaluate the HDM
        residual norm at each solution, return (argmax, norms, solve result)."""
        res = self.solve_rom_batched(mus)
        norms = self.hdm_residual_norms(mus, res["w"], res["tau"])
        return int(np.argmax(norms)), norms, res

    # -- batched queries ---------------------------------------------------
    def set_eq_weights_batched(self, sets):
        """sets: list of (elems, rho) per query."""
        offsets = np.zeros(len(sets) + 1, dtype=np.int64)
        offsets[1:] = np.cumsum([len(e) for e, _ in sets])
        elems = np.ascontiguousarray(np.concatenate([e for e, _ in sets]), dtype=np.int32)
        rho = _f64(np.concatenate([r for _, r in sets]))
        self.B = len(sets)
        self._check(load().ift_set_eq_weights_batched(self._h, self.B, offsets.ctypes.data_as(
            ctypes.POINTER(ctypes.c_int64)), _pi(elems), _pd(rho)))

    def reduced_residual_jacobian_batched(self, mus, ys, zs):
        B, k = self.B, self.ku + self.kx
        S = np.zeros(B * self.ku)
        T = np.zeros(max(B * self.kx, 1))
        H = np.zeros(B * k * k)
        J = np.zeros(B)
        zz = _f64(zs) if self.kx else np.zeros(1)
        st = load().ift_reduced_residual_jacobian_batched(self._h, _pd(_f64(mus)), _pd(_f64(ys)), _pd(zz), _pd(S),
                                                          _pd(T), _pd(H), _pd(J))
        if st not in (IFT_OK, -5):
            self._check(st)
        return {"S": S.reshape(B, self.ku), "T": T[:B * self.kx].reshape(B, self.kx), "H": H.reshape(B, k, k),
                "J": J, "status": int(st)}

    def solve_rom_batched(self, mus, y0=None, z0=None):
        B = self.B
        y = np.zeros(B * self.ku) if y0 is None else _f64(y0).ravel().copy()
        z = np.zeros(max(B * self.kx, 1)) if z0 is None else np.concatenate([_f64(z0).ravel(), np.zeros(1)])
        info = (SolveInfo * B)()
        st = load().ift_solve_rom_batched(self._h, _pd(_f64(mus)), _pd(y), _pd(z), info)
        if st != -5:  # non-physical queries are reported per query in info
            self._check(st, allow_positive=True)
        return {"status": int(st), "w": y.reshape(B, self.ku), "tau": z[:B * self.kx].reshape(B, self.kx),
                "info": [{"status": i.status, "init_iters": i.init_iters, "iters": i.iters, "trials": i.trials,
                          "J": i.J, "normS": i.normS, "normT": i.normT, "g0": i.g0, "fp32_iters": i.fp32_iters,
                          "fp32_trials": i.fp32_trials, "h_evals": i.h_evals} for i in info]}

    def solve_rom_batched_dev(self, mus, y, z, status=None, stream=None):
        self._check(load().ift_solve_rom_batched_dev(self._h, _tptr(mus), _tptr(y), _tptr(z), _tptr(status),
                                                     ctypes.c_void_p(stream) if stream else None))

    def solve_rom_dev(self, mu, y, z, stream=None, want_info=True):
        info = SolveInfo()
        st = load().ift_solve_rom_dev(self._h, _tptr(mu), _tptr(y), _tptr(z),
                                      ctypes.byref(info) if want_info else None,
                                      ctypes.c_void_p(stream) if stream else None)
        self._check(st, allow_positive=True)
        if not want_info:
            return None
        return {"status": int(st), "init_iters": info.init_iters, "iters": info.iters, "trials": info.trials,
                "J": info.J, "normS": info.normS, "normT": info.normT, "g0": info.g0, "fp32_iters": info.fp32_iters,
                "fp32_trials": info.fp32_trials, "h_evals": info.h_evals}


class MLP:
    """The learned warm start: a GELU network n_in -> width^depth -> n_out trained and
    evaluated by the library's FP32 kernels (the ift_mlp_* calls)."""

    def __init__(self, n_in, width, depth, n_out, seed=0, stream=None):
        lib = load()
        h = ctypes.c_void_p()
        st = lib.ift_mlp_create(n_in, width, depth, n_out, seed, ctypes.c_void_p(stream) if stream else None,
                                ctypes.byref(h))
        if st != IFT_OK:
            raise IFTError(st, "ift_mlp_create failed")
        self._h = h
        self.n_in, self.width, self.depth, self.n_out = n_in, width, depth, n_out
        n = ctypes.c_int64()
        lib.ift_mlp_num_params(h, ctypes.byref(n))
        self.n_params = int(n.value)

    def close(self):
        if getattr(self, "_h", None):
            load().ift_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _check(st, what):
        if st != IFT_OK:
            raise IFTError(st, what + " failed")

    def get_params(self):
        out = np.zeros(self.n_params)
        self._check(load().ift_mlp_get_params(self._h, _pd(out)), "ift_mlp_get_params")
        return out

    def set_params(self, params):
        params = _f64(params)
        assert params.size == self.n_params
        self._check(load().ift_mlp_set_params(self._h, _pd(params)), "ift_mlp_set_params")

    def get_scaling(self):
        xm, xs, tm, ts = np.zeros(self.n_in), np.zeros(self.n_in), np.zeros(self.n_out), np.zeros(self.n_out)
        self._check(load().ift_mlp_get_scaling(self._h, _pd(xm), _pd(xs), _pd(tm), _pd(ts)), "ift_mlp_get_scaling")
        return xm, xs, tm, ts

    def set_scaling(self, xm, xs, tm, ts):
        xm, xs, tm, ts = (_f64(v) for v in (xm, xs, tm, ts))
        self._check(load().ift_mlp_set_scaling(self._h, _pd(xm), _pd(xs), _pd(tm), _pd(ts)), "ift_mlp_set_scaling")

    def loss_grad(self, x, t, want_grad=True):
        x, t = _f64(x), _f64(t)
        loss = np.zeros(1)
        grad = np.zeros(self.n_params) if want_grad else None
        self._check(load().ift_mlp_loss_grad(self._h, x.shape[0], _pd(x), _pd(t), _pd(loss), _pd(grad)),
                    "ift_mlp_loss_grad")
        return float(loss[0]), grad

    def train(self, x, t, epochs, batch, lr, seed=0):
        x, t = _f64(x), _f64(t)
        loss = np.zeros(1)
        self._check(load().ift_mlp_train(self._h, x.shape[0], _pd(x), _pd(t), epochs, batch, lr, seed, _pd(loss)),
                    "ift_mlp_train")
        return float(loss[0])

    def predict(self, x):
        x = _f64(x)
        out = np.zeros((x.shape[0], self.n_out))
        self._check(load().ift_mlp_predict(self._h, x.shape[0], _pd(x), _pd(out)), "ift_mlp_predict")
        return out

    def predict_bf16(self, x):
        """The same network evaluated on the tensor cores with BF16 operands and FP32
        accumulation (ift_mlp_predict_bf16)."""
        x = _f64(x)
        out = np.zeros((x.shape[0], self.n_out))
        self._check(load().ift_mlp_predict_bf16(self._h, x.shape[0], _pd(x), _pd(out)), "ift_mlp_predict_bf16")
        return out


def nearest_start(x_train, y_train, x_query, scale=None):
    """Outputs of the nearest training point for each query (computed on the device)."""
    x_train, y_train, x_query = _f64(x_train), _f64(y_train), _f64(x_query)
    out = np.zeros((x_query.shape[0], y_train.shape[1]))
    st = load().ift_nearest_start(x_train.shape[0], x_train.shape[1], _pd(x_train), y_train.shape[1], _pd(y_train),
                                  x_query.shape[0], _pd(x_query), None if scale is None else _pd(_f64(scale)),
                                  _pd(out))
    if st != IFT_OK:
        raise IFTError(st, "ift_nearest_start failed")
    return out
