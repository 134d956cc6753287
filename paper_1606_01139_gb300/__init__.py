"""Python binding of libswi_gb300 (the GB300 partitioned shift-without-invert solver).

Argument marshalling only: every step runs in the library's CUDA kernels.  The
names mirror the C ABI in ``include/swi.h`` (``swi_create`` -> ``create`` ...).
Host arrays are numpy; device arrays may be torch CUDA tensors (their
``data_ptr()`` is passed with ``on_device=1``).  The library is loaded lazily
and loading fails loudly if it has not been built (``build()`` or
``python -m paper_1606_01139_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libswi_gb300.so")

SWI_OK, SWI_EINVAL, SWI_ENOMEM, SWI_ECUDA, SWI_ENOCONV, SWI_HOLES, SWI_ETIMEOUT, SWI_ENOTIMPL, SWI_ESTATE = range(9)
STATUS_NAMES = {0: "SWI_OK", 1: "SWI_EINVAL", 2: "SWI_ENOMEM", 3: "SWI_ECUDA", 4: "SWI_ENOCONV",
                5: "SWI_HOLES", 6: "SWI_ETIMEOUT", 7: "SWI_ENOTIMPL", 8: "SWI_ESTATE"}
BC_ODD, BC_ZERO = 0, 1
PREC_F64, PREC_MIXED = 0, 1
ARITH_DS, ARITH_F64 = 2, 1
CONTRACT_F64, CONTRACT_F32 = 0, 1

# Every entry point declared in include/swi.h.
EXPORTS = ("swi_create", "swi_set_potential", "swi_set_absorber", "swi_set_windows", "swi_set_windows_complex",
           "swi_plan_windows", "swi_plan_windows_sampled",
           "swi_apply", "swi_apply_ds", "swi_apply_c64", "swi_solve", "swi_solve_batch", "swi_solve_more", "swi_fill_holes",
           "swi_get_windows", "swi_refine", "swi_get_window_info", "swi_get_eigenpairs", "swi_copy_eigenpairs",
           "swi_set_eigenpairs", "swi_residuals", "swi_transmission", "swi_set_contraction", "swi_grad", "swi_profile",
           "swi_profile_read", "swi_transmission_noalloc", "swi_check_schur", "swi_last_error", "swi_launch_count",
           "swi_destroy")

KERNEL_CLASSES = ("stencil", "gram", "update", "cholqr", "schur", "rotate", "merge", "proj", "trans", "grad")


class KernelStats(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("ms", C.c_double), ("flops", C.c_double), ("bytes", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("block", C.c_int), ("max_basis", C.c_int), ("keep", C.c_int), ("arith", C.c_int),
                ("max_matvecs", C.c_longlong), ("rel_tol", C.c_double), ("eq_rtol", C.c_double),
                ("drop_tol", C.c_double), ("seed", C.c_ulonglong), ("n_keep", C.c_int), ("reserved1", C.c_int)]


class RefineOpts(C.Structure):
    _fields_ = [("max_sweeps", C.c_int), ("group", C.c_int), ("arith", C.c_int), ("reserved", C.c_int),
                ("rel_tol", C.c_double), ("eq_rtol", C.c_double), ("drop_tol", C.c_double),
                ("near_tol", C.c_double)]


class RefineInfo(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("n_pairs", C.c_int), ("n_converged", C.c_int), ("n_dropped", C.c_int),
                ("matvecs", C.c_longlong), ("max_rel_res_in", C.c_double), ("max_rel_res", C.c_double),
                ("t_s", C.c_double)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class PlanOpts(C.Structure):
    _fields_ = [("sample_req", C.c_int), ("max_samples", C.c_int), ("sample_tol", C.c_double),
                ("inflate", C.c_double), ("extra", C.c_int), ("counts_rule", C.c_int),
                ("max_matvecs", C.c_longlong)]


class PlanInfo(C.Structure):
    _fields_ = [("e_min", C.c_double), ("e_max", C.c_double), ("e_top", C.c_double), ("samples", C.c_int),
                ("windows", C.c_int), ("matvecs", C.c_longlong), ("t_s", C.c_double)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class WindowInfo(C.Structure):
    _fields_ = [("sigma", C.c_double), ("n_req", C.c_int), ("n_conv", C.c_int), ("matvecs", C.c_longlong),
                ("restarts", C.c_int), ("basis", C.c_int), ("max_res", C.c_double), ("schur_retries", C.c_int),
                ("reserved", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("n_windows", C.c_int), ("n_pairs", C.c_int), ("n_converged", C.c_int),
                ("n_duplicates", C.c_int), ("n_holes", C.c_int), ("reserved", C.c_int),
                ("matvecs", C.c_longlong), ("max_rel_res", C.c_double), ("anorm", C.c_double),
                ("t_krylov_s", C.c_double), ("t_merge_s", C.c_double)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_ if not f[0].startswith("reserved")}


_lib = None


def load(path: str = LIB_PATH):
    """Load libswi_gb300.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1606_01139_gb300.build.build()")
    lib = C.CDLL(path)
    P, I, D, VP = C.POINTER, C.c_int, C.c_double, C.c_void_p
    sig = {
        "swi_create": (I, [P(VP), I, I, I, D, I, I, VP]),
        "swi_set_potential": (I, [VP, VP, I]),
        "swi_set_absorber": (I, [VP, VP, VP, I]),
        "swi_set_windows": (I, [VP, I, VP, VP]),
        "swi_set_windows_complex": (I, [VP, I, VP, VP, VP]),
        "swi_plan_windows": (I, [VP, I, I, D, D, D, VP, VP]),
        "swi_plan_windows_sampled": (I, [VP, I, I, P(PlanOpts), VP, VP, P(PlanInfo)]),
        "swi_apply": (I, [VP, I, VP, VP, VP, I]),
        "swi_apply_ds": (I, [VP, I, VP, VP, VP, I]),
        "swi_apply_c64": (I, [VP, I, VP, VP, VP, I]),
        "swi_solve": (I, [VP, P(SolveOpts), P(SolveInfo)]),
        "swi_solve_batch": (I, [I, VP, P(SolveOpts), I, P(SolveInfo), VP]),
        "swi_solve_more": (I, [VP, I, VP, VP, P(SolveOpts), P(SolveInfo)]),
        "swi_fill_holes": (I, [VP, D, D, I, P(SolveOpts), P(SolveInfo), P(I)]),
        "swi_get_windows": (I, [VP, I, VP, VP, P(I)]),
        "swi_refine": (I, [VP, P(RefineOpts), P(RefineInfo)]),
        "swi_get_window_info": (I, [VP, I, P(WindowInfo), P(I)]),
        "swi_get_eigenpairs": (I, [VP, P(I), P(VP), P(VP), P(I)]),
        "swi_copy_eigenpairs": (I, [VP, VP, VP, I]),
        "swi_set_eigenpairs": (I, [VP, I, VP, VP, I]),
        "swi_residuals": (I, [VP, VP]),
        "swi_transmission": (I, [VP, I, VP, VP]),
        "swi_set_contraction": (I, [VP, I]),
        "swi_grad": (I, [VP, I, VP, VP, VP, I, VP]),
        "swi_profile": (I, [VP, I]),
        "swi_transmission_noalloc": (I, [VP, I, VP, VP]),
        "swi_check_schur": (I, [VP, I, I, I, VP, VP, I, VP, VP, VP]),
        "swi_profile_read": (I, [VP, P(KernelStats)]),
        "swi_last_error": (C.c_char_p, [VP]),
        "swi_launch_count": (C.c_longlong, [VP]),
        "swi_destroy": (None, [VP]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SwiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(a):
    """Host numpy array -> void*, or torch tensor -> data_ptr (device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())


def _is_device(a) -> int:
    return 0 if (a is None or isinstance(a, np.ndarray)) else 1


def _c_arr(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


class Context:
    """One solver context (one grid, one potential) on the current CUDA device."""

    def __init__(self, nx, ny, nz, h, bc=BC_ODD, precision=PREC_F64, stream=None):
        lib = load()
        self._lib = lib
        self.nx, self.ny, self.nz, self.h = int(nx), int(ny), int(nz), float(h)
        self.N = self.nx * self.ny * self.nz
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:  # torch absent: legacy default stream
                stream = 0
        h_ = C.c_void_p()
        rc = lib.swi_create(C.byref(h_), self.nx, self.ny, self.nz, self.h, int(bc), int(precision),
                            C.c_void_p(stream))
        if rc != SWI_OK:
            raise SwiError(rc, lib.swi_last_error(None).decode())
        self._h = h_

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.swi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, allow=(SWI_OK,)):
        if rc not in allow:
            raise SwiError(rc, self._lib.swi_last_error(self._h).decode())
        return rc

    # -- inputs
    def set_potential(self, V):
        if _is_device(V):
            return self._check(self._lib.swi_set_potential(self._h, _ptr(V), 1))
        V = _c_arr(V, np.float64)
        return self._check(self._lib.swi_set_potential(self._h, _ptr(V), 0))

    def set_absorber(self, gamma_L, gamma_R):
        if _is_device(gamma_L):
            return self._check(self._lib.swi_set_absorber(self._h, _ptr(gamma_L), _ptr(gamma_R), 1))
        gl, gr = _c_arr(gamma_L, np.float64), _c_arr(gamma_R, np.float64)
        return self._check(self._lib.swi_set_absorber(self._h, _ptr(gl), _ptr(gr), 0))

    def set_windows(self, sigma, n_req):
        s, n = _c_arr(sigma, np.float64), _c_arr(n_req, np.int32)
        return self._check(self._lib.swi_set_windows(self._h, len(s), _ptr(s), _ptr(n)))

    def set_windows_complex(self, sigma, n_req):
        """Windows at complex shifts (sigma: complex array, increasing by (Re, Im))."""
        z = np.asarray(sigma, dtype=np.complex128)
        re, im, n = _c_arr(z.real, np.float64), _c_arr(z.imag, np.float64), _c_arr(n_req, np.int32)
        return self._check(self._lib.swi_set_windows_complex(self._h, len(re), _ptr(re), _ptr(im), _ptr(n)))

    def plan_windows(self, n_r, p, e_min, e_max, inflate=1.0):
        s = np.zeros(p)
        n = np.zeros(p, dtype=np.int32)
        self._check(self._lib.swi_plan_windows(self._h, int(n_r), int(p), float(e_min), float(e_max),
                                               float(inflate), _ptr(s), _ptr(n)))
        return s, n

    def plan_windows_sampled(self, n_r, p, sample_req=0, max_samples=0, sample_tol=0.0, inflate=0.0, extra=0,
                             counts_rule=0, max_matvecs=0):
        """Windows from extremal estimates and density sampling (Section 2.2.1); returns (sigma, n_req, info)."""
        o = PlanOpts(sample_req=sample_req, max_samples=max_samples, sample_tol=sample_tol, inflate=inflate,
                     extra=extra, counts_rule=counts_rule, max_matvecs=max_matvecs)
        s = np.zeros(p)
        n = np.zeros(p, dtype=np.int32)
        info = PlanInfo()
        self._check(self._lib.swi_plan_windows_sampled(self._h, int(n_r), int(p), C.byref(o), _ptr(s), _ptr(n),
                                                       C.byref(info)))
        return s[:info.windows], n[:info.windows], info.as_dict()

    # -- operator
    def apply(self, X, sigma):
        """(A - sigma_c) X[:, c] for X of shape (N, nvec) complex128 (numpy or torch CUDA)."""
        sig = _c_arr(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (X.shape[1],)), np.float64)
        if _is_device(X):
            import torch
            Y = torch.empty_like(X)
            self._check(self._lib.swi_apply(self._h, X.shape[1], _ptr(sig), _ptr(X), _ptr(Y), 1))
            return Y
        X = _c_arr(X, np.complex128)
        Y = np.empty_like(X)
        self._check(self._lib.swi_apply(self._h, X.shape[1], _ptr(sig), _ptr(X), _ptr(Y), 0))
        return Y

    def apply_ds(self, X, sigma):
        """apply() in double-single arithmetic (the operator of the double-single Krylov loop)."""
        sig = _c_arr(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (X.shape[1],)), np.float64)
        if _is_device(X):
            import torch
            Y = torch.empty_like(X)
            self._check(self._lib.swi_apply_ds(self._h, X.shape[1], _ptr(sig), _ptr(X), _ptr(Y), 1))
            return Y
        X = _c_arr(X, np.complex128)
        Y = np.empty_like(X)
        self._check(self._lib.swi_apply_ds(self._h, X.shape[1], _ptr(sig), _ptr(X), _ptr(Y), 0))
        return Y

    def apply_c64(self, X, sigma):
        """(A - sigma_c) X[:, c] on complex64 vectors in FP32 arithmetic (numpy, or a torch CUDA
        tensor: then the call is ordered on the context's stream and does not synchronise)."""
        sig = _c_arr(np.broadcast_to(np.asarray(sigma, dtype=np.float32), (X.shape[1],)), np.float32)
        if _is_device(X):
            import torch
            Y = torch.empty_like(X)
            self._check(self._lib.swi_apply_c64(self._h, X.shape[1], _ptr(sig), _ptr(X), _ptr(Y), 1))
            return Y
        X = _c_arr(X, np.complex64)
        Y = np.empty_like(X)
        self._check(self._lib.swi_apply_c64(self._h, X.shape[1], _ptr(sig), _ptr(X), _ptr(Y), 0))
        return Y

    # -- solve
    def solve(self, block=2, rel_tol=1e-10, max_basis=0, keep=0, max_matvecs=0, eq_rtol=0.0, drop_tol=0.0,
              seed=1, n_keep=0, arith=ARITH_DS, allow=(SWI_OK, SWI_ENOCONV, SWI_HOLES)):
        """Windowed solve; arith = ARITH_DS (double-single products, default) or ARITH_F64 (native).

        block=1 runs single-vector windows (complex128 bases, double-single products), block=2
        the same loop with two new vectors per window and step (both vectors of a doubly
        degenerate eigenvalue); a PREC_MIXED context runs only these, on complex64 bases
        (block 0, 1 or 2)."""
        o = SolveOpts(block=block, max_basis=max_basis, keep=keep, max_matvecs=max_matvecs, rel_tol=rel_tol,
                      eq_rtol=eq_rtol, drop_tol=drop_tol, seed=seed, n_keep=n_keep, arith=arith)
        info = SolveInfo()
        rc = self._check(self._lib.swi_solve(self._h, C.byref(o), C.byref(info)), allow)
        d = info.as_dict()
        d["status"] = STATUS_NAMES[rc]
        return d

    def solve_more(self, sigma, n_req, block=2, rel_tol=1e-10, max_basis=0, keep=0, max_matvecs=0, eq_rtol=0.0,
                   drop_tol=0.0, seed=1, n_keep=0, arith=ARITH_DS, allow=(SWI_OK, SWI_ENOCONV, SWI_HOLES)):
        """Continuation: solve new windows and merge them with the current pairs (Algorithm 2)."""
        s, n = _c_arr(sigma, np.float64), _c_arr(n_req, np.int32)
        o = SolveOpts(block=block, max_basis=max_basis, keep=keep, max_matvecs=max_matvecs, rel_tol=rel_tol,
                      eq_rtol=eq_rtol, drop_tol=drop_tol, seed=seed, n_keep=n_keep, arith=arith)
        info = SolveInfo()
        rc = self._check(self._lib.swi_solve_more(self._h, len(s), _ptr(s), _ptr(n), C.byref(o), C.byref(info)), allow)
        d = info.as_dict()
        d["status"] = STATUS_NAMES[rc]
        return d

    def fill_holes(self, e_min, e_max, max_rounds=0, block=2, rel_tol=1e-10, max_basis=0, keep=0, max_matvecs=0,
                   eq_rtol=0.0, drop_tol=0.0, seed=1, n_keep=0, arith=ARITH_DS,
                   allow=(SWI_OK, SWI_ENOCONV, SWI_HOLES)):
        """Algorithm 1's hole loop on the current windows; returns the info dict with "status", "windows_added"."""
        o = SolveOpts(block=block, max_basis=max_basis, keep=keep, max_matvecs=max_matvecs, rel_tol=rel_tol,
                      eq_rtol=eq_rtol, drop_tol=drop_tol, seed=seed, n_keep=n_keep, arith=arith)
        info = SolveInfo()
        added = C.c_int()
        rc = self._check(self._lib.swi_fill_holes(self._h, float(e_min), float(e_max), int(max_rounds), C.byref(o),
                                                  C.byref(info), C.byref(added)), allow)
        d = info.as_dict()
        d["status"] = STATUS_NAMES[rc]
        d["windows_added"] = added.value
        return d

    def windows(self):
        """(sigma[p], holes[p]) of the current pairs' windows (holes[j]: interface j, j + 1 without redundancy)."""
        p = C.c_int()
        self._check(self._lib.swi_get_windows(self._h, 0, None, None, C.byref(p)))
        s = np.zeros(max(1, p.value))
        h = np.zeros(max(1, p.value), dtype=np.int32)
        self._check(self._lib.swi_get_windows(self._h, p.value, _ptr(s), _ptr(h), C.byref(p)))
        return s[:p.value], h[:p.value]

    def window_info(self):
        p = C.c_int()
        self._check(self._lib.swi_get_window_info(self._h, 0, None, C.byref(p)))
        arr = (WindowInfo * max(1, p.value))()
        self._check(self._lib.swi_get_window_info(self._h, p.value, arr, C.byref(p)))
        return [{f[0]: getattr(arr[j], f[0]) for f in WindowInfo._fields_} for j in range(p.value)]

    def n_pairs(self):
        n = C.c_int()
        self._check(self._lib.swi_get_eigenpairs(self._h, C.byref(n), None, None, None))
        return n.value

    def eigenpairs(self):
        """(eps[n], U[N, n]) copied to host numpy arrays."""
        n = self.n_pairs()
        eps = np.empty(n, dtype=np.complex128)
        U = np.empty((self.N, n), dtype=np.complex128)
        self._check(self._lib.swi_copy_eigenpairs(self._h, _ptr(eps), _ptr(U), 0))
        return eps, U

    def eigenvalues(self):
        n = self.n_pairs()
        eps = np.empty(n, dtype=np.complex128)
        self._check(self._lib.swi_copy_eigenpairs(self._h, _ptr(eps), None, 0))
        return eps

    def set_eigenpairs(self, eps, U):
        if _is_device(U):
            return self._check(self._lib.swi_set_eigenpairs(self._h, U.shape[1], _ptr(eps), _ptr(U), 1))
        e, Uc = _c_arr(eps, np.complex128), _c_arr(U, np.complex128)
        return self._check(self._lib.swi_set_eigenpairs(self._h, Uc.shape[1], _ptr(e), _ptr(Uc), 0))

    def refine(self, max_sweeps=3, group=16, rel_tol=1e-10, arith=ARITH_DS, eq_rtol=0.0, drop_tol=0.0,
               near_tol=0.0, allow=(SWI_OK, SWI_ENOCONV)):
        """Residual-correction sweeps on the current pairs (Rayleigh-Ritz on span[U_g, R_u] per group of
        `group` consecutive pairs, then Algorithm 2 as one window); returns the info dict with "status"."""
        o = RefineOpts(max_sweeps=max_sweeps, group=group, arith=arith, rel_tol=rel_tol, eq_rtol=eq_rtol,
                       drop_tol=drop_tol, near_tol=near_tol)
        info = RefineInfo()
        rc = self._check(self._lib.swi_refine(self._h, C.byref(o), C.byref(info)), allow)
        d = info.as_dict()
        d["status"] = STATUS_NAMES[rc]
        return d

    def residuals(self):
        r = np.empty(self.n_pairs())
        self._check(self._lib.swi_residuals(self._h, _ptr(r)))
        return r

    # -- transport
    def transmission(self, E):
        E = _c_arr(np.atleast_1d(E), np.float64)
        T = np.empty_like(E)
        self._check(self._lib.swi_transmission(self._h, len(E), _ptr(E), _ptr(T)))
        return T

    def set_contraction(self, contraction):
        """Arithmetic of transmission() and grad(): CONTRACT_F64 (default) or CONTRACT_F32
        (FP32 products with FP32 accumulation for the projections and the adjoint)."""
        return self._check(self._lib.swi_set_contraction(self._h, int(contraction)))

    def transmission_noalloc(self, E):
        """T(E) through swi_transmission_noalloc: no device allocation during the call.

        For callers that must not allocate device memory while it runs (a host
        framework that owns the whole memory budget); at most 64 pairs and 1024
        energies, and calls must not overlap on the GPU (shared scratch).
        """
        E = _c_arr(np.atleast_1d(E), np.float64)
        T = np.empty_like(E)
        self._check(self._lib.swi_transmission_noalloc(self._h, len(E), _ptr(E), _ptr(T)))
        return T

    def check_schur(self, H, B=None, keep=None, arith=ARITH_DS):
        """The device's thick-restart Schur step on a host matrix H (m x m): (T, Z, info) with
        H Z = Z T, the `keep` Ritz values of smallest magnitude first; info = (kept, -, status, work)."""
        H = _c_arr(np.asarray(H), np.complex128)
        m = H.shape[0]
        b = 1 if B is None else np.atleast_2d(B).shape[0]
        Bc = None if B is None else _c_arr(np.atleast_2d(B), np.complex128)
        keep = m // 2 if keep is None else int(keep)
        T = np.empty((m, m), np.complex128)
        Z = np.empty((m, m), np.complex128)
        info = np.zeros(4, np.int32)
        self._check(self._lib.swi_check_schur(self._h, m, b, keep, _ptr(H), None if Bc is None else _ptr(Bc), int(arith),
                                              _ptr(T), _ptr(Z), _ptr(info)))
        return T, Z, info

    def grad(self, E, dLdT, dLdV_out=None):
        """(dL/dV[N], dL/dE[nE]) for the weights dL/dT (dL/dE_e = dLdT_e dT_e/dE_e).

        dLdV_out may be a torch CUDA float64 tensor of length N."""
        E = _c_arr(np.atleast_1d(E), np.float64)
        w = _c_arr(np.atleast_1d(dLdT), np.float64)
        dE = np.empty_like(E)
        if dLdV_out is not None and _is_device(dLdV_out):
            self._check(self._lib.swi_grad(self._h, len(E), _ptr(E), _ptr(w), _ptr(dLdV_out), 1, _ptr(dE)))
            return dLdV_out, dE
        dV = np.empty(self.N)
        self._check(self._lib.swi_grad(self._h, len(E), _ptr(E), _ptr(w), _ptr(dV), 0, _ptr(dE)))
        return dV, dE

    def launch_count(self):
        return int(self._lib.swi_launch_count(self._h))

    def profile(self, enable=True):
        """Start (and clear) or stop per-kernel-class CUDA-event timing."""
        return self._check(self._lib.swi_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{class: {launches, ms, flops, bytes}} summed over the recorded launches."""
        arr = (KernelStats * len(KERNEL_CLASSES))()
        self._check(self._lib.swi_profile_read(self._h, arr))
        return {name: {"launches": arr[k].launches, "ms": arr[k].ms, "flops": arr[k].flops,
                       "bytes": arr[k].bytes} for k, name in enumerate(KERNEL_CLASSES)}


def solve_batch(contexts, block=2, rel_tol=1e-10, max_basis=0, keep=0, max_matvecs=0, eq_rtol=0.0, drop_tol=0.0,
                seed=1, n_keep=0, arith=ARITH_DS, workers=0):
    """swi_solve_batch: the windows of several contexts (systems of uneven grids) solved at once.

    Returns one info dict per context (with "status"); contexts keep their merged pairs."""
    lib = load()
    n = len(contexts)
    handles = (C.c_void_p * n)(*[c._h for c in contexts])
    o = SolveOpts(block=block, max_basis=max_basis, keep=keep, max_matvecs=max_matvecs, rel_tol=rel_tol,
                  eq_rtol=eq_rtol, drop_tol=drop_tol, seed=seed, n_keep=n_keep, arith=arith)
    infos = (SolveInfo * n)()
    st = np.zeros(n, dtype=np.int32)
    rc = lib.swi_solve_batch(n, C.cast(handles, C.c_void_p), C.byref(o), int(workers), infos, _ptr(st))
    if rc == SWI_EINVAL and np.all(st == 0):
        raise SwiError(rc, lib.swi_last_error(None).decode())
    out = []
    for k in range(n):
        d = infos[k].as_dict()
        d["status"] = STATUS_NAMES[int(st[k])]
        out.append(d)
    return out


def transmission_function():
    """torch.autograd.Function: T(E) forward through the library, adjoint dT/dV and dT/dE backward.

    ``TransmissionFn.apply(V, E, ctx)``: V is a float64 tensor of the potential
    (the context must already hold the eigenpairs of A(V)); E a float64 tensor
    of energies.  Backward returns dL/dV (length N, on V's device) and dL/dE.
    """
    import torch

    class TransmissionFn(torch.autograd.Function):
        @staticmethod
        def forward(fctx, V, E, sctx):
            fctx.sctx = sctx
            fctx.E = E.detach().cpu().numpy().astype(np.float64)
            fctx.V_device = V.device
            T = sctx.transmission(fctx.E)
            return torch.as_tensor(T, dtype=torch.float64, device=E.device)

        @staticmethod
        def backward(fctx, gT):
            w = gT.detach().cpu().numpy().astype(np.float64)
            if fctx.V_device.type == "cuda":
                dV = torch.empty(fctx.sctx.N, dtype=torch.float64, device=fctx.V_device)
                dV, dLdE = fctx.sctx.grad(fctx.E, w, dLdV_out=dV)
            else:
                dVn, dLdE = fctx.sctx.grad(fctx.E, w)
                dV = torch.as_tensor(dVn, dtype=torch.float64)
            dE = torch.as_tensor(dLdE, dtype=torch.float64, device=gT.device)
            return dV, dE, None

    return TransmissionFn
