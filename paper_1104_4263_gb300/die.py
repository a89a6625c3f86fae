"""Thin Python binding of libdie (ctypes): argument marshalling only.

Every step of the computation runs in the CUDA library; this module converts
PyTorch tensors to device pointers and streams, and C status codes to exceptions.
It never falls back to any other implementation: if the library is missing or the
GPU is absent, the calls raise.

Vectors are torch tensors on the current CUDA device, shape (2, n2, n1) (or flat
2*n1*n2), dtype complex128 (or complex64 for the FP32 operator products).
"""
from __future__ import annotations

import ctypes as ct
import math
import os

from .build import LIB

DIE_FP64 = 0
DIE_FP32_INNER = 1

STATUS = {0: "DIE_OK", 1: "DIE_EINVAL", 2: "DIE_ENOMEM", 3: "DIE_ECUDA", 4: "DIE_ESINGULAR",
          5: "DIE_ENOCONV", 6: "DIE_EBREAKDOWN", 7: "DIE_ENAN", 8: "DIE_ETIMEOUT", 9: "DIE_EUNSUPPORTED"}


class DieError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)} ({_lib().die_status_str(code).decode()})")


DIE_TE = 0
DIE_TM = 1
DIE_TE_MAG = 2          # (E1, E2, H3) with magnetic contrast: three planes


class Desc(ct.Structure):
    _fields_ = [("n1", ct.c_int), ("n2", ct.c_int), ("h", ct.c_double), ("k_b", ct.c_double),
                ("prec", ct.c_int), ("M1", ct.c_int), ("M2", ct.c_int), ("pol", ct.c_int)]


class GmresOpts(ct.Structure):
    _fields_ = [("restart", ct.c_int), ("max_iters", ct.c_int), ("tol", ct.c_double), ("regularized", ct.c_int),
                ("use_x0", ct.c_int), ("inner", ct.c_int), ("timing", ct.c_int), ("reorth_eta", ct.c_double),
                ("graph", ct.c_int)]


class GmresReport(ct.Structure):
    _fields_ = [("cycles", ct.c_int), ("iters", ct.c_int), ("n_apply", ct.c_int),
                ("rel_res_solved", ct.c_double), ("rel_res_orig", ct.c_double),
                ("t_matvec", ct.c_double), ("t_orth", ct.c_double), ("t_defl", ct.c_double),
                ("t_total", ct.c_double), ("history", ct.POINTER(ct.c_double)), ("history_cap", ct.c_int),
                ("history_len", ct.c_int), ("n_reorth", ct.c_int), ("graph_cycles", ct.c_int)]


class DeflOpts(ct.Structure):
    _fields_ = [("r", ct.c_int), ("r_max", ct.c_int), ("tol", ct.c_double), ("regularized", ct.c_int),
                ("inner", ct.c_int), ("krylov_dim", ct.c_int), ("max_restarts", ct.c_int),
                ("seed", ct.c_ulonglong)]


class FnoDesc(ct.Structure):
    _fields_ = [("c_in", ct.c_int), ("c_out", ct.c_int), ("width", ct.c_int), ("modes", ct.c_int),
                ("layers", ct.c_int), ("hidden", ct.c_int), ("H", ct.c_int), ("W", ct.c_int), ("max_batch", ct.c_int)]


ABI_VERSION = 3
STRUCTS = (Desc, GmresOpts, GmresReport, DeflOpts)     # the order of die_abi_sizes


EXPORTS = {
    "dieop_create": (ct.c_int, [ct.POINTER(Desc), ct.c_void_p, ct.c_int, ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "dieop_info": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_longlong)]),
    "dieop_set_permittivity": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p]),
    "dieop_set_permeability": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p]),
    "dieop_autotune": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.POINTER(ct.c_int), ct.POINTER(ct.c_double)]),
    "dieop_set_tile_rows": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "dieop_tile_rows": (ct.c_int, [ct.c_void_p]),
    "fno_encode_pair": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "dieop_apply": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "dieop_apply_regularized": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "dieop_apply_regularizer": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "dieop_apply_batch": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p]),
    "dieop_rhs_plane_wave": (ct.c_int, [ct.c_void_p, ct.c_double, ct.c_void_p, ct.c_void_p]),
    "dieop_destroy": (None, [ct.c_void_p]),
    "gmres_solve": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.POINTER(GmresOpts), ct.c_void_p, ct.c_void_p,
                               ct.POINTER(GmresReport), ct.c_void_p]),
    "gmres_basis": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p]),
    "gmres_solve_batch": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.POINTER(GmresOpts), ct.c_int, ct.c_void_p,
                                     ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "gmres_solve_many": (ct.c_int, [ct.c_int, ct.c_void_p, ct.c_void_p, ct.POINTER(GmresOpts), ct.c_void_p,
                                    ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "deflation_build": (ct.c_int, [ct.c_void_p, ct.POINTER(DeflOpts), ct.c_void_p, ct.POINTER(ct.c_void_p),
                                   ct.POINTER(ct.c_double), ct.POINTER(ct.c_int)]),
    "deflation_apply": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "deflation_apply_noalloc": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "deflation_destroy": (None, [ct.c_void_p]),
    "die_deflation_radius": (ct.c_double, [ct.c_void_p, ct.c_longlong, ct.c_int]),
    "die_memory_plan": (ct.c_int, [ct.c_double, ct.c_double, ct.c_double, ct.c_double, ct.c_double,
                                   ct.POINTER(ct.c_double)]),
    "die_prof_begin": (ct.c_int, []),
    "die_prof_end": (ct.c_int, []),
    "die_prof_kernels": (ct.c_int, []),
    "die_prof_name": (ct.c_char_p, [ct.c_int]),
    "die_prof_read": (ct.c_int, [ct.c_int, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_double)]),
    "die_status_str": (ct.c_char_p, [ct.c_int]),
    "die_fp64_peak": (ct.c_int, [ct.POINTER(ct.c_double), ct.c_void_p]),
    "die_gemm_bf16": (ct.c_int, [ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_float, ct.c_void_p, ct.c_longlong,
                                 ct.c_longlong, ct.c_longlong, ct.c_void_p, ct.c_longlong, ct.c_longlong,
                                 ct.c_longlong, ct.c_float, ct.c_void_p, ct.c_longlong, ct.c_longlong,
                                 ct.c_longlong, ct.c_int, ct.c_void_p]),
    "fno_create": (ct.c_int, [ct.POINTER(FnoDesc), ct.POINTER(ct.c_void_p)]),
    "fno_destroy": (None, [ct.c_void_p]),
    "fno_param_count": (ct.c_longlong, [ct.c_void_p]),
    "fno_set_params": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "fno_get_params": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "fno_forward": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "fno_backward": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "fno_zero_grads": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "fno_get_grads": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "fno_train_step": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_float,
                                  ct.POINTER(ct.c_float), ct.c_void_p]),
    "fno_precondition": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "fgmres_solve": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.POINTER(GmresOpts), ct.c_int, ct.c_int,
                                ct.c_void_p, ct.c_void_p, ct.POINTER(GmresReport), ct.POINTER(ct.c_int), ct.c_void_p]),
    "die_abi_version": (ct.c_int, []),
    "die_abi_sizes": (ct.c_int, [ct.POINTER(ct.c_longlong), ct.c_int]),
}

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libdie is not built ({LIB} missing): run __graft_entry__.build() "
                               "or python -m paper_1104_4263_gb300.build")
        lib = ct.CDLL(LIB)
        for name, (res, args) in EXPORTS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if lib.die_abi_version() != ABI_VERSION:
            raise RuntimeError("libdie ABI version mismatch")
        sizes = (ct.c_longlong * 4)()
        if lib.die_abi_sizes(sizes, 4) != 0 or list(sizes) != [ct.sizeof(t) for t in STRUCTS]:
            raise RuntimeError("libdie structure layouts differ from the binding's")
        _LIB = lib
    return _LIB


def lib():
    """The loaded ctypes library (loads it on first use)."""
    return _lib()


def _check(code: int, what: str):
    if code != 0:
        raise DieError(code, what)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


def _ptr(t):
    if not t.is_cuda:
        raise ValueError("libdie takes CUDA tensors (device memory)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ct.c_void_p(t.data_ptr())


def deflation_radius(eps_r) -> float:
    """Section 5 deflation radius for a permittivity map (numpy complex array)."""
    import numpy as np
    e = np.ascontiguousarray(np.asarray(eps_r, dtype=np.complex128).reshape(-1))
    return float(_lib().die_deflation_radius(e.ctypes.data_as(ct.c_void_p), e.size, 1000))


def fp64_peak_tflops(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device (die_fp64_peak), TFLOP/s."""
    v = ct.c_double()
    _check(_lib().die_fp64_peak(ct.byref(v), _stream(stream)), "die_fp64_peak")
    return float(v.value)


def memory_plan(M: float, beta: float, x: float, k_ppw: float, eps_max: float) -> dict:
    """Section 5's memory rule (die_memory_plan): N_max, [a/lambda]_max and alpha."""
    out = (ct.c_double * 3)()
    _check(_lib().die_memory_plan(float(M), float(beta), float(x), float(k_ppw), float(eps_max), out),
           "die_memory_plan")
    return {"N_max": out[0], "a_over_lambda_max": out[1], "alpha": out[2]}


class KernelTimer:
    """Context manager: per-kernel-class launch counts and total milliseconds
    (CUDA events around every library launch inside the block)."""

    def __enter__(self):
        _check(_lib().die_prof_begin(), "die_prof_begin")
        self.result = {}
        return self

    def __exit__(self, *exc):
        code = _lib().die_prof_end()
        L = _lib()
        for i in range(L.die_prof_kernels()):
            n = ct.c_longlong()
            ms = ct.c_double()
            _check(L.die_prof_read(i, ct.byref(n), ct.byref(ms)), "die_prof_read")
            if n.value:
                self.result[L.die_prof_name(i).decode()] = {"launches": n.value, "ms": ms.value}
        self.overflow = code != 0
        return False


class Operator:
    """The discretised TE operator A = I - G X on an n1 x n2 grid (a dieop_t handle).
    pol = DIE_TE_MAG: the (E1, E2, H3) system with magnetic contrast mu_r (field vectors
    of shape (3, n2, n1))."""

    def __init__(self, eps_r, h: float, k_b: float = 2 * math.pi, prec: int = DIE_FP64,
                 M1: int = 0, M2: int = 0, stream=None, pol: int = DIE_TE, mu_r=None):
        import numpy as np
        import torch
        eps = eps_r
        if isinstance(eps, torch.Tensor):
            eps_t = eps.to(torch.complex128).contiguous()
            n2, n1 = eps_t.shape
            on_dev = 1 if eps_t.is_cuda else 0
            if not on_dev:
                eps_np = eps_t.numpy()
        else:
            eps_np = np.ascontiguousarray(np.asarray(eps, dtype=np.complex128))
            n2, n1 = eps_np.shape
            on_dev = 0
        self.n1, self.n2, self.h, self.k_b, self.prec, self.pol = n1, n2, h, k_b, prec, pol
        desc = Desc(n1, n2, h, k_b, prec, M1, M2, pol)
        handle = ct.c_void_p()
        ptr = _ptr(eps_t) if on_dev else eps_np.ctypes.data_as(ct.c_void_p)
        _check(_lib().dieop_create(ct.byref(desc), ptr, on_dev, _stream(stream), ct.byref(handle)), "dieop_create")
        self._h = handle
        info = (ct.c_longlong * 6)()
        _check(_lib().dieop_info(self._h, info), "dieop_info")
        self.M1, self.M2 = int(info[2]), int(info[3])
        self.N = n1 * n2
        self.planes = 3 if pol == DIE_TE_MAG else 2
        if mu_r is not None:
            self.set_permeability(mu_r, stream)

    @property
    def handle(self):
        return self._h

    def set_permittivity(self, eps_r, stream=None):
        """Replace the permittivity map (same grid and h; deflation handles of the old map
        become invalid)."""
        import numpy as np
        import torch
        if isinstance(eps_r, torch.Tensor) and eps_r.is_cuda:
            e = eps_r.to(torch.complex128).contiguous()
            if tuple(e.shape) != (self.n2, self.n1):
                raise ValueError("eps_r must have shape (n2, n1)")
            _check(_lib().dieop_set_permittivity(self._h, _ptr(e), 1, _stream(stream)), "dieop_set_permittivity")
            return
        e = np.ascontiguousarray(np.asarray(eps_r, dtype=np.complex128))
        if e.shape != (self.n2, self.n1):
            raise ValueError("eps_r must have shape (n2, n1)")
        _check(_lib().dieop_set_permittivity(self._h, e.ctypes.data_as(ct.c_void_p), 0, _stream(stream)),
               "dieop_set_permittivity")

    def autotune(self, force: bool = False, stream=None) -> dict:
        """Time the complex64 regularised product at every tile height of the row passes
        and keep the fastest (dieop_autotune); returns the height and the microseconds per
        product at heights 1, 2, 4, 8 (0: not a candidate, or reused without timing)."""
        tr = ct.c_int()
        us = (ct.c_double * 4)()
        _check(_lib().dieop_autotune(self._h, int(bool(force)), _stream(stream), ct.byref(tr), us), "dieop_autotune")
        return {"tile_rows": tr.value, "us_per_product": {h: us[i] for i, h in enumerate((1, 2, 4, 8))}}

    def set_tile_rows(self, rows: int):
        """Tile height of the complex64 row passes: 0 (default), 1, 2, 4 or 8."""
        _check(_lib().dieop_set_tile_rows(self._h, int(rows)), "dieop_set_tile_rows")

    @property
    def tile_rows(self) -> int:
        return _lib().dieop_tile_rows(self._h)

    def set_permeability(self, mu_r, stream=None):
        """The relative permeability map of a DIE_TE_MAG operator (chi_m = mu_r - 1)."""
        import numpy as np
        import torch
        if isinstance(mu_r, torch.Tensor) and mu_r.is_cuda:
            m = mu_r.to(torch.complex128).contiguous()
            if tuple(m.shape) != (self.n2, self.n1):
                raise ValueError("mu_r must have shape (n2, n1)")
            _check(_lib().dieop_set_permeability(self._h, _ptr(m), 1, _stream(stream)), "dieop_set_permeability")
            return
        m = np.ascontiguousarray(np.asarray(mu_r, dtype=np.complex128))
        if m.shape != (self.n2, self.n1):
            raise ValueError("mu_r must have shape (n2, n1)")
        _check(_lib().dieop_set_permeability(self._h, m.ctypes.data_as(ct.c_void_p), 0, _stream(stream)),
               "dieop_set_permeability")

    def close(self):
        if getattr(self, "_h", None):
            _lib().dieop_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _io_dtype(self):
        import torch
        return torch.complex128 if self.prec == DIE_FP64 else torch.complex64

    def _out(self, x, y):
        import torch
        if x.dtype != self._io_dtype():
            raise TypeError(f"expected {self._io_dtype()}, got {x.dtype}")
        if x.numel() != self.planes * self.N:
            raise ValueError("vector must hold planes * n1 * n2 complex values")
        return torch.empty_like(x) if y is None else y

    def apply(self, x, y=None, stream=None):
        """y = A x (Eqs. (4.1)-(4.5))."""
        y = self._out(x, y)
        _check(_lib().dieop_apply(self._h, _ptr(x), _ptr(y), _stream(stream)), "dieop_apply")
        return y

    def apply_regularized(self, x, y=None, stream=None):
        """y = A(chi') A(chi) x (Eq. (3.19), Section 5)."""
        y = self._out(x, y)
        _check(_lib().dieop_apply_regularized(self._h, _ptr(x), _ptr(y), _stream(stream)), "dieop_apply_regularized")
        return y

    def apply_batch(self, x, y=None, regularized: bool = False, stream=None):
        """y_k = A x_k, or A(chi') A(chi) x_k when regularized, for the leading dimension k
        of x (shape (nrhs, 2, n2, n1)), in one launch per pass."""
        import torch
        if not isinstance(x, torch.Tensor) or not x.is_cuda or not x.is_contiguous():
            raise TypeError("x must be a contiguous CUDA tensor")
        if x.dtype != self._io_dtype():
            raise TypeError(f"expected {self._io_dtype()}, got {x.dtype}")
        if x.dim() < 1 or x.numel() % (self.planes * self.N) != 0:
            raise ValueError("x must hold nrhs field vectors of 2 * n1 * n2 complex values")
        nrhs = x.numel() // (self.planes * self.N)
        y = torch.empty_like(x) if y is None else y
        _check(_lib().dieop_apply_batch(self._h, nrhs, _ptr(x), _ptr(y), int(bool(regularized)), _stream(stream)),
               "dieop_apply_batch")
        return y

    def apply_regularizer(self, x, y=None, stream=None):
        """y = A(chi') x."""
        y = self._out(x, y)
        _check(_lib().dieop_apply_regularizer(self._h, _ptr(x), _ptr(y), _stream(stream)), "dieop_apply_regularizer")
        return y

    def plane_wave(self, psi: float, out=None, stream=None):
        """Incident TE plane wave at angle psi (complex128, shape (planes, n2, n1))."""
        import torch
        b = torch.empty((self.planes, self.n2, self.n1), dtype=torch.complex128, device="cuda") if out is None else out
        _check(_lib().dieop_rhs_plane_wave(self._h, float(psi), _ptr(b), _stream(stream)), "dieop_rhs_plane_wave")
        return b

    def solve(self, b, x=None, restart: int = 30, tol: float = 1e-6, max_iters: int = 100000,
              regularized: bool = False, inner: int = DIE_FP64, deflation: "Deflation | None" = None,
              timing: bool = False, history: int = 0, stream=None, raise_on_noconv: bool = False,
              reorth_eta: float = 0.0, graph: bool = False):
        """Restarted GMRES; returns (x, report dict).  x (complex128) may hold an initial guess.
        graph: run each cycle's Arnoldi steps as one CUDA graph launch (captured once)."""
        import numpy as np
        import torch
        if b.dtype != torch.complex128:
            raise TypeError("solve takes complex128 vectors")
        use_x0 = x is not None
        if x is None:
            x = torch.empty_like(b)
        opts = GmresOpts(restart, max_iters, tol, int(bool(regularized)), int(use_x0), inner, int(bool(timing)),
                         float(reorth_eta), int(bool(graph)))
        rep = GmresReport()
        hist = None
        if history > 0:
            hist = np.zeros(history, dtype=np.float64)
            rep.history = hist.ctypes.data_as(ct.POINTER(ct.c_double))
            rep.history_cap = history
        d = deflation.handle if deflation is not None else None
        code = _lib().gmres_solve(self._h, d, ct.byref(opts), _ptr(b), _ptr(x), ct.byref(rep), _stream(stream))
        if code not in (0, 5) or (code == 5 and raise_on_noconv):
            raise DieError(code, "gmres_solve")
        out = {"status": STATUS[code], "converged": code == 0, "cycles": rep.cycles, "iters": rep.iters,
               "n_apply": rep.n_apply, "rel_res_solved": rep.rel_res_solved, "rel_res_orig": rep.rel_res_orig,
               "t_matvec": rep.t_matvec, "t_orth": rep.t_orth, "t_defl": rep.t_defl, "t_total": rep.t_total,
               "n_reorth": rep.n_reorth, "graph_cycles": rep.graph_cycles}
        if hist is not None:
            out["history"] = hist[:rep.history_len].copy()
        return x, out

    def basis(self, first: int, count: int, stream=None):
        """Vectors first .. first + count - 1 of the Krylov basis the last gmres_solve on
        this operator left (complex128, shape (count, 2, n2, n1)); see gmres_basis."""
        import torch
        out = torch.empty((count, self.planes, self.n2, self.n1), dtype=torch.complex128, device="cuda")
        _check(_lib().gmres_basis(self._h, int(first), int(count), _ptr(out), _stream(stream)), "gmres_basis")
        return out

    def solve_batch(self, B, X=None, restart: int = 30, tol: float = 1e-6, max_iters: int = 100000,
                    regularized: bool = False, inner: int = DIE_FP64, deflation: "Deflation | None" = None,
                    stream=None, reorth_eta: float = 0.0, graph: bool = False):
        """Concurrent restarted GMRES on the right-hand sides B[k] (complex128, shape
        (nrhs, 2, n2, n1)); returns (X, list of report dicts)."""
        import torch
        if B.dtype != torch.complex128 or not B.is_cuda or not B.is_contiguous():
            raise TypeError("solve_batch takes a contiguous complex128 CUDA tensor")
        if B.numel() % (self.planes * self.N) != 0:
            raise ValueError("B must hold nrhs field vectors of planes * n1 * n2 values")
        nrhs = B.numel() // (self.planes * self.N)
        use_x0 = X is not None
        if X is None:
            X = torch.empty_like(B)
        opts = GmresOpts(restart, max_iters, tol, int(bool(regularized)), int(use_x0), inner, 0, float(reorth_eta),
                         int(bool(graph)))
        reps = (GmresReport * nrhs)()
        d = deflation.handle if deflation is not None else None
        code = _lib().gmres_solve_batch(self._h, d, ct.byref(opts), nrhs, _ptr(B), _ptr(X),
                                        ct.cast(reps, ct.c_void_p), _stream(stream))
        if code not in (0, 5):
            raise DieError(code, "gmres_solve_batch")
        outs = []
        for r in reps:
            ok = r.rel_res_solved <= tol
            outs.append({"converged": bool(ok), "cycles": r.cycles, "iters": r.iters, "n_apply": r.n_apply,
                         "rel_res_solved": r.rel_res_solved, "rel_res_orig": r.rel_res_orig,
                         "t_total": r.t_total, "n_reorth": r.n_reorth, "graph_cycles": r.graph_cycles})
        return X, outs


class Deflation:
    """P^-1 = I + V (T^-1 - I) V^* for the r largest-magnitude eigenvalues (Eq. (4.12))."""

    def __init__(self, op: Operator, r: int, tol: float = 1e-4, regularized: bool = True,
                 inner: int = DIE_FP64, krylov_dim: int = 0, max_restarts: int = 0, seed: int = 0,
                 r_max: int = 0, stream=None, allow_noconv: bool = True):
        self.op = op
        opts = DeflOpts(r, r_max, tol, int(bool(regularized)), inner, krylov_dim, max_restarts, seed)
        cap = max(r, r_max, 64)
        eig = (ct.c_double * (2 * cap))()
        rout = ct.c_int(0)
        h = ct.c_void_p()
        code = _lib().deflation_build(op.handle, ct.byref(opts), _stream(stream), ct.byref(h), eig, ct.byref(rout))
        if code != 0 and not (code == 5 and allow_noconv and h.value):
            raise DieError(code, "deflation_build")
        self._h = h
        self.converged = code == 0
        self.r = rout.value
        import numpy as np
        e = np.array(eig[:2 * self.r]).reshape(-1, 2)
        self.eigenvalues = e[:, 0] + 1j * e[:, 1]

    @property
    def handle(self):
        return self._h

    def apply(self, x, z=None, stream=None):
        import torch
        z = torch.empty_like(x) if z is None else z
        _check(_lib().deflation_apply(self._h, _ptr(x), _ptr(z), _stream(stream)), "deflation_apply")
        return z

    def close(self):
        if getattr(self, "_h", None):
            _lib().deflation_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_many(ops, bs, deflations=None, xs=None, restart: int = 30, tol: float = 1e-6, max_iters: int = 100000,
               regularized: bool = False, inner: int = DIE_FP64, stream=None, reorth_eta: float = 0.0,
               graph: bool = False):
    """Concurrent restarted GMRES on systems of different operators (gmres_solve_many):
    system k solves ops[k] with deflations[k] (or None) from bs[k] (complex128 CUDA tensor
    of shape (2, n2, n1) of ops[k]); xs: None or initial guesses.  Returns (xs, reports)."""
    import torch
    count = len(ops)
    if len(bs) != count or (deflations is not None and len(deflations) != count):
        raise ValueError("ops, bs and deflations must have the same length")
    for op, b in zip(ops, bs):
        if b.dtype != torch.complex128 or not b.is_cuda or not b.is_contiguous() or b.numel() != op.planes * op.N:
            raise TypeError("solve_many takes contiguous complex128 CUDA tensors of 2 * n1 * n2 values")
    use_x0 = xs is not None
    xs = [torch.empty_like(b) for b in bs] if xs is None else list(xs)
    opts = GmresOpts(restart, max_iters, tol, int(bool(regularized)), int(use_x0), inner, 0, float(reorth_eta),
                     int(bool(graph)))
    hops = (ct.c_void_p * count)(*[op.handle for op in ops])
    hdef = None
    if deflations is not None:
        hdef = (ct.c_void_p * count)(*[d.handle if d is not None else None for d in deflations])
    pb = (ct.c_void_p * count)(*[_ptr(b) for b in bs])
    px = (ct.c_void_p * count)(*[_ptr(x) for x in xs])
    reps = (GmresReport * count)()
    code = _lib().gmres_solve_many(count, ct.cast(hops, ct.c_void_p), ct.cast(hdef, ct.c_void_p) if hdef else None,
                                   ct.byref(opts), ct.cast(pb, ct.c_void_p), ct.cast(px, ct.c_void_p),
                                   ct.cast(reps, ct.c_void_p), _stream(stream))
    if code not in (0, 5):
        raise DieError(code, "gmres_solve_many")
    outs = [{"converged": bool(r.rel_res_solved <= tol), "cycles": r.cycles, "iters": r.iters,
             "n_apply": r.n_apply, "rel_res_solved": r.rel_res_solved, "rel_res_orig": r.rel_res_orig,
             "t_total": r.t_total, "n_reorth": r.n_reorth, "graph_cycles": r.graph_cycles} for r in reps]
    return xs, outs


def gemm_bf16(A, B, C=None, alpha: float = 1.0, beta: float = 0.0, stream=None):
    """C = alpha A B^T + beta C on the tensor cores (BF16 operands, FP32 accumulation), for
    float32 CUDA tensors A (M x K) and B (N x K) of any strides (or batched, 3-D)."""
    import torch
    if A.dtype != torch.float32 or B.dtype != torch.float32 or not A.is_cuda or not B.is_cuda:
        raise TypeError("gemm_bf16 takes float32 CUDA tensors")
    batched = A.dim() == 3
    A3 = A if batched else A.unsqueeze(0)
    B3 = B if batched else B.unsqueeze(0)
    bt, M, K = A3.shape
    N = B3.shape[1]
    if B3.shape[2] != K or B3.shape[0] != bt:
        raise ValueError("shapes do not match")
    if C is None:
        C = torch.zeros((bt, M, N) if batched else (M, N), dtype=torch.float32, device=A.device)
    C3 = C if batched else C.unsqueeze(0)
    sa, sb, sc = A3.stride(), B3.stride(), C3.stride()
    _check(_lib().die_gemm_bf16(M, N, K, bt, float(alpha), ct.c_void_p(A3.data_ptr()), sa[1], sa[2], sa[0],
                                ct.c_void_p(B3.data_ptr()), sb[1], sb[2], sb[0], float(beta),
                                ct.c_void_p(C3.data_ptr()), sc[1], sc[2], sc[0], 1, _stream(stream)), "die_gemm_bf16")
    return C


class FNO:
    """Fourier neural operator on the tensor cores (an fno_t handle); see include/die_fno.h."""

    def __init__(self, c_in=6, c_out=4, width=32, modes=16, layers=4, hidden=128, H=128, W=128, max_batch=16):
        self.desc = FnoDesc(c_in, c_out, width, modes, layers, hidden, H, W, max_batch)
        h = ct.c_void_p()
        _check(_lib().fno_create(ct.byref(self.desc), ct.byref(h)), "fno_create")
        self._h = h
        self.n_params = int(_lib().fno_param_count(self._h))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib().fno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        import numpy as np
        a = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {a.size}")
        _check(_lib().fno_set_params(self._h, a.ctypes.data_as(ct.c_void_p)), "fno_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(self.n_params, dtype=np.float32)
        _check(_lib().fno_get_params(self._h, a.ctypes.data_as(ct.c_void_p)), "fno_get_params")
        return a

    def get_grads(self):
        import numpy as np
        a = np.empty(self.n_params, dtype=np.float32)
        _check(_lib().fno_get_grads(self._h, a.ctypes.data_as(ct.c_void_p)), "fno_get_grads")
        return a

    def zero_grads(self, stream=None):
        _check(_lib().fno_zero_grads(self._h, _stream(stream)), "fno_zero_grads")

    def forward(self, x, y=None, stream=None):
        import torch
        d = self.desc
        if x.dtype != torch.float32 or x.dim() != 4 or tuple(x.shape[1:]) != (d.c_in, d.H, d.W):
            raise ValueError("x must be float32 (batch, c_in, H, W)")
        y = torch.empty((x.shape[0], d.c_out, d.H, d.W), dtype=torch.float32, device=x.device) if y is None else y
        _check(_lib().fno_forward(self._h, x.shape[0], _ptr(x), _ptr(y), _stream(stream)), "fno_forward")
        return y

    def backward(self, gy, want_gx: bool = False, stream=None):
        import torch
        d = self.desc
        gx = torch.empty((gy.shape[0], d.c_in, d.H, d.W), dtype=torch.float32, device=gy.device) if want_gx else None
        _check(_lib().fno_backward(self._h, gy.shape[0], _ptr(gy), _ptr(gx) if gx is not None else None,
                                   _stream(stream)), "fno_backward")
        return gx

    def train_step(self, x, t, lr: float, stream=None) -> float:
        loss = ct.c_float()
        _check(_lib().fno_train_step(self._h, x.shape[0], _ptr(x), _ptr(t), float(lr), ct.byref(loss),
                                     _stream(stream)), "fno_train_step")
        return float(loss.value)

    def precondition(self, op: "Operator", v, z=None, stream=None):
        import torch
        z = torch.empty_like(v) if z is None else z
        _check(_lib().fno_precondition(self._h, op.handle, _ptr(v), _ptr(z), _stream(stream)), "fno_precondition")
        return z


def encode_pair(op: "Operator", b, u=None, x=None, t=None, stream=None):
    """Network input x (float32, 6 x n2 x n1) of the right-hand side b and, when u is given,
    the target t (4 x n2 x n1) of the solution u (fno_encode_pair)."""
    import torch
    x = torch.empty((6, op.n2, op.n1), dtype=torch.float32, device="cuda") if x is None else x
    if u is not None and t is None:
        t = torch.empty((4, op.n2, op.n1), dtype=torch.float32, device="cuda")
    _check(_lib().fno_encode_pair(op.handle, _ptr(b), _ptr(u) if u is not None else None, _ptr(x),
                                  _ptr(t) if u is not None else None, _stream(stream)), "fno_encode_pair")
    return x, t


def fgmres(op: "Operator", b, net: "FNO | None" = None, deflation: "Deflation | None" = None, x=None,
           restart: int = 30, tol: float = 1e-6, max_iters: int = 300, fallback_restart: int = 30,
           fallback_iters: int = 0, reorth_eta: float = 0.0, stream=None):
    """Flexible GMRES with the network as initial guess and right preconditioner (fgmres_solve);
    returns (x, report dict)."""
    import torch
    if b.dtype != torch.complex128:
        raise TypeError("fgmres takes complex128 vectors")
    use_x0 = x is not None
    x = torch.empty_like(b) if x is None else x
    opts = GmresOpts(restart, max_iters, tol, 0, int(use_x0), DIE_FP64, 0, float(reorth_eta), 0)
    rep = GmresReport()
    used = ct.c_int(0)
    code = _lib().fgmres_solve(op.handle, net.handle if net is not None else None,
                               deflation.handle if deflation is not None else None, ct.byref(opts),
                               fallback_restart, fallback_iters, _ptr(b), _ptr(x), ct.byref(rep), ct.byref(used),
                               _stream(stream))
    if code not in (0, 5):
        raise DieError(code, "fgmres_solve")
    return x, {"status": STATUS[code], "converged": code == 0, "cycles": rep.cycles, "iters": rep.iters,
               "rel_res_orig": rep.rel_res_orig, "used_fallback": bool(used.value)}
