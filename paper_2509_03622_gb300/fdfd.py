"""Thin ctypes binding of libfdfd.so (include/fdfd.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (complex64 fields,
float32 permittivity); the binding passes their data pointers.  Importing
this module raises if the library has not been built -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfdfd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")

lib = C.CDLL(LIB_PATH)

OK, NOT_CONVERGED, STAGNATED = 0, 1, 2
EINVAL, ECUDA, ENUMERIC, ETIMEOUT, ENOSETUP, ENOMEM = -1, -2, -3, -4, -5, -6
PRECOND_NONE, PRECOND_JACOBI, PRECOND_SCHWARZ = 0, 1, 2
PREC_BF16, PREC_FP8 = 0, 1


class Desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("wavelength", C.c_double),
                ("npml", C.c_int * 4), ("pml_m", C.c_double), ("pml_lnR", C.c_double),
                ("eps", C.c_void_p), ("stream", C.c_void_p), ("max_restart", C.c_int)]


class SchwarzDesc(C.Structure):
    _fields_ = [("k_coarse", C.c_int), ("precision", C.c_int), ("weights", C.c_void_p),
                ("n_weights", C.c_size_t), ("inner_iters", C.c_int), ("ritz_tol", C.c_double),
                ("r_rank", C.c_int), ("modulation", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("restart", C.c_int), ("max_iters", C.c_int), ("tol", C.c_double),
                ("precond", C.c_int), ("use_x0", C.c_int), ("use_graphs", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("relres_true", C.c_double), ("relres_est", C.c_double), ("t_solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(C.Structure):
    _fields_ = [("n_win", C.c_int), ("nwx", C.c_int), ("nwy", C.c_int), ("k_coarse", C.c_int),
                ("n_coarse", C.c_int), ("workspace_bytes", C.c_size_t), ("graphs_cached", C.c_int),
                ("graphs_ok", C.c_int), ("tuned_dfty_split", C.c_int), ("n_coarse_kept", C.c_int)]


class DesignDesc(C.Structure):
    _fields_ = [("x0", C.c_int), ("y0", C.c_int), ("w", C.c_int), ("h", C.c_int), ("radius", C.c_float),
                ("beta", C.c_float), ("eta", C.c_float), ("eps_lo", C.c_float), ("eps_hi", C.c_float)]


class AdamDesc(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 18), ("launches", C.c_longlong * 18), ("total_launches", C.c_longlong)]


PROF_CLASSES = ["stencil", "cgs_dots", "cgs_update", "residual64", "vector_misc", "nno_pack", "traces", "coarse",
                "nno_lift", "nno_dft_x", "nno_dft_y", "nno_mix", "nno_idft_y", "nno_idft_x_mix_act", "nno_proj",
                "local_krylov", "rhs_norm", "unused"]

_P = C.c_void_p
_SIGS = {
    "fdfd_create": ([C.POINTER(Desc), C.POINTER(_P)], C.c_int),
    "fdfd_set_eps": ([_P, _P], C.c_int),
    "schwarz_setup": ([_P, C.POINTER(SchwarzDesc)], C.c_int),
    "fdfd_destroy": ([_P], None),
    "fdfd_status_string": ([C.c_int], C.c_char_p),
    "fdfd_get_info": ([_P, C.POINTER(Info)], C.c_int),
    "fdfd_solve": ([_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveStats)], C.c_int),
    "fdfd_solve_host": ([_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveStats)], C.c_int),
    "fdfd_solve_adjoint": ([_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveStats)], C.c_int),
    "fdfd_grad_eps": ([_P, _P, _P, _P, C.c_int], C.c_int),
    "fdfd_apply_A": ([_P, _P, _P, C.c_int], C.c_int),
    "fdfd_precond_apply": ([_P, _P, _P], C.c_int),
    "fdfd_schwarz_stationary": ([_P, _P, _P, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_int),
                                 C.POINTER(C.c_double)], C.c_int),
    "fdfd_nno_solve": ([_P, _P, _P, _P, C.c_int, _P], C.c_int),
    "fdfd_trace_extract": ([_P, _P, _P], C.c_int),
    "fdfd_local_apply": ([_P, _P, _P, _P, C.c_int], C.c_int),
    "fdfd_batch_create": ([C.POINTER(_P), C.c_int, C.c_int, C.POINTER(_P)], C.c_int),
    "fdfd_solve_batched": ([_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(SolveOpts), C.POINTER(SolveStats)], C.c_int),
    "fdfd_batch_destroy": ([_P], None),
    "fdfd_nno_solve_noalloc": ([_P, _P, _P, _P, C.c_int, _P], C.c_int),
    "fdfd_coarse_export": ([_P, _P, _P], C.c_int),
    "fdfd_coarse_solve": ([_P, _P, _P], C.c_int),
    "fdfd_coarse_ritz": ([_P, _P, _P], C.c_int),
    "fdfd_design_eps": ([_P, C.POINTER(DesignDesc), _P, _P, _P], C.c_int),
    "fdfd_design_grad": ([_P, C.POINTER(DesignDesc), _P, _P, _P, _P], C.c_int),
    "fdfd_adam_step": ([_P, C.POINTER(AdamDesc), C.c_int, C.c_float, _P, _P, _P, _P, C.c_int], C.c_int),
    "fdfd_mode_overlap": ([_P, C.c_int, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.c_double, _P, _P], C.c_int),
    "fdfd_mode_overlap_grad": ([C.c_int, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                _P, C.c_int, _P], C.c_int),
    "fdfd_adjoint_rhs": ([_P, _P, _P], C.c_int),
    "fdfd_profile_start": ([_P], C.c_int),
    "fdfd_selftest_gemm": ([_P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
    "fdfd_selftest_wait": ([], C.c_int),
    "fdfd_nno_mark_failed": ([_P], C.c_int),
    "fdfd_profile_stop": ([_P, C.POINTER(Profile)], C.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class FDFDError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {lib.fdfd_status_string(code).decode()} ({code})")
        self.code = code


def _check(code, where):
    if code < 0:
        raise FDFDError(code, where)
    return code


def _ptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def status_string(code: int) -> str:
    return lib.fdfd_status_string(code).decode()


def mode_overlap(E, mode, port_x: int, y0: int, dx: float, c, stream=None):
    """c (float64 CUDA tensor [2], re / im) = dx sum conj(mode) E along the
    vertical line x = port_x from row y0 (fdfd_mode_overlap), on `stream`
    (default: PyTorch's current stream)."""
    import torch
    if c.dtype != torch.float64 or c.numel() < 2:
        raise TypeError("c must be a float64 tensor of 2 elements")
    if E.dtype != torch.complex64 or mode.dtype != torch.complex64 or E.dim() != 2:
        raise TypeError("E must be a 2-D complex64 field and mode a complex64 profile")
    st = stream if stream is not None else torch.cuda.current_stream(E.device).cuda_stream
    ny, nx = E.shape
    _check(lib.fdfd_mode_overlap(_ptr(E), nx, ny, _ptr(mode), mode.numel(), int(port_x), int(y0), float(dx),
                                 _ptr(c), C.c_void_p(st)), "fdfd_mode_overlap")


def mode_overlap_grad(shape, mode, port_x: int, y0: int, dx: float, gc: complex, grad_E, accumulate=False,
                      stream=None):
    """grad_E (=|+=) gc * mode * dx on the port line (fdfd_mode_overlap_grad)."""
    import torch
    if grad_E.dtype != torch.complex64 or mode.dtype != torch.complex64 or tuple(grad_E.shape) != tuple(shape):
        raise TypeError("grad_E must be a complex64 field of the given shape and mode a complex64 profile")
    st = stream if stream is not None else torch.cuda.current_stream(grad_E.device).cuda_stream
    ny, nx = shape
    _check(lib.fdfd_mode_overlap_grad(nx, ny, _ptr(mode), mode.numel(), int(port_x), int(y0), float(dx),
                                      float(gc.real), float(gc.imag), _ptr(grad_E), int(accumulate),
                                      C.c_void_p(st)), "fdfd_mode_overlap_grad")


def selftest_wait() -> int:
    """Bounded-wait diagnostic: the raw status (FDFD_ETIMEOUT expected)."""
    return lib.fdfd_selftest_wait()


def selftest_gemm(A, B, C_out, a_mn_major=False):
    """tcgen05 GEMM diagnostic: C_out = A @ B^T (A [M][K] or [K][M] bf16, B [N][K] bf16)."""
    M = A.shape[1] if a_mn_major else A.shape[0]
    K = A.shape[0] if a_mn_major else A.shape[1]
    _check(lib.fdfd_selftest_gemm(_ptr(A), _ptr(B), _ptr(C_out), M, B.shape[0], K, int(a_mn_major)),
           "fdfd_selftest_gemm")


class Solver:
    """Owns one fdfd_handle (fdfd_create ... fdfd_destroy)."""

    def __init__(self, eps, dx: float, wavelength: float, npml=20, pml_m: float = 3.0,
                 pml_lnR: float = -30.0, stream=None, max_restart: int = 0):
        import torch
        if eps.dtype != torch.float32 or eps.dim() != 2:
            raise TypeError("eps must be a 2D float32 CUDA tensor")
        ny, nx = eps.shape
        d = Desc()
        d.nx, d.ny, d.dx, d.wavelength = nx, ny, dx, wavelength
        np_ = (npml,) * 4 if np.isscalar(npml) else tuple(npml)
        d.npml = (C.c_int * 4)(*np_)
        d.pml_m, d.pml_lnR = pml_m, pml_lnR
        d.max_restart = int(max_restart)
        d.eps = _ptr(eps).value
        s = stream if stream is not None else torch.cuda.current_stream()
        d.stream = C.c_void_p(s.cuda_stream).value
        self.stream = s
        h = C.c_void_p()
        _check(lib.fdfd_create(C.byref(d), C.byref(h)), "fdfd_create")
        self.h = h
        self.nx, self.ny = nx, ny
        self.dx, self.wavelength = dx, wavelength

    def close(self):
        if getattr(self, "h", None):
            lib.fdfd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = Info()
        _check(lib.fdfd_get_info(self.h, C.byref(i)), "fdfd_get_info")
        return {k: getattr(i, k) for k, _ in i._fields_}

    def set_eps(self, eps):
        _check(lib.fdfd_set_eps(self.h, _ptr(eps)), "fdfd_set_eps")

    def schwarz_setup(self, weights_blob: np.ndarray, k_coarse: int = 0, precision: int = PREC_BF16,
                      inner_iters: int = 0, ritz_tol: float = 0.0, rank: int = 0, modulation: bool = False):
        """rank, modulation: the layout of the blob (modified FNO; see
        workloads.weight_order)."""
        blob = np.ascontiguousarray(weights_blob, dtype=np.float32)
        sd = SchwarzDesc()
        sd.k_coarse, sd.precision, sd.inner_iters, sd.ritz_tol = k_coarse, precision, inner_iters, float(ritz_tol)
        sd.r_rank, sd.modulation = int(rank), int(bool(modulation))
        sd.weights = blob.ctypes.data
        sd.n_weights = blob.size
        _check(lib.schwarz_setup(self.h, C.byref(sd)), "schwarz_setup")

    # replay each Arnoldi step as a CUDA graph (set False for eager launches)
    use_graphs = True

    def _opts(self, restart, max_iters, tol, precond, use_x0):
        o = SolveOpts()
        o.restart, o.max_iters, o.tol, o.precond, o.use_x0 = restart, max_iters, tol, precond, int(use_x0)
        o.use_graphs = int(self.use_graphs)
        return o

    def solve(self, J, E, restart=30, max_iters=1000, tol=1e-6, precond=PRECOND_SCHWARZ, use_x0=False):
        st = SolveStats()
        o = self._opts(restart, max_iters, tol, precond, use_x0)
        rc = _check(lib.fdfd_solve(self.h, _ptr(J), _ptr(E), C.byref(o), C.byref(st)), "fdfd_solve")
        return rc, st.as_dict()

    def solve_host(self, J: np.ndarray, E: np.ndarray, restart=30, max_iters=1000, tol=1e-6,
                   precond=PRECOND_SCHWARZ, use_x0=False):
        assert J.dtype == np.complex64 and E.dtype == np.complex64 and J.flags.c_contiguous
        st = SolveStats()
        o = self._opts(restart, max_iters, tol, precond, use_x0)
        rc = _check(lib.fdfd_solve_host(self.h, J.ctypes.data, E.ctypes.data, C.byref(o), C.byref(st)),
                    "fdfd_solve_host")
        return rc, st.as_dict()

    def solve_adjoint(self, g, lam, restart=30, max_iters=1000, tol=1e-6, precond=PRECOND_SCHWARZ,
                      use_x0=False):
        st = SolveStats()
        o = self._opts(restart, max_iters, tol, precond, use_x0)
        rc = _check(lib.fdfd_solve_adjoint(self.h, _ptr(g), _ptr(lam), C.byref(o), C.byref(st)),
                    "fdfd_solve_adjoint")
        return rc, st.as_dict()

    def adjoint_rhs(self, grad_E, g):
        """g = conj(grad_E) / 2: the adjoint right-hand side dL/dE from
        autograd's field gradient (fdfd_adjoint_rhs)."""
        import torch
        if grad_E.dtype != torch.complex64 or g.dtype != torch.complex64:
            raise TypeError("grad_E and g must be complex64")
        if grad_E.numel() != self.nx * self.ny or g.numel() != self.nx * self.ny:
            raise ValueError("grad_E and g must cover the handle's grid")
        _check(lib.fdfd_adjoint_rhs(self.h, _ptr(grad_E), _ptr(g)), "fdfd_adjoint_rhs")

    def grad_eps(self, E, lam, grad, accumulate=False):
        _check(lib.fdfd_grad_eps(self.h, _ptr(E), _ptr(lam), _ptr(grad), int(accumulate)), "fdfd_grad_eps")

    def apply_A(self, x, y, transpose=False):
        _check(lib.fdfd_apply_A(self.h, _ptr(x), _ptr(y), int(transpose)), "fdfd_apply_A")

    def precond_apply(self, v, z):
        _check(lib.fdfd_precond_apply(self.h, _ptr(v), _ptr(z)), "fdfd_precond_apply")

    def schwarz_stationary(self, b, u, max_iters=200, tol=1e-6, momentum=0.0):
        """Algorithm 3: the stationary Schwarz iteration for A~ u = b.
        Returns (iterations, relative residual)."""
        it, rr = C.c_int(0), C.c_double(0.0)
        _check(lib.fdfd_schwarz_stationary(self.h, _ptr(b), _ptr(u), int(max_iters), float(tol), float(momentum),
                                           C.byref(it), C.byref(rr)), "fdfd_schwarz_stationary")
        return it.value, rr.value

    def nno_solve(self, r_win, g_win, win_id, e_win):
        n = r_win.shape[0]
        _check(lib.fdfd_nno_solve(self.h, _ptr(r_win), _ptr(g_win), _ptr(win_id), n, _ptr(e_win)),
               "fdfd_nno_solve")

    def nno_solve_noalloc(self, r_win, g_win, win_id, e_win):
        """fdfd_nno_solve without any device allocation (at most 4 windows)."""
        n = r_win.shape[0]
        _check(lib.fdfd_nno_solve_noalloc(self.h, _ptr(r_win), _ptr(g_win), _ptr(win_id), n, _ptr(e_win)),
               "fdfd_nno_solve_noalloc")

    def local_apply(self, x_win, y_win, win_id):
        _check(lib.fdfd_local_apply(self.h, _ptr(x_win), _ptr(y_win), _ptr(win_id), x_win.shape[0]),
               "fdfd_local_apply")

    def trace_extract(self, u, g):
        _check(lib.fdfd_trace_extract(self.h, _ptr(u), _ptr(g)), "fdfd_trace_extract")

    def nno_mark_failed(self):
        """Failure injection: mark the neural operator failed (as a timed-out device wait does)."""
        _check(lib.fdfd_nno_mark_failed(self.h), "fdfd_nno_mark_failed")

    def profile_start(self):
        _check(lib.fdfd_profile_start(self.h), "fdfd_profile_start")

    def profile_stop(self) -> dict:
        p = Profile()
        _check(lib.fdfd_profile_stop(self.h, C.byref(p)), "fdfd_profile_stop")
        return {"ms": {c: p.ms[i] for i, c in enumerate(PROF_CLASSES)},
                "launches": {c: p.launches[i] for i, c in enumerate(PROF_CLASSES)},
                "total_launches": p.total_launches}

    def coarse_export(self):
        inf = self.info()
        nw, k = inf["n_win"], inf["k_coarse"]
        Q = np.zeros((nw, k, 4, 80, 2), dtype=np.float64)
        G = np.zeros((nw, 9, k, k, 2), dtype=np.float64)
        _check(lib.fdfd_coarse_export(self.h, Q.ctypes.data, G.ctypes.data), "fdfd_coarse_export")
        return Q[..., 0] + 1j * Q[..., 1], G[..., 0] + 1j * G[..., 1]

    def coarse_solve(self, ebc, z):
        """z = G^-1 (-Q^H ebc) for device tensors ebc [n_win][4][80] and
        z [n_win][k] (complex64)."""
        _check(lib.fdfd_coarse_solve(self.h, _ptr(ebc), _ptr(z)), "fdfd_coarse_solve")


    def coarse_ritz(self):
        """(Ritz values [n_win][k], Ritz matrices [n_win][k][k]) of a set-up
        with ritz_tol > 0."""
        inf = self.info()
        nw, k = inf["n_win"], inf["k_coarse"]
        eta = np.zeros((nw, k, 2), dtype=np.float64)
        H = np.zeros((nw, k, k, 2), dtype=np.float64)
        _check(lib.fdfd_coarse_ritz(self.h, eta.ctypes.data, H.ctypes.data), "fdfd_coarse_ritz")
        return eta[..., 0] + 1j * eta[..., 1], H[..., 0] + 1j * H[..., 1]


class Batch:
    """Lock-step solves of several problems (fdfd_batch_create ... destroy)."""

    def __init__(self, solvers, max_windows: int = 0):
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        b = C.c_void_p()
        _check(lib.fdfd_batch_create(arr, len(self.solvers), max_windows, C.byref(b)), "fdfd_batch_create")
        self.b = b

    def close(self):
        if getattr(self, "b", None):
            lib.fdfd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, Js, Es, restart=30, max_iters=1000, tol=1e-6, precond=PRECOND_SCHWARZ, use_x0=False):
        n = len(self.solvers)
        jp = (C.c_void_p * n)(*[_ptr(J).value for J in Js])
        ep = (C.c_void_p * n)(*[_ptr(E).value for E in Es])
        st = (SolveStats * n)()
        o = self.solvers[0]._opts(restart, max_iters, tol, precond, use_x0)
        rc = _check(lib.fdfd_solve_batched(self.b, jp, ep, C.byref(o), st), "fdfd_solve_batched")
        return rc, [s.as_dict() for s in st]
