"""Python binding of the B300 QR-CTMRG library (libqrctm.so).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libqrctm.so``.  PyTorch supplies device memory (the workspace and
the caller's tensors) and the CUDA stream.  If the shared library is missing
the first call into it raises; there is no CPU fallback.

The functions mirror the C ABI in ``include/qrctm.h``:

    ctx = QRCTM(d=2, D=6, chi=144, precision="split")
    ctx.init_env(A)                      # A: cuda float64, C4v symmetric
    iters, delta = ctx.run_to_convergence(tol=1e-10, max_iter=500)
    E = ctx.energy(J1=1.0, J2=0.0)
"""
from __future__ import annotations

import ctypes
import os

__all__ = ["QRCTM", "QRCTMError", "Energy", "lib", "c4v_symmetrize", "householder_qr",
           "gemm_tf32x3", "gemm_tf32x3_presplit", "tf32_split", "LIB_PATH"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libqrctm.so")


STATUS = {
    0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "NOT_CONVERGED", 4: "NUMERIC",
    5: "NOT_SYMMETRIC", 6: "WORKSPACE", 7: "TIMEOUT", 8: "STATE",
}
PRECISION = {"fp64": 0, "split": 1}
LAYERS = {"auto": 0, "double": 1, "split": 2, "network": 3}
GRAD_MODE = {"implicit": 0, "unroll": 1}
METHOD = {"qr": 0, "eigen": 1}
PHASES = ["ct", "qr", "x1", "absorb", "project", "corner", "symnorm", "spectrum", "energy",
          "grad", "warmup", "qr_panel"]


class QRCTMError(RuntimeError):
    def __init__(self, code, where, msg=""):
        self.code = code
        self.status = STATUS.get(code, str(code))
        super().__init__(f"{where}: {self.status}" + (f" ({msg})" if msg else ""))


class Config(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("D", ctypes.c_int), ("chi", ctypes.c_int),
        ("precision", ctypes.c_int), ("layers", ctypes.c_int),
        ("warmup_steps", ctypes.c_int), ("check_every", ctypes.c_int),
        ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
        ("grad_max_iter", ctypes.c_int), ("grad_tol", ctypes.c_double),
        ("with_nnn", ctypes.c_int), ("with_grad", ctypes.c_int),
        ("stream", ctypes.c_void_p), ("method", ctypes.c_int),
        ("opt_history", ctypes.c_int), ("grad_store", ctypes.c_int),
    ]


class Model(ctypes.Structure):
    _fields_ = [("J1", ctypes.c_double), ("J2", ctypes.c_double),
                ("sublattice_rotation", ctypes.c_int)]


class LbfgsOptions(ctypes.Structure):
    _fields_ = [
        ("history", ctypes.c_int), ("nograd_steps", ctypes.c_int), ("k_unroll", ctypes.c_int),
        ("max_ls", ctypes.c_int), ("c1", ctypes.c_double), ("step0", ctypes.c_double),
        ("env_tol", ctypes.c_double), ("env_max_iter", ctypes.c_int),
    ]


_vp, _dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_sig = {
    "qrctm_version": ([], ctypes.c_char_p),
    "qrctm_workspace_bytes": ([ctypes.POINTER(Config)], ctypes.c_size_t),
    "qrctm_create": ([ctypes.POINTER(Config), _vp, ctypes.c_size_t, ctypes.POINTER(_vp)],
                     ctypes.c_int),
    "qrctm_destroy": ([_vp], None),
    "qrctm_init_env": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "qrctm_step": ([_vp, ctypes.c_int, _dp], ctypes.c_int),
    "qrctm_run_to_convergence": ([_vp, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), _dp], ctypes.c_int),
    "qrctm_energy": ([_vp, ctypes.POINTER(Model), _dp], ctypes.c_int),
    "qrctm_energy_grad": ([_vp, ctypes.POINTER(Model), ctypes.c_int, ctypes.c_int, _vp, _dp],
                          ctypes.c_int),
    "qrctm_get_env": ([_vp, _vp, _vp, _dp], ctypes.c_int),
    "qrctm_init_env_host": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "qrctm_get_env_host": ([_vp, _vp, _vp, _dp], ctypes.c_int),
    "qrctm_init_env_network": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "qrctm_optimize": ([_vp, ctypes.POINTER(Model), ctypes.POINTER(LbfgsOptions), ctypes.c_int,
                        _vp, _dp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                       ctypes.c_int),
    "qrctm_network_observables": ([_vp, _vp, _dp, _dp], ctypes.c_int),
    "qrctm_iterations": ([_vp], ctypes.c_int),
    "qrctm_grad_iterations": ([_vp], ctypes.c_int),
    "qrctm_grad_residual": ([_vp], ctypes.c_double),
    "qrctm_grad_fixed_point_residual": ([_vp], ctypes.c_double),
    "qrctm_set_profiling": ([_vp, ctypes.c_int], ctypes.c_int),
    "qrctm_phase_times": ([_vp, _dp, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "qrctm_kernel_launches": ([], ctypes.c_ulonglong),
    "qrctm_last_error": ([_vp], ctypes.c_char_p),
    "qrctm_c4v_symmetrize": ([ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp,
                              ctypes.c_size_t, _vp], ctypes.c_int),
    "qrctm_c4v_symmetrize_workspace_bytes": ([], ctypes.c_size_t),
    "qrctm_qr_workspace_bytes": ([ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
    "qrctm_householder_qr": ([ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                              _vp], ctypes.c_int),
    "qrctm_gemm_tf32x3": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_longlong, _vp,
                           ctypes.c_longlong, _vp, ctypes.c_longlong, _vp, ctypes.c_longlong, _vp,
                           _vp], ctypes.c_int),
    "qrctm_householder_qr_bounded": ([ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                                      ctypes.c_size_t, _vp, ctypes.c_longlong, ctypes.c_int],
                                     ctypes.c_int),
    "qrctm_householder_qr_noalloc": ([ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp],
                                     ctypes.c_int),
    "qrctm_gemm_tf32x3_presplit": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                    ctypes.c_longlong, _vp, _vp, ctypes.c_longlong, _vp,
                                    ctypes.c_longlong, _vp, ctypes.c_longlong, _vp, _vp],
                                   ctypes.c_int),
    "qrctm_tf32_split": ([ctypes.c_longlong, ctypes.c_int, _vp, ctypes.c_longlong, _vp, _vp],
                         ctypes.c_int),
}
EXPORTED = sorted(_sig)
_LIB = None


def _load():
    """Load libqrctm.so once and bind its signatures; raise if it is missing."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2505_00494_b300.build` "
                "(nvcc, sm_103a). There is no CPU fallback.")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (args, ret) in _sig.items():
            f = getattr(handle, name)
            f.argtypes = args
            f.restype = ret
        _LIB = handle
    return _LIB


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("expected a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t):
    """Pointer of a contiguous host float64 tensor (None passes NULL)."""
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64:
        raise TypeError("expected a host (CPU) float64 tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _workspace(nbytes, device, zero=False):
    torch = _torch()
    alloc = torch.zeros if zero else torch.empty
    ws = alloc(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    if ws.data_ptr() % 256 != 0:
        raise RuntimeError("workspace not 256-byte aligned")
    return ws


class QRCTM:
    """A QR-CTMRG context over a torch-allocated device workspace."""

    def __init__(self, d, D, chi, precision="fp64", layers="auto", warmup_steps=0,
                 check_every=1, tol=1e-10, max_iter=500, grad_max_iter=0, grad_tol=0.0,
                 with_nnn=False, with_grad=False, stream=None, device="cuda", method="qr",
                 opt_history=0, grad_store="auto"):
        """grad_store: tapes of this many steps kept for unrolled gradients (an
        unrolled gradient of k <= grad_store steps records each step's tape on
        the way forward instead of re-running the step on the way back);
        "auto": up to 24 (the largest k of the paper's runs) within a quarter
        of the device memory still free after the rest of the workspace, 0
        without with_grad."""
        torch = _torch()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.cfg = Config(d, D, chi, PRECISION[precision], LAYERS[layers], warmup_steps,
                          check_every, tol, max_iter, grad_max_iter, grad_tol, int(with_nnn),
                          int(with_grad), ctypes.c_void_p(self.stream.cuda_stream),
                          METHOD[method], opt_history, 0)
        if with_grad and grad_store == "auto":
            base = _load().qrctm_workspace_bytes(ctypes.byref(self.cfg))
            self.cfg.grad_store = 1
            tape = _load().qrctm_workspace_bytes(ctypes.byref(self.cfg)) - base
            free = torch.cuda.mem_get_info(torch.device(device))[0] - base
            self.cfg.grad_store = int(max(0, min(24, (free // 4) // max(tape, 1)))) if base else 0
        elif grad_store != "auto":
            self.cfg.grad_store = int(grad_store)
        nbytes = _load().qrctm_workspace_bytes(ctypes.byref(self.cfg))
        if nbytes == 0:
            raise QRCTMError(1, "qrctm_workspace_bytes", "invalid configuration")
        self.workspace_bytes = nbytes
        self.ws = _workspace(nbytes, device)
        self.d, self.D, self.chi = d, D, chi
        # bond of T's inner leg: D^2 (ket and bra), or D for a network tensor
        self.D2 = D if layers == "network" else D * D
        h = ctypes.c_void_p()
        self.h = None
        self._check(_load().qrctm_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.ws.data_ptr()),
                                     nbytes, ctypes.byref(h)), "qrctm_create")
        self.h = h

    def _check(self, code, where):
        if code != 0:
            msg = _load().qrctm_last_error(self.h).decode() if self.h else ""
            raise QRCTMError(code, where, msg)

    def close(self):
        if getattr(self, "h", None):
            _load().qrctm_destroy(self.h)
            self.h = None
        if getattr(self, "ws", None) is not None:
            # the workspace (with a gradient's tape store, tens of GB) goes back
            # to torch once the context's queued work is done
            self.stream.synchronize()
            self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init_env(self, A, C0=None, T0=None):
        self.A = A
        self._check(_load().qrctm_init_env(self.h, _ptr(A), _ptr(C0), _ptr(T0)), "qrctm_init_env")

    def init_env_host(self, A, C0=None, T0=None):
        """qrctm_init_env from host float64 tensors (pinned for asynchronous
        copies); the copies run inside the library call."""
        self.A = None
        self._check(_load().qrctm_init_env_host(self.h, _hptr(A), _hptr(C0), _hptr(T0)),
                    "qrctm_init_env_host")

    def get_env_host(self, C, T, spectrum=False):
        """Copy (C, T) into host float64 tensors C (chi, chi), T (chi, D2, chi)
        inside the library call; optional sorted |eig C| as a NumPy array."""
        import numpy as np
        s = np.zeros(self.chi) if spectrum else None
        sp = s.ctypes.data_as(_dp) if spectrum else None
        self._check(_load().qrctm_get_env_host(self.h, _hptr(C), _hptr(T), sp),
                    "qrctm_get_env_host")
        return s

    def init_env_network(self, a, v=None, C0=None, T0=None):
        """Classical network tensor a[u,l,d,r] (bond D) fed directly; v: the
        boundary vector (None = all ones); (C0, T0): a starting environment
        used as it is instead of the boundary and warm-up."""
        self.A = a
        self._check(_load().qrctm_init_env_network(self.h, _ptr(a), _ptr(v), _ptr(C0), _ptr(T0)),
                    "qrctm_init_env_network")

    def network_observables(self, a_obs=None):
        """(ln kappa, <O>) at the current environment; <O> is None without a_obs."""
        lk = ctypes.c_double(0.0)
        ob = ctypes.c_double(0.0)
        self._check(_load().qrctm_network_observables(self.h, _ptr(a_obs), ctypes.byref(lk),
                                                      ctypes.byref(ob)),
                    "qrctm_network_observables")
        return lk.value, (ob.value if a_obs is not None else None)

    def step(self, n=1, want_delta=True):
        dlt = ctypes.c_double(0.0)
        self._check(_load().qrctm_step(self.h, n, ctypes.byref(dlt) if want_delta else None),
                    "qrctm_step")
        return dlt.value if want_delta else None

    def run_to_convergence(self, tol=0.0, max_iter=0, raise_on_max=False):
        it = ctypes.c_int(0)
        dlt = ctypes.c_double(0.0)
        code = _load().qrctm_run_to_convergence(self.h, tol, max_iter, ctypes.byref(it),
                                            ctypes.byref(dlt))
        if code == 3 and not raise_on_max:
            return it.value, dlt.value
        self._check(code, "qrctm_run_to_convergence")
        return it.value, dlt.value

    def energy(self, J1=1.0, J2=0.0, rotation=True):
        e = ctypes.c_double(0.0)
        m = Model(J1, J2, int(rotation))
        self._check(_load().qrctm_energy(self.h, ctypes.byref(m), ctypes.byref(e)), "qrctm_energy")
        return e.value

    def energy_grad(self, J1=1.0, J2=0.0, mode="implicit", k_unroll=20, grad=None, rotation=True):
        torch = _torch()
        if grad is None:
            grad = torch.empty((self.d,) + (self.D,) * 4, dtype=torch.float64, device="cuda")
        e = ctypes.c_double(0.0)
        m = Model(J1, J2, int(rotation))
        self._check(_load().qrctm_energy_grad(self.h, ctypes.byref(m), GRAD_MODE[mode], k_unroll,
                                          _ptr(grad), ctypes.byref(e)), "qrctm_energy_grad")
        return e.value, grad

    def optimize(self, A, n_steps, J1=1.0, J2=0.0, k_unroll=10, nograd_steps=2, history=0,
                 max_ls=0, c1=0.0, step0=0.0, env_tol=0.0, env_max_iter=0,
                 raise_on_line_search=False, rotation=True):
        """L-BFGS on the energy per site; A (device, C4v) is updated in place.
        Returns (energies of the accepted points, evaluations, line search
        failed)."""
        import numpy as np
        opt = LbfgsOptions(history, nograd_steps, k_unroll, max_ls, c1, step0, env_tol,
                           env_max_iter)
        en = np.zeros(n_steps + 1)
        steps, evals = ctypes.c_int(0), ctypes.c_int(0)
        m = Model(J1, J2, int(rotation))
        code = _load().qrctm_optimize(self.h, ctypes.byref(m), ctypes.byref(opt), n_steps, _ptr(A),
                                      en.ctypes.data_as(_dp), ctypes.byref(steps),
                                      ctypes.byref(evals))
        failed = code == 3
        if code != 0 and not (failed and not raise_on_line_search):
            self._check(code, "qrctm_optimize")
        self.A = A
        return en[:steps.value + 1], evals.value, failed

    def get_env(self, spectrum=True):
        torch = _torch()
        import numpy as np
        D2 = self.D2
        C = torch.empty((self.chi, self.chi), dtype=torch.float64, device="cuda")
        T = torch.empty((self.chi, D2, self.chi), dtype=torch.float64, device="cuda")
        s = np.zeros(self.chi) if spectrum else None
        sp = s.ctypes.data_as(_dp) if spectrum else None
        self._check(_load().qrctm_get_env(self.h, _ptr(C), _ptr(T), sp), "qrctm_get_env")
        return C, T, s

    def set_profiling(self, enable=True):
        self._check(_load().qrctm_set_profiling(self.h, int(enable)), "qrctm_set_profiling")

    def phase_times(self):
        """{phase: (milliseconds, occurrences)} since the previous call."""
        n = len(PHASES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        self._check(_load().qrctm_phase_times(self.h, ms, cnt), "qrctm_phase_times")
        return {PHASES[i]: (ms[i], cnt[i]) for i in range(n)}

    @property
    def grad_iterations(self):
        return _load().qrctm_grad_iterations(self.h)

    @property
    def grad_residual(self):
        return _load().qrctm_grad_residual(self.h)

    @property
    def grad_fixed_point_residual(self):
        """||G(x) - x|| / ||x|| of the environment at the last implicit gradient."""
        return _load().qrctm_grad_fixed_point_residual(self.h)

    @property
    def iterations(self):
        return _load().qrctm_iterations(self.h)


def kernel_launches():
    return _load().qrctm_kernel_launches()


def c4v_symmetrize(X, normalize=True, stream=None):
    """Y = sym(X) (optionally / ||.||_F) on the device."""
    torch = _torch()
    d, D = X.shape[0], X.shape[1]
    Y = torch.empty_like(X)
    nb = _load().qrctm_c4v_symmetrize_workspace_bytes()
    ws = _workspace(nb, X.device)
    code = _load().qrctm_c4v_symmetrize(d, D, _ptr(X), _ptr(Y), int(normalize),
                                    ctypes.c_void_p(ws.data_ptr()), nb, _stream_ptr(stream))
    if code != 0:
        raise QRCTMError(code, "qrctm_c4v_symmetrize")
    return Y


def gemm_tf32x3(A, B, stream=None, split_k=True):
    """C = A @ B.T (C FP64) from FP32 CUDA matrices A (M x K), B (N x K) on the
    tensor cores in split TF32x3 precision (K chunks summed in FP64 when
    split_k)."""
    torch = _torch()
    M, K = A.shape
    N = B.shape[0]
    if A.dtype != torch.float32 or B.dtype != torch.float32:
        raise TypeError("A and B must be float32")
    C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    nwork = (1 << 22) if split_k else 0
    work = torch.empty(max(nwork, 1), dtype=torch.float32, device=A.device)
    code = _load().qrctm_gemm_tf32x3(M, N, K, ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                     ctypes.c_void_p(B.data_ptr()), B.stride(0),
                                     ctypes.c_void_p(C.data_ptr()), N,
                                     ctypes.c_void_p(work.data_ptr()) if nwork else None, nwork,
                                     ctypes.c_void_p(err.data_ptr()), _stream_ptr(stream))
    if code != 0:
        raise QRCTMError(code, "qrctm_gemm_tf32x3")
    return C


def tf32_split(X, stream=None):
    """Split an FP32 CUDA matrix in place for the TF32x3 product: X becomes
    its TF32 heads; returns the tail plane (same shape)."""
    torch = _torch()
    if X.dtype != torch.float32 or X.dim() != 2 or X.stride(1) != 1:
        raise TypeError("X must be a row-contiguous float32 matrix")
    lo = torch.empty_like(X)
    code = _load().qrctm_tf32_split(X.shape[0], X.shape[1], ctypes.c_void_p(X.data_ptr()),
                                    X.stride(0), ctypes.c_void_p(lo.data_ptr()),
                                    _stream_ptr(stream))
    if code != 0:
        raise QRCTMError(code, "qrctm_tf32_split")
    return lo


def gemm_tf32x3_presplit(A, A_lo, B, B_lo, stream=None, split_k=True):
    """gemm_tf32x3 on pre-split operands (head planes A, B and tail planes
    A_lo, B_lo from tf32_split; A_lo may be None for a plain FP32 A)."""
    torch = _torch()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    nwork = (1 << 22) if split_k else 0
    work = torch.empty(max(nwork, 1), dtype=torch.float32, device=A.device)
    vp = ctypes.c_void_p
    code = _load().qrctm_gemm_tf32x3_presplit(
        M, N, K, vp(A.data_ptr()), vp(A_lo.data_ptr()) if A_lo is not None else None,
        A.stride(0), vp(B.data_ptr()), vp(B_lo.data_ptr()), B.stride(0), vp(C.data_ptr()), N,
        vp(work.data_ptr()) if nwork else None, nwork, vp(err.data_ptr()), _stream_ptr(stream))
    if code != 0:
        raise QRCTMError(code, "qrctm_gemm_tf32x3_presplit")
    return C


def householder_qr(M, stream=None, workspace=None, wait_spins=None, extra_arrivals=0):
    """Q, R of an m x n float64 CUDA matrix M (a row-major torch tensor).

    The library works on column-major storage, so M is passed as the storage
    of M^T; Q comes back the same way and is returned as an (m, n) view.
    ``wait_spins`` / ``extra_arrivals`` go to qrctm_householder_qr_bounded
    (the bound of the panel's device waits; extra arrivals make every wait
    run out, for testing the timeout path)."""
    torch = _torch()
    m, n = M.shape
    Mcm = M.t().contiguous()
    Qcm = torch.empty((n, m), dtype=torch.float64, device=M.device)
    R = torch.empty((n, n), dtype=torch.float64, device=M.device)
    nb = _load().qrctm_qr_workspace_bytes(m, n)
    ws = workspace if workspace is not None else _workspace(nb, M.device, zero=True)
    if wait_spins is None and not extra_arrivals:
        code = _load().qrctm_householder_qr(m, n, _ptr(Mcm), _ptr(Qcm), _ptr(R),
                                            ctypes.c_void_p(ws.data_ptr()), nb,
                                            _stream_ptr(stream))
    else:
        code = _load().qrctm_householder_qr_bounded(m, n, _ptr(Mcm), _ptr(Qcm), _ptr(R),
                                                    ctypes.c_void_p(ws.data_ptr()), nb,
                                                    _stream_ptr(stream), int(wait_spins or 0),
                                                    int(extra_arrivals))
    if code != 0:
        raise QRCTMError(code, "qrctm_householder_qr")
    return Qcm.t(), R


def _energy_function():
    torch = _torch()

    class Energy(torch.autograd.Function):
        """E(A): energy per site at the converged QR-CTMRG environment of A,
        differentiable through the library's hand-written adjoint.

            E = Energy.apply(A, ctx, J1, J2, tol, max_iter, mode, k_unroll)
            E.backward()            # A.grad = dE/dA (C4v-projected)

        ``ctx`` is a QRCTM context built with with_grad=True (and with_nnn=True
        when J2 != 0).  Forward builds the environment from the bulk boundary
        (qrctm_init_env), iterates to the spectrum tolerance and evaluates the
        energy; the converged (C, T) are kept with the autograd node, so the
        backward pass (qrctm_energy_grad, implicit fixed point or k unrolled
        steps) does not depend on later use of the context."""

        @staticmethod
        def forward(fctx, A, ctx, J1=1.0, J2=0.0, tol=1e-10, max_iter=500, mode="implicit",
                    k_unroll=20):
            A = A.detach().contiguous()
            ctx.init_env(A)
            ctx.run_to_convergence(tol=tol, max_iter=max_iter)
            E = ctx.energy(J1, J2)
            C, T, _ = ctx.get_env(spectrum=False)
            fctx.save_for_backward(A, C, T)
            fctx.args = (ctx, J1, J2, mode, k_unroll)
            return torch.tensor(E, dtype=torch.float64, device=A.device)

        @staticmethod
        def backward(fctx, gE):
            A, C, T = fctx.saved_tensors
            ctx, J1, J2, mode, k_unroll = fctx.args
            ctx.init_env(A, C, T)
            _, g = ctx.energy_grad(J1, J2, mode=mode, k_unroll=k_unroll)
            return (gE * g,) + (None,) * 7

    return Energy


def __getattr__(name):
    """Lazy attributes: ``lib`` (the loaded library) and ``Energy`` (the
    autograd function, built on first use so that importing the package does
    not import torch)."""
    if name == "lib":
        return _load()
    if name == "Energy":
        fn = _energy_function()
        globals()["Energy"] = fn
        return fn
    raise AttributeError(name)
