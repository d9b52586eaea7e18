"""Thin Python binding of libpwa.so: the C ABI of include/pwa.h with the same names.

Only argument marshalling happens here (torch tensors -> device pointers, the current CUDA
stream -> void*); every step of the computation runs in the library's CUDA kernels.  There is
no fallback: if libpwa.so is missing or no GPU is visible the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpwa.so")

PWA_OK = 0
PWA_ERR_INVALID_ARG = -1
PWA_ERR_NO_DEVICE = -2
PWA_ERR_CUDA = -3
PWA_ERR_NONFINITE = -4
PWA_ERR_TIMEOUT = -5
PWA_ERR_WORKSPACE = -6
PWA_NOT_CONVERGED = 1


class PWAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


class pwa_wave(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int), ("lambda_", ctypes.c_int), ("mass", ctypes.c_double),
                ("width", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libpwa.so (built by paper_1108_5882_gb300.build).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"libpwa.so not built ({p}); run paper_1108_5882_gb300.build.build()")
        lib = ctypes.CDLL(p)
        S = ctypes.c_int
        lib.pwa_abi_version.restype = ctypes.c_int
        lib.pwa_status_string.argtypes = [ctypes.c_int]
        lib.pwa_status_string.restype = ctypes.c_char_p
        lib.pwa_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
        lib.pwa_create.restype = S
        lib.pwa_destroy.argtypes = [_vp]
        lib.pwa_destroy.restype = None
        lib.pwa_last_error.argtypes = [_vp]
        lib.pwa_last_error.restype = ctypes.c_char_p
        lib.pwa_workspace_size.argtypes = [_vp, ctypes.c_int, _i64, ctypes.c_int]
        lib.pwa_workspace_size.restype = ctypes.c_size_t
        lib.pwa_reserve.argtypes = [_vp, ctypes.c_int, _i64, ctypes.c_int]
        lib.pwa_reserve.restype = S
        lib.pwa_batched_shape.argtypes = [ctypes.c_int, _i64, ctypes.c_int]
        lib.pwa_batched_shape.restype = ctypes.c_int
        lib.pwa_sync_status.argtypes = [_vp, _vp]
        lib.pwa_sync_status.restype = S
        lib.pwa_amplitudes.argtypes = [_vp, ctypes.POINTER(pwa_wave), ctypes.c_int, _vp, _i64, _i64, _vp, _vp,
                                       _vp, _vp]
        lib.pwa_amplitudes.restype = S
        lib.pwa_amplitudes_barrier.argtypes = [_vp, ctypes.POINTER(pwa_wave), ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, _vp, _i64, _i64, _vp, _vp]
        lib.pwa_amplitudes_barrier.restype = S
        lib.pwa_normint.argtypes = [_vp, _vp, ctypes.c_int, _i64, _i64, _vp, ctypes.c_double, _vp, _vp]
        lib.pwa_normint.restype = S
        lib.pwa_normint_from_kinematics.argtypes = [_vp, ctypes.POINTER(pwa_wave), ctypes.c_int, _vp, _i64, _i64, _vp,
                                                    ctypes.c_double, _vp, _vp]
        lib.pwa_normint_from_kinematics.restype = S
        lib.pwa_nll.argtypes = [_vp, _vp, ctypes.c_int, _i64, _i64, _vp, ctypes.c_int, _vp, ctypes.c_double, _vp,
                                _vp]
        lib.pwa_nll.restype = S
        lib.pwa_nll_grad.argtypes = [_vp, _vp, ctypes.c_int, _i64, _i64, _vp, ctypes.c_int, _vp,
                                     ctypes.c_double, _vp, _vp, _vp]
        lib.pwa_nll_grad.restype = S
        lib.pwa_nll_grad_incoherent.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _i64, _i64, _vp, ctypes.c_int,
                                                _vp, ctypes.c_double, _vp, _vp, _vp]
        lib.pwa_nll_grad_incoherent.restype = S
        lib.pwa_hessian.argtypes = [_vp, _vp, ctypes.c_int, _i64, _i64, _vp, _vp, ctypes.c_double, ctypes.c_int, _vp,
                                    _vp]
        lib.pwa_hessian.restype = S
        _register_optional(lib)
        _lib = lib
        return lib


def _register_optional(lib):
    """Entry points added after the first ABI version (bound when present)."""
    S = ctypes.c_int
    lib.pwa_envelope.argtypes = [ctypes.POINTER(pwa_wave), ctypes.c_int, _vp, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int]
    lib.pwa_envelope.restype = ctypes.c_double
    lib.pwa_nll_grad_shape.argtypes = [_vp, _vp, _vp, ctypes.c_int, _i64, _i64, _vp, _vp, _i64, _i64, _vp,
                                       ctypes.c_double, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _vp,
                                       ctypes.c_double, _vp, _vp, _vp]
    lib.pwa_nll_grad_shape.restype = S
    lib.pwa_fit_shape_batch.argtypes = [_vp, ctypes.POINTER(pwa_shape_fit_desc), ctypes.c_int,
                                        ctypes.POINTER(pwa_fit_opts), ctypes.POINTER(pwa_fit_result), _vp]
    lib.pwa_fit_shape_batch.restype = S
    lib.pwa_nll_grad_uneven.argtypes = [_vp, ctypes.POINTER(pwa_uneven_channel), ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
    lib.pwa_nll_grad_uneven.restype = S
    lib.pwa_moments.argtypes = [_vp, _vp, _i64, _i64, ctypes.c_int, ctypes.c_double, ctypes.c_double, _vp, _vp]
    lib.pwa_moments.restype = S
    lib.pwa_toy_moments.argtypes = [_vp, ctypes.POINTER(pwa_wave), ctypes.c_int, _vp, ctypes.c_int, _vp,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, _vp, _vp, _vp]
    lib.pwa_toy_moments.restype = S
    lib.pwa_mlp_gemm.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _i64, _i64, _vp,
                                 ctypes.c_int, _i64, _i64, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _i64, _vp]
    lib.pwa_mlp_relu_backward.argtypes = [_vp, _vp, _vp, _i64, _vp]
    lib.pwa_mlp_bias_grad.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
    lib.pwa_mlp_wta_loss.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, _vp,
                                     _vp, _vp, _vp]
    lib.pwa_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_int, _vp]
    lib.pwa_mlp_to_bf16.argtypes = [_vp, _vp, _vp, _i64, ctypes.c_float, _vp]
    for f in ("pwa_mlp_gemm", "pwa_mlp_relu_backward", "pwa_mlp_bias_grad", "pwa_mlp_wta_loss", "pwa_mlp_adam",
              "pwa_mlp_to_bf16"):
        getattr(lib, f).restype = S
    lib.pwa_fit_default_opts.argtypes = [ctypes.POINTER(pwa_fit_opts)]
    lib.pwa_fit_default_opts.restype = None
    lib.pwa_fit_batch.argtypes = [_vp, ctypes.POINTER(pwa_fit_desc), ctypes.c_int, ctypes.POINTER(pwa_fit_opts),
                                  ctypes.POINTER(pwa_fit_result), _vp]
    lib.pwa_fit_batch.restype = S
    if hasattr(lib, "pwa_generate"):
        lib.pwa_generate.argtypes = [_vp, ctypes.POINTER(pwa_wave), ctypes.c_int, _vp, ctypes.c_uint64,
                                     ctypes.c_uint32, _i64, _i64, ctypes.c_double, _vp, _i64, _i64, _vp, _vp]
        lib.pwa_generate.restype = S


class pwa_fit_desc(ctypes.Structure):
    _fields_ = [("A", _vp), ("K", ctypes.c_int), ("n", _i64), ("ld", _i64), ("Psi", _vp), ("n_factor", ctypes.c_double),
                ("P", ctypes.c_int), ("V0", _vp), ("V_out", _vp)]


class pwa_fit_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("history", ctypes.c_int), ("gtol", ctypes.c_double),
                ("check_every", ctypes.c_int), ("gauge_fix", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("polar", ctypes.c_int)]


class pwa_fit_result(ctypes.Structure):
    _fields_ = [("nll", ctypes.c_double), ("grad_max", ctypes.c_double), ("iterations", ctypes.c_int),
                ("evaluations", ctypes.c_int), ("status", ctypes.c_int)]


class pwa_shape_fit_desc(ctypes.Structure):
    _fields_ = [("waves", ctypes.POINTER(pwa_wave)), ("K", ctypes.c_int), ("kin", _vp), ("n", _i64), ("ld", _i64),
                ("kin_mc", _vp), ("n_mc", _i64), ("ld_mc", _i64), ("w_mc", _vp), ("n_gen", ctypes.c_double),
                ("n_factor", ctypes.c_double), ("F", ctypes.c_int), ("float_wave", ctypes.POINTER(ctypes.c_int)),
                ("float_kind", ctypes.POINTER(ctypes.c_int)), ("A", _vp), ("A_mc", _vp), ("dA", _vp), ("dA_mc", _vp),
                ("V0", _vp), ("x_out", _vp)]


class pwa_uneven_channel(ctypes.Structure):
    _fields_ = [("waves", ctypes.POINTER(pwa_wave)), ("K", ctypes.c_int), ("kin", _vp), ("n", _i64), ("ld", _i64),
                ("kin_mc", _vp), ("n_mc", _i64), ("ld_mc", _i64), ("w_mc", _vp), ("n_gen", ctypes.c_double),
                ("n_factor", ctypes.c_double), ("F", ctypes.c_int), ("float_wave", ctypes.POINTER(ctypes.c_int)),
                ("float_kind", ctypes.POINTER(ctypes.c_int))]


def status_string(s: int) -> str:
    try:
        return load().pwa_status_string(int(s)).decode()
    except ImportError:
        return f"status {s}"


def _stream_ptr(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _check_cuda(t, name, dtype):
    if t is None:
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Handle:
    """Owns a pwa_handle (device workspace, status word) bound to one CUDA device."""

    def __init__(self, device: int | None = None):
        self.lib = load()
        if device is None:
            device = torch.cuda.current_device() if torch.cuda.is_available() else 0
        self.device = device
        h = ctypes.c_void_p()
        st = self.lib.pwa_create(ctypes.byref(h), int(device))
        if st != PWA_OK:
            raise PWAError(st, self.lib.pwa_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.pwa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != PWA_OK:
            raise PWAError(st, self.lib.pwa_last_error(self.h).decode())

    # ------------------------------------------------------------------ entry points
    def pwa_workspace_size(self, K, n, P):
        return int(self.lib.pwa_workspace_size(self.h, int(K), int(n), int(P)))

    def pwa_reserve(self, K, n, P):
        self._chk(self.lib.pwa_reserve(self.h, int(K), int(n), int(P)))

    def pwa_batched_shape(self, K, n, P):
        return int(self.lib.pwa_batched_shape(int(K), int(n), int(P)))

    def pwa_sync_status(self, stream=None):
        return int(self.lib.pwa_sync_status(self.h, _stream_ptr(stream)))

    def pwa_amplitudes(self, waves, kin, n, A, dA_dM=None, dA_dW=None, stream=None):
        """waves: list of (J, lambda, mass, width); kin float32 [3][ld]; A complex64 [K][ld]."""
        K = len(waves)
        arr = (pwa_wave * K)(*[pwa_wave(int(j), int(l), float(m), float(w)) for (j, l, m, w) in waves])
        _check_cuda(kin, "kin", torch.float32)
        _check_cuda(A, "A", torch.complex64)
        _check_cuda(dA_dM, "dA_dM", torch.complex64)
        _check_cuda(dA_dW, "dA_dW", torch.complex64)
        ld = A.shape[1]
        if kin.shape[1] != ld:
            raise ValueError("kin and A must share the leading dimension")
        self._chk(self.lib.pwa_amplitudes(self.h, arr, K, _ptr(kin), int(n), int(ld), _ptr(A), _ptr(dA_dM),
                                          _ptr(dA_dW), _stream_ptr(stream)))

    def pwa_amplitudes_barrier(self, waves, m1, m2, R, kin, n, A, stream=None):
        """As pwa_amplitudes with a mass-dependent width and Blatt-Weisskopf barrier factors
        (daughter masses m1, m2, L = J, radius R in GeV^-1)."""
        _check_cuda(kin, "kin", torch.float32)
        _check_cuda(A, "A", torch.complex64)
        ld = A.shape[1]
        if kin.shape[1] != ld:
            raise ValueError("kin and A must share the leading dimension")
        self._chk(self.lib.pwa_amplitudes_barrier(self.h, _wave_array(waves), len(waves), float(m1), float(m2),
                                                  float(R), _ptr(kin), int(n), int(ld), _ptr(A),
                                                  _stream_ptr(stream)))

    def pwa_normint(self, A_mc, n_mc, Psi, w=None, n_gen=None, stream=None):
        """A_mc complex64 [K][ld]; Psi complex128 [K][K] output; w float32 [n_mc] or None."""
        _check_cuda(A_mc, "A_mc", torch.complex64)
        _check_cuda(Psi, "Psi", torch.complex128)
        _check_cuda(w, "w", torch.float32)
        K, ld = A_mc.shape
        n_gen = float(n_mc if n_gen is None else n_gen)
        self._chk(self.lib.pwa_normint(self.h, _ptr(A_mc), K, int(n_mc), int(ld), _ptr(w), n_gen, _ptr(Psi),
                                       _stream_ptr(stream)))

    def pwa_normint_from_kinematics(self, waves, kin, n_mc, Psi, w=None, n_gen=None, stream=None):
        """Psi complex128 [K][K] from MC kinematics float32 [3][ld] (amplitudes computed on chip)."""
        K = len(waves)
        arr = (pwa_wave * K)(*[pwa_wave(int(j), int(l), float(m), float(wd)) for (j, l, m, wd) in waves])
        _check_cuda(kin, "kin", torch.float32)
        _check_cuda(Psi, "Psi", torch.complex128)
        _check_cuda(w, "w", torch.float32)
        ld = kin.shape[1]
        n_gen = float(n_mc if n_gen is None else n_gen)
        self._chk(self.lib.pwa_normint_from_kinematics(self.h, arr, K, _ptr(kin), int(n_mc), int(ld), _ptr(w), n_gen,
                                                       _ptr(Psi), _stream_ptr(stream)))

    def pwa_nll(self, A, n, V, Psi, n_factor, nll, stream=None):
        _check_cuda(A, "A", torch.complex64)
        _check_cuda(V, "V", torch.complex64)
        _check_cuda(Psi, "Psi", torch.complex128)
        _check_cuda(nll, "nll", torch.float64)
        K, ld = A.shape
        P = V.shape[0]
        self._chk(self.lib.pwa_nll(self.h, _ptr(A), K, int(n), int(ld), _ptr(V), P, _ptr(Psi), float(n_factor),
                                   _ptr(nll), _stream_ptr(stream)))

    def pwa_hessian(self, A, n, V, Psi, n_factor, H, exact=False, stream=None):
        """A complex64 [K][ld], V complex64 [K] (one set), Psi complex128 [K][K]; H float64 [2K][2K]."""
        _check_cuda(A, "A", torch.complex64)
        _check_cuda(V, "V", torch.complex64)
        _check_cuda(Psi, "Psi", torch.complex128)
        _check_cuda(H, "H", torch.float64)
        K, ld = A.shape
        self._chk(self.lib.pwa_hessian(self.h, _ptr(A), K, int(n), int(ld), _ptr(V), _ptr(Psi), float(n_factor),
                                       1 if exact else 0, _ptr(H), _stream_ptr(stream)))

    def pwa_nll_grad_incoherent(self, A, n, V, Psi, n_factor, nll, grad=None, stream=None):
        """A complex64 [K][H][ld] (intensity summed over the H states), V complex64 [P][K], Psi
        complex128 [K][K] (summed over the states); nll float64 [P], grad float64 [P][2K] or None."""
        _check_cuda(A, "A", torch.complex64)
        _check_cuda(V, "V", torch.complex64)
        _check_cuda(Psi, "Psi", torch.complex128)
        _check_cuda(nll, "nll", torch.float64)
        if grad is not None:
            _check_cuda(grad, "grad", torch.float64)
        K, H, ld = A.shape
        P = V.shape[0]
        self._chk(self.lib.pwa_nll_grad_incoherent(self.h, _ptr(A), K, H, int(n), int(ld), _ptr(V), P, _ptr(Psi),
                                                   float(n_factor), _ptr(nll),
                                                   _ptr(grad) if grad is not None else None, _stream_ptr(stream)))

    def pwa_nll_grad(self, A, n, V, Psi, n_factor, nll, grad, stream=None):
        """A complex64 [K][ld], V complex64 [P][K], Psi complex128 [K][K];
        nll float64 [P], grad float64 [P][2K] outputs."""
        _check_cuda(A, "A", torch.complex64)
        _check_cuda(V, "V", torch.complex64)
        _check_cuda(Psi, "Psi", torch.complex128)
        _check_cuda(nll, "nll", torch.float64)
        _check_cuda(grad, "grad", torch.float64)
        K, ld = A.shape
        P = V.shape[0]
        self._chk(self.lib.pwa_nll_grad(self.h, _ptr(A), K, int(n), int(ld), _ptr(V), P, _ptr(Psi),
                                        float(n_factor), _ptr(nll), _ptr(grad), _stream_ptr(stream)))


def _wave_array(waves):
    K = len(waves)
    return (pwa_wave * K)(*[pwa_wave(int(j), int(l), float(m), float(w)) for (j, l, m, w) in waves])


def pwa_envelope(waves, V, m_lo=0.99, m_hi=3.0, n_intervals=4096) -> float:
    """Host bound C >= max I over the phase space; V: complex64 array-like [K] on the host."""
    import numpy as np
    lib = load()
    Vh = np.ascontiguousarray(np.asarray(V, dtype=np.complex64)).view(np.float32)
    c = lib.pwa_envelope(_wave_array(waves), len(waves), Vh.ctypes.data_as(ctypes.c_void_p), float(m_lo),
                         float(m_hi), int(n_intervals))
    if c < 0:
        raise ValueError("pwa_envelope: invalid arguments")
    return float(c)


def _gen(self, waves, V, seed, stream_id, cand0, n_cand, envelope, kin, max_out, n_acc, stream=None):
    """kin float32 [3][ld_out] output; n_acc int64 [1] device output."""
    _check_cuda(V, "V", torch.complex64)
    _check_cuda(kin, "kin", torch.float32)
    _check_cuda(n_acc, "n_accepted", torch.int64)
    self._chk(self.lib.pwa_generate(self.h, _wave_array(waves), len(waves), _ptr(V), int(seed), int(stream_id),
                                    int(cand0), int(n_cand), float(envelope), _ptr(kin), int(kin.shape[1]),
                                    int(max_out), _ptr(n_acc), _stream_ptr(stream)))


Handle.pwa_generate = _gen


def fit_opts(**kw) -> pwa_fit_opts:
    o = pwa_fit_opts()
    load().pwa_fit_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _fit_batch(self, fits, opts=None, stream=None):
    """fits: list of dicts with A (complex64 [K][ld]), n, Psi (complex128 [K][K]), n_factor,
    V0 (complex64 [P][K]) and optionally V_out (complex128 [P][K]).  Returns a list of
    per-start result dicts in (fit, start) order."""
    arr = (pwa_fit_desc * len(fits))()
    P_tot = 0
    for i, f in enumerate(fits):
        _check_cuda(f["A"], "A", torch.complex64)
        _check_cuda(f["Psi"], "Psi", torch.complex128)
        _check_cuda(f["V0"], "V0", torch.complex64)
        _check_cuda(f.get("V_out"), "V_out", torch.complex128)
        K, ld = f["A"].shape
        P = f["V0"].shape[0]
        arr[i] = pwa_fit_desc(f["A"].data_ptr(), K, int(f["n"]), ld, f["Psi"].data_ptr(), float(f["n_factor"]), P,
                              f["V0"].data_ptr(), f["V_out"].data_ptr() if f.get("V_out") is not None else None)
        P_tot += P
    res = (pwa_fit_result * P_tot)()
    o = opts if opts is not None else fit_opts()
    self._chk(self.lib.pwa_fit_batch(self.h, arr, len(fits), ctypes.byref(o), res, _stream_ptr(stream)))
    return [dict(nll=r.nll, grad_max=r.grad_max, iterations=r.iterations, evaluations=r.evaluations, status=r.status)
            for r in res]


Handle.pwa_fit_batch = _fit_batch


def _nll_grad_shape(self, A, dA, n, A_mc, dA_mc, n_mc, float_wave, V, n_factor, nll, grad, w_mc=None, n_gen=None,
                    stream=None):
    """Floating-shape -lnL: A [K][ld], dA [F][ld], A_mc [K][ld_mc], dA_mc [F][ld_mc] complex64;
    V complex64 [K]; nll float64 [1], grad float64 [2K+F] outputs."""
    for t, nm in ((A, "A"), (A_mc, "A_mc"), (V, "V")):
        _check_cuda(t, nm, torch.complex64)
    _check_cuda(dA, "dA", torch.complex64)
    _check_cuda(dA_mc, "dA_mc", torch.complex64)
    _check_cuda(nll, "nll", torch.float64)
    _check_cuda(grad, "grad", torch.float64)
    _check_cuda(w_mc, "w_mc", torch.float32)
    K, ld = A.shape
    ld_mc = A_mc.shape[1]
    F = len(float_wave)
    fw = (ctypes.c_int * max(F, 1))(*[int(x) for x in float_wave])
    self._chk(self.lib.pwa_nll_grad_shape(self.h, _ptr(A), _ptr(dA), K, int(n), ld, _ptr(A_mc), _ptr(dA_mc),
                                          int(n_mc), ld_mc, _ptr(w_mc), float(n_mc if n_gen is None else n_gen), fw,
                                          F, _ptr(V), float(n_factor), _ptr(nll), _ptr(grad), _stream_ptr(stream)))


Handle.pwa_nll_grad_shape = _nll_grad_shape


def _uneven_array(channels):
    """pwa_uneven_channel[] from dicts with waves [(J, lambda, M, W)], kin / kin_mc (float32 [3][ld]
    CUDA), n, n_mc, optional n_gen, n_factor, w_mc, float_wave, float_kind.  Returns the array and
    the host buffers it points into (keep them alive for the call)."""
    arr = (pwa_uneven_channel * len(channels))()
    keep = []
    for i, c in enumerate(channels):
        K = len(c["waves"])
        fwv = c.get("float_wave", [])
        F = len(fwv)
        _check_cuda(c["kin"], "kin", torch.float32)
        _check_cuda(c["kin_mc"], "kin_mc", torch.float32)
        _check_cuda(c.get("w_mc"), "w_mc", torch.float32)
        wv = _wave_array(c["waves"])
        fw = (ctypes.c_int * max(F, 1))(*[int(x) for x in fwv])
        fk = (ctypes.c_int * max(F, 1))(*[int(x) for x in c.get("float_kind", [])])
        keep += [wv, fw, fk]
        arr[i] = pwa_uneven_channel(wv, K, c["kin"].data_ptr(), int(c["n"]), c["kin"].shape[1], c["kin_mc"].data_ptr(),
                                    int(c["n_mc"]), c["kin_mc"].shape[1],
                                    c["w_mc"].data_ptr() if c.get("w_mc") is not None else None,
                                    float(c.get("n_gen", c["n_mc"])), float(c.get("n_factor", c["n"])), F, fw, fk)
    return arr, keep


def _nll_grad_uneven(self, channels, V, theta, nll, grad, stream=None):
    """f and gradient of many channels in one launch.  V complex64 [sum K] (CUDA), theta float64
    [sum F] or None, nll float64 [n_ch], grad float64 [sum (2K + F)] (outputs)."""
    _check_cuda(V, "V", torch.complex64)
    _check_cuda(theta, "theta", torch.float64)
    _check_cuda(nll, "nll", torch.float64)
    _check_cuda(grad, "grad", torch.float64)
    arr, keep = _uneven_array(channels)
    self._chk(self.lib.pwa_nll_grad_uneven(self.h, arr, len(channels), _ptr(V), _ptr(theta), _ptr(nll), _ptr(grad),
                                           _stream_ptr(stream)))
    del keep


Handle.pwa_nll_grad_uneven = _nll_grad_uneven


def _fit_shape_batch(self, channels, opts=None, stream=None):
    """channels: list of dicts with waves [(J, lambda, M, W)], kin / kin_mc (float32 [3][ld] CUDA),
    n, n_mc, n_gen, n_factor, float_wave, float_kind, V0 (complex64 [K] CUDA), optional w_mc and
    x_out (float64 [2K+F] CUDA).  Returns per-channel results."""
    arr = (pwa_shape_fit_desc * len(channels))()
    keep = []
    for i, c in enumerate(channels):
        K = len(c["waves"])
        F = len(c["float_wave"])
        ld, ld_mc = c["kin"].shape[1], c["kin_mc"].shape[1]
        wv = _wave_array(c["waves"])
        fw = (ctypes.c_int * max(F, 1))(*[int(x) for x in c["float_wave"]])
        fk = (ctypes.c_int * max(F, 1))(*[int(x) for x in c["float_kind"]])
        _check_cuda(c["V0"], "V0", torch.complex64)
        _check_cuda(c.get("x_out"), "x_out", torch.float64)
        keep += [wv, fw, fk]
        arr[i] = pwa_shape_fit_desc(wv, K, c["kin"].data_ptr(), int(c["n"]), ld, c["kin_mc"].data_ptr(), int(c["n_mc"]),
                                    ld_mc, c["w_mc"].data_ptr() if c.get("w_mc") is not None else None,
                                    float(c.get("n_gen", c["n_mc"])), float(c.get("n_factor", c["n"])), F, fw, fk,
                                    None, None, None, None, c["V0"].data_ptr(),
                                    c["x_out"].data_ptr() if c.get("x_out") is not None else None)
    res = (pwa_fit_result * len(channels))()
    o = opts if opts is not None else fit_opts()
    self._chk(self.lib.pwa_fit_shape_batch(self.h, arr, len(channels), ctypes.byref(o), res, _stream_ptr(stream)))
    torch.cuda.synchronize()
    del keep
    return [dict(nll=r.nll, grad_max=r.grad_max, iterations=r.iterations, evaluations=r.evaluations, status=r.status)
            for r in res]


Handle.pwa_fit_shape_batch = _fit_shape_batch


def _moments(self, kin, n, feat, n_bins=40, m_lo=0.99, m_hi=3.0, stream=None):
    _check_cuda(kin, "kin", torch.float32)
    _check_cuda(feat, "feat", torch.float64)
    self._chk(self.lib.pwa_moments(self.h, _ptr(kin), int(n), int(kin.shape[1]), int(n_bins), float(m_lo),
                                   float(m_hi), _ptr(feat), _stream_ptr(stream)))


def _toy_moments(self, waves, V, Psi_flat, n_target, seed, stream_base, feat, n_acc, n_bins=40, stream=None):
    """V complex64 [T][K]; Psi_flat complex128 [K][K]; feat float64 [T][n_bins*25]; n_acc int64 [T]."""
    _check_cuda(V, "V", torch.complex64)
    _check_cuda(Psi_flat, "Psi_flat", torch.complex128)
    _check_cuda(feat, "feat", torch.float64)
    _check_cuda(n_acc, "n_acc", torch.int64)
    self._chk(self.lib.pwa_toy_moments(self.h, _wave_array(waves), len(waves), _ptr(V), int(V.shape[0]),
                                       _ptr(Psi_flat), float(n_target), int(seed), int(stream_base), int(n_bins),
                                       _ptr(feat), _ptr(n_acc), _stream_ptr(stream)))


Handle.pwa_moments = _moments


def _dtype_code(t):
    if t.dtype == torch.float32:
        return 0
    if t.dtype == torch.bfloat16:
        return 1
    raise ValueError("float32 or bfloat16 expected")


def _mlp_gemm(self, M, N, Kc, A, sa, B, sb, C=None, C_bf16=None, bias=None, relu=False, accumulate=False, ldc=None,
              stream=None):
    """C[m][n] = sum_k A(m,k) B(n,k) (+bias) (ReLU); sa = (sam, sak), sb = (sbn, sbk) element strides."""
    for t, nm in ((A, "A"), (B, "B")):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{nm} must be a contiguous CUDA tensor")
    _check_cuda(C, "C", torch.float32)
    _check_cuda(C_bf16, "C_bf16", torch.bfloat16)
    _check_cuda(bias, "bias", torch.float32)
    self._chk(self.lib.pwa_mlp_gemm(self.h, int(M), int(N), int(Kc), _ptr(A), _dtype_code(A), int(sa[0]), int(sa[1]),
                                    _ptr(B), _dtype_code(B), int(sb[0]), int(sb[1]), _ptr(bias), int(relu),
                                    int(accumulate), _ptr(C), _ptr(C_bf16), int(ldc if ldc is not None else N),
                                    _stream_ptr(stream)))


def _mlp_relu_backward(self, Y_bf16, dY, stream=None):
    _check_cuda(Y_bf16, "Y", torch.bfloat16)
    _check_cuda(dY, "dY", torch.float32)
    self._chk(self.lib.pwa_mlp_relu_backward(self.h, _ptr(Y_bf16), _ptr(dY), int(dY.numel()), _stream_ptr(stream)))


def _mlp_bias_grad(self, dY, db, stream=None):
    _check_cuda(dY, "dY", torch.float32)
    _check_cuda(db, "db", torch.float32)
    B, N = dY.shape
    self._chk(self.lib.pwa_mlp_bias_grad(self.h, _ptr(dY), int(B), int(N), _ptr(db), _stream_ptr(stream)))


def _mlp_wta_loss(self, out, target, C, K, eps, loss, dout=None, winner=None, stream=None):
    _check_cuda(out, "out", torch.float32)
    _check_cuda(target, "target", torch.float32)
    _check_cuda(loss, "loss", torch.float32)
    _check_cuda(dout, "dout", torch.float32)
    _check_cuda(winner, "winner", torch.int32)
    B = target.shape[0]
    self._chk(self.lib.pwa_mlp_wta_loss(self.h, _ptr(out), _ptr(target), int(B), int(C), int(K), float(eps),
                                        _ptr(loss), _ptr(dout), _ptr(winner), _stream_ptr(stream)))


def _mlp_adam(self, p, g, m, v, p_bf16, lr, step, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    for t, nm in ((p, "p"), (g, "g"), (m, "m"), (v, "v")):
        _check_cuda(t, nm, torch.float32)
    _check_cuda(p_bf16, "p_bf16", torch.bfloat16)
    self._chk(self.lib.pwa_mlp_adam(self.h, _ptr(p), _ptr(g), _ptr(m), _ptr(v), _ptr(p_bf16), int(p.numel()),
                                    float(lr), float(b1), float(b2), float(eps), int(step), _stream_ptr(stream)))


def _mlp_to_bf16(self, x, y, scale=1.0, stream=None):
    _check_cuda(x, "x", torch.float64)
    _check_cuda(y, "y", torch.bfloat16)
    self._chk(self.lib.pwa_mlp_to_bf16(self.h, _ptr(x), _ptr(y), int(x.numel()), float(scale), _stream_ptr(stream)))


Handle.pwa_mlp_gemm = _mlp_gemm
Handle.pwa_mlp_relu_backward = _mlp_relu_backward
Handle.pwa_mlp_bias_grad = _mlp_bias_grad
Handle.pwa_mlp_wta_loss = _mlp_wta_loss
Handle.pwa_mlp_adam = _mlp_adam
Handle.pwa_mlp_to_bf16 = _mlp_to_bf16
Handle.pwa_toy_moments = _toy_moments


def waves_from(ws) -> list[tuple[int, int, float, float]]:
    """inputs.WaveSet -> list of (J, lambda, mass, width)."""
    return [(int(ws.J[a]), int(ws.lam[a]), float(ws.M[a]), float(ws.W[a])) for a in range(ws.K)]
