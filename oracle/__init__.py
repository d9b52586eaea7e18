"""FP64 CPU oracle for the partial-wave-analysis likelihood (Berger, arXiv:1108.5882, Sec. 2).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  The oracle shares no code with the CUDA library and never
imports it.  The arithmetic lives in plain C (``pwa_oracle.c``, FP64, single-threaded); this
module compiles it with gcc on first use and marshals numpy arrays through ctypes.

Functions and the passages they follow:
  amplitudes   -- A_a(Omega) of Eq. 1 under the fixed-width unit-peak Breit-Wigner reading
  amplitudes_barrier, breakup_q, barrier2 -- the same with a mass-dependent width and
                  Blatt-Weisskopf barrier factors (L = J, spinless daughters)
  normint      -- Psi_ab, the inner bracket of Eq. 3 (MC sum over accepted events / N_gen)
  nll_grad     -- -lnL of Eq. 3 (extended form, footnote 2) and its gradient in V
  nll_double_sum -- Eq. 3 in its printed K^2 double-sum form, long double (pin only)
  envelope, generate, candidates -- accept-reject toys from I of Eq. 1 (Philox4x32-10 candidates)
  moments      -- per-mass-bin averages of the real Y_LM (features of the learned proposer)
  nll_grad_shape, nll_shape_from_kin -- the objective with floating masses and widths (Sec. 2)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = [os.path.join(_HERE, f) for f in ("pwa_oracle.c", "pwa_oracle_gen.c")]
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, strict IEEE FP64)."""
    srcs = list(_SRC)
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_amplitudes.argtypes = [ctypes.c_int, _ip, _ip, _dp, _dp, _i64, _fp, _i64,
                                           _dp, _dp, _dp]
            lib.orc_amplitudes.restype = None
            lib.orc_normint.argtypes = [ctypes.c_int, _i64, _fp, _i64, _fp, ctypes.c_double, _dp]
            lib.orc_normint.restype = None
            lib.orc_nll_grad.argtypes = [ctypes.c_int, _i64, _fp, _i64, ctypes.c_int, _dp, _dp,
                                         ctypes.c_double, _dp, _dp, _dp, _dp]
            lib.orc_nll_grad.restype = ctypes.c_int
            lib.orc_nll_grad_incoherent.argtypes = [ctypes.c_int, ctypes.c_int, _i64, _fp, _i64, ctypes.c_int, _dp,
                                                    _dp, ctypes.c_double, _dp, _dp, _dp, _dp]
            lib.orc_nll_grad_incoherent.restype = ctypes.c_int
            lib.orc_hessian.argtypes = [ctypes.c_int, _i64, _fp, _i64, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp]
            lib.orc_hessian.restype = ctypes.c_int
            lib.orc_nll_double_sum.argtypes = [ctypes.c_int, _i64, _fp, _i64, _dp, _dp,
                                               ctypes.c_double]
            lib.orc_nll_double_sum.restype = ctypes.c_double
            lib.orc_legendre.argtypes = [ctypes.c_int, ctypes.c_double]
            lib.orc_legendre.restype = ctypes.c_double
            lib.orc_breakup_q.argtypes = [ctypes.c_double] * 3
            lib.orc_breakup_q.restype = ctypes.c_double
            lib.orc_barrier2.argtypes = [ctypes.c_int, ctypes.c_double]
            lib.orc_barrier2.restype = ctypes.c_double
            lib.orc_amplitudes_barrier.argtypes = [ctypes.c_int, _ip, _ip, _dp, _dp, ctypes.c_double,
                                                   ctypes.c_double, ctypes.c_double, _i64, _fp, _i64, _dp]
            lib.orc_amplitudes_barrier.restype = None
            _register_gen(lib)
            _lib = lib
    return _lib


def _register_gen(lib):
    # generator, moments and floating-shape functions (pwa_oracle_gen.c, pwa_oracle.c)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.orc_philox4x32.argtypes = [u32p, u32p, u32p]
    lib.orc_philox4x32.restype = None
    lib.orc_envelope.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.orc_envelope.restype = ctypes.c_double
    lib.orc_generate.argtypes = [ctypes.c_int, _ip, _ip, _dp, _dp, _dp, ctypes.c_uint64, ctypes.c_uint32, _i64,
                                 _i64, ctypes.c_double, _fp, _i64, _i64, _dp]
    lib.orc_generate.restype = ctypes.c_int64
    lib.orc_candidates.argtypes = [ctypes.c_int, _ip, _ip, _dp, _dp, _dp, ctypes.c_uint64, ctypes.c_uint32, _i64,
                                   _i64, _fp, _fp, _dp, _dp]
    lib.orc_candidates.restype = None
    lib.orc_ylm_real.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.orc_ylm_real.restype = ctypes.c_double
    lib.orc_moments.argtypes = [_i64, _fp, _i64, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
    lib.orc_moments.restype = None
    lib.orc_nll_grad_shape.argtypes = [ctypes.c_int, _i64, _fp, _fp, _i64, _i64, _fp, _fp, _i64, _fp, ctypes.c_double,
                                       _ip, ctypes.c_int, _dp, ctypes.c_double, _dp, _dp, _dp]
    lib.orc_nll_grad_shape.restype = ctypes.c_int
    lib.orc_nll_shape_from_kin.argtypes = [ctypes.c_int, _ip, _ip, _dp, _dp, _i64, _fp, _i64, _fp, ctypes.c_double,
                                           _dp, ctypes.c_double]
    lib.orc_nll_shape_from_kin.restype = ctypes.c_double


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _c64_as_f32(A):
    """complex64 [K][ld] -> contiguous float32 view [K][2*ld] (interleaved re, im)."""
    A = np.ascontiguousarray(A, dtype=np.complex64)
    return A.view(np.float32)


def legendre(J: int, x: float) -> float:
    return _load().orc_legendre(int(J), float(x))


def amplitudes(J, lam, M, W, kin, derivs: bool = False):
    """A_a(Omega_i), complex128 [K][n] (plus dA/dM, dA/dGamma if ``derivs``).

    kin: float32 [3][n] (m, cos theta, phi).  J, lam: int per wave; M, W: float64 per wave."""
    lib = _load()
    J = np.ascontiguousarray(J, dtype=np.int32)
    lam = np.ascontiguousarray(lam, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    kin = np.ascontiguousarray(kin, dtype=np.float32)
    K = J.shape[0]
    n = kin.shape[1]
    A = np.zeros((K, n), dtype=np.complex128)
    dM = np.zeros((K, n), dtype=np.complex128) if derivs else None
    dW = np.zeros((K, n), dtype=np.complex128) if derivs else None
    lib.orc_amplitudes(K, _ptr(J, _ip), _ptr(lam, _ip), _ptr(M, _dp), _ptr(W, _dp), n,
                       _ptr(kin, _fp), n, _ptr(A, _dp), _ptr(dM, _dp), _ptr(dW, _dp))
    return (A, dM, dW) if derivs else A


def breakup_q(m, m1, m2):
    """Two-body breakup momentum q(m) for m -> m1 + m2 (0 at and below threshold)."""
    return _load().orc_breakup_q(float(m), float(m1), float(m2))


def barrier2(L, z):
    """Squared Blatt-Weisskopf factor B_L^2 at z = (q R)^2, L <= 4, normalised to 1 at z -> inf."""
    return _load().orc_barrier2(int(L), float(z))


def amplitudes_barrier(J, lam, M, W, m1, m2, R, kin):
    """A_a(Omega_i), complex128 [K][n], with the mass-dependent width and Blatt-Weisskopf
    barrier factors of a decay into spinless daughters m1, m2 (L = J, radius R in GeV^-1)."""
    lib = _load()
    J = np.ascontiguousarray(J, dtype=np.int32)
    lam = np.ascontiguousarray(lam, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    kin = np.ascontiguousarray(kin, dtype=np.float32)
    K, n = J.shape[0], kin.shape[1]
    A = np.zeros((K, n), dtype=np.complex128)
    lib.orc_amplitudes_barrier(K, _ptr(J, _ip), _ptr(lam, _ip), _ptr(M, _dp), _ptr(W, _dp), float(m1), float(m2),
                               float(R), n, _ptr(kin, _fp), n, _ptr(A, _dp))
    return A


def normint(A, w=None, n_gen=None):
    """Psi (complex128 [K][K]) from complex64 MC amplitudes A [K][n]; w optional float32 [n]."""
    lib = _load()
    K, n = A.shape
    Af = _c64_as_f32(A)
    wf = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    if n_gen is None:
        n_gen = float(n)
    Psi = np.zeros((K, K), dtype=np.complex128)
    lib.orc_normint(K, n, _ptr(Af, _fp), n, _ptr(wf, _fp), float(n_gen), _ptr(Psi, _dp))
    return Psi


def nll_grad(A, V, Psi, n_factor=None, with_cond: bool = False):
    """(-lnL [P], grad [P][2K] as (Re g, Im g) pairs) for complex64 A [K][n], V [P][K]
    (any complex dtype, promoted to complex128) and Psi complex128 [K][K].

    With ``with_cond`` also returns the condition scales (cond_f [P], cond_g [P][K]) the
    parity tolerances are measured against, and the count of sets with I_i <= 0."""
    lib = _load()
    K, n = A.shape
    Af = _c64_as_f32(A)
    V = np.ascontiguousarray(np.atleast_2d(V), dtype=np.complex128)
    P = V.shape[0]
    assert V.shape[1] == K
    Psi = np.ascontiguousarray(Psi, dtype=np.complex128)
    if n_factor is None:
        n_factor = float(n)
    nll = np.zeros(P, dtype=np.float64)
    grad = np.zeros((P, 2 * K), dtype=np.float64)
    cf = np.zeros(P, dtype=np.float64)
    cg = np.zeros((P, K), dtype=np.float64)
    bad = lib.orc_nll_grad(K, n, _ptr(Af, _fp), n, P, _ptr(V, _dp), _ptr(Psi, _dp),
                           float(n_factor), _ptr(nll, _dp), _ptr(grad, _dp), _ptr(cf, _dp),
                           _ptr(cg, _dp))
    if with_cond:
        return nll, grad, cf, cg, bad
    return nll, grad


def nll_grad_incoherent(A, V, Psi, n_factor=None, with_cond: bool = False):
    """-lnL and gradient with the intensity summed incoherently over H states:
    A complex64 [K][H][n], I_i = sum_h |sum_a V_a A[a][h][i]|^2, Psi = the normalisation
    integral summed over h (normint_incoherent).  Outputs as nll_grad."""
    lib = _load()
    K, H, n = A.shape
    Af = _c64_as_f32(np.ascontiguousarray(A).reshape(K, H * n)).reshape(-1)
    V = np.ascontiguousarray(np.atleast_2d(V), dtype=np.complex128)
    P = V.shape[0]
    assert V.shape[1] == K
    Psi = np.ascontiguousarray(Psi, dtype=np.complex128)
    if n_factor is None:
        n_factor = float(n)
    nll = np.zeros(P, dtype=np.float64)
    grad = np.zeros((P, 2 * K), dtype=np.float64)
    cf = np.zeros(P, dtype=np.float64)
    cg = np.zeros((P, K), dtype=np.float64)
    bad = lib.orc_nll_grad_incoherent(K, H, n, _ptr(Af, _fp), n, P, _ptr(V, _dp), _ptr(Psi, _dp), float(n_factor),
                                      _ptr(nll, _dp), _ptr(grad, _dp), _ptr(cf, _dp), _ptr(cg, _dp))
    if with_cond:
        return nll, grad, cf, cg, bad
    return nll, grad


def hessian(A, V, Psi, n_factor=None, exact=False, with_cond: bool = False):
    """Second derivatives of -lnL in theta = (Re V_0, Im V_0, ...) for one set V [K]: the Fumili
    outer-product form sum_i r_i r_i^T (exact=False) or the exact Hessian.  [2K][2K] float64."""
    lib = _load()
    K, n = A.shape
    Af = _c64_as_f32(A)
    V = np.ascontiguousarray(np.asarray(V).reshape(K), dtype=np.complex128)
    Psi = np.ascontiguousarray(Psi, dtype=np.complex128)
    if n_factor is None:
        n_factor = float(n)
    H = np.zeros((2 * K, 2 * K), dtype=np.float64)
    cond = np.zeros((2 * K, 2 * K), dtype=np.float64)
    bad = lib.orc_hessian(K, n, _ptr(Af, _fp), n, _ptr(V, _dp), _ptr(Psi, _dp), float(n_factor), 1 if exact else 0,
                          _ptr(H, _dp), _ptr(cond, _dp))
    if with_cond:
        return H, cond, bad
    return H


def normint_incoherent(A, n_gen=None, w=None):
    """Psi summed over the H states of A complex64 [K][H][n]: the (event, state) pairs are the
    terms of one MC sum, so this is normint over the K x (H n) array (weights repeat per state)."""
    K, H, n = A.shape
    ww = None if w is None else np.tile(np.asarray(w, dtype=np.float32), H)
    return normint(np.ascontiguousarray(A).reshape(K, H * n), n_gen=float(n if n_gen is None else n_gen), w=ww)


def nll_double_sum(A, V, Psi, n_factor=None) -> float:
    """Eq. 3 as printed (K^2 double sum per event), long double; tiny inputs only."""
    lib = _load()
    K, n = A.shape
    Af = _c64_as_f32(A)
    V = np.ascontiguousarray(V, dtype=np.complex128).reshape(K)
    Psi = np.ascontiguousarray(Psi, dtype=np.complex128)
    if n_factor is None:
        n_factor = float(n)
    return lib.orc_nll_double_sum(K, n, _ptr(Af, _fp), n, _ptr(V, _dp), _ptr(Psi, _dp),
                                  float(n_factor))


# ------------------------------------------------------------------ toy generator -------------

def philox4x32(ctr, key):
    """Philox4x32-10 of one 128-bit counter under a 64-bit key -> 4 uint32."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32(c, k, o)
    return [int(x) for x in o]


def envelope(M, W, V, m_lo=0.99, m_hi=3.0, n_int=4096) -> float:
    """Rigorous bound C >= max I(Omega) over the flat phase space (see pwa_oracle_gen.c)."""
    lib = _load()
    M = np.ascontiguousarray(M, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.complex128)
    return lib.orc_envelope(M.shape[0], _ptr(M, _dp), _ptr(W, _dp), _ptr(V, _dp), m_lo, m_hi, n_int)


def generate(J, lam, M, W, V, seed, stream, cand0, n_cand, C, max_out):
    """Accept-reject toys: returns (kin float32 [3][n_out], n_accepted, max I/C)."""
    lib = _load()
    J = np.ascontiguousarray(J, dtype=np.int32)
    lam = np.ascontiguousarray(lam, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.complex128)
    kin = np.zeros((3, max(int(max_out), 1)), dtype=np.float32)
    mr = np.zeros(1, dtype=np.float64)
    na = lib.orc_generate(J.shape[0], _ptr(J, _ip), _ptr(lam, _ip), _ptr(M, _dp), _ptr(W, _dp), _ptr(V, _dp),
                          int(seed), int(stream), int(cand0), int(n_cand), float(C), _ptr(kin, _fp),
                          kin.shape[1], int(max_out), _ptr(mr, _dp))
    n_out = min(int(na), int(max_out))
    return np.ascontiguousarray(kin[:, :n_out]), int(na), float(mr[0])


def candidates(J, lam, M, W, V, seed, stream, cand0, n_cand):
    """Every candidate of an accept-reject range, for decision-by-decision checks: returns
    (kin float32 [3][n_cand], u float32 [n_cand], I float64 [n_cand], s float64 [n_cand]) with I the
    FP64 intensity of Eq. 1 at the candidate and s = sum_a |V_a||A_a| (the rounding scale of u)."""
    lib = _load()
    J = np.ascontiguousarray(J, dtype=np.int32)
    lam = np.ascontiguousarray(lam, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.complex128)
    n_cand = int(n_cand)
    kin = np.zeros((3, n_cand), dtype=np.float32)
    u = np.zeros(n_cand, dtype=np.float32)
    Iv = np.zeros(n_cand, dtype=np.float64)
    s = np.zeros(n_cand, dtype=np.float64)
    lib.orc_candidates(J.shape[0], _ptr(J, _ip), _ptr(lam, _ip), _ptr(M, _dp), _ptr(W, _dp), _ptr(V, _dp), int(seed),
                       int(stream), int(cand0), n_cand, _ptr(kin, _fp), _ptr(u, _fp), _ptr(Iv, _dp), _ptr(s, _dp))
    return kin, u, Iv, s


# ------------------------------------------------------------------ floating masses/widths -----

def nll_grad_shape(A, dA, A_mc, dA_mc, fwave, V, n_factor=None, w_mc=None, n_gen=None):
    """f, grad_V [2K], grad_shape [F] with the streamed MC normalisation (floating M, Gamma).

    A [K][n], dA [F][n], A_mc [K][n_mc], dA_mc [F][n_mc]: complex64; fwave: wave index per
    floating parameter; V complex [K]."""
    lib = _load()
    K, n = A.shape
    n_mc = A_mc.shape[1]
    F = len(fwave)
    Af, dAf = _c64_as_f32(A), _c64_as_f32(dA.reshape(F, n))
    Amf, dAmf = _c64_as_f32(A_mc), _c64_as_f32(dA_mc.reshape(F, n_mc))
    fw = np.ascontiguousarray(fwave, dtype=np.int32)
    Vd = np.ascontiguousarray(V, dtype=np.complex128).reshape(K)
    wf = None if w_mc is None else np.ascontiguousarray(w_mc, dtype=np.float32)
    nll = np.zeros(1)
    gV = np.zeros(2 * K)
    gS = np.zeros(max(F, 1))
    bad = lib.orc_nll_grad_shape(K, n, _ptr(Af, _fp), _ptr(dAf, _fp), n, n_mc, _ptr(Amf, _fp), _ptr(dAmf, _fp), n_mc,
                                 _ptr(wf, _fp), float(n_mc if n_gen is None else n_gen), _ptr(fw, _ip), F,
                                 _ptr(Vd, _dp), float(n if n_factor is None else n_factor), _ptr(nll, _dp),
                                 _ptr(gV, _dp), _ptr(gS, _dp))
    return nll[0], gV, gS[:F], bad


def nll_shape_from_kin(J, lam, M, W, kin, kin_mc, V, n_factor=None, n_gen=None):
    """The floating-parameter objective in FP64 straight from the kinematics."""
    lib = _load()
    J = np.ascontiguousarray(J, dtype=np.int32)
    lam = np.ascontiguousarray(lam, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    kin = np.ascontiguousarray(kin, dtype=np.float32)
    kin_mc = np.ascontiguousarray(kin_mc, dtype=np.float32)
    Vd = np.ascontiguousarray(V, dtype=np.complex128)
    n, n_mc = kin.shape[1], kin_mc.shape[1]
    return lib.orc_nll_shape_from_kin(J.shape[0], _ptr(J, _ip), _ptr(lam, _ip), _ptr(M, _dp), _ptr(W, _dp), n,
                                      _ptr(kin, _fp), n_mc, _ptr(kin_mc, _fp), float(n_mc if n_gen is None else n_gen),
                                      _ptr(Vd, _dp), float(n if n_factor is None else n_factor))


# ------------------------------------------------------------------ angular moments ------------

def ylm_real(L, M, ct, phi) -> float:
    return _load().orc_ylm_real(int(L), int(M), float(ct), float(phi))


def moments(kin, n_bins=40, m_lo=0.99, m_hi=3.0):
    """feat [n_bins][25] = (1/n) sum over events of each mass bin of the real Y_LM, L <= 4."""
    lib = _load()
    kin = np.ascontiguousarray(kin, dtype=np.float32)
    n = kin.shape[1]
    feat = np.zeros((n_bins, 25))
    lib.orc_moments(n, _ptr(kin, _fp), n, int(n_bins), float(m_lo), float(m_hi), _ptr(feat, _dp))
    return feat
