"""The allocation-free entry point pwa_nll_grad_noalloc, called through the C ABI.

It exists for callers that cannot allocate device memory (under a memory manager that forbids
allocation after start-up, as a plug-in of a program that owns the device memory, or in a
latency-critical loop that must not take the allocator's locks): it uses scratch compiled into
the library instead of a handle and its workspace.  Its results must agree with the FP64
oracle and with the handle-based pwa_nll_grad within the tolerances the parity tests use, on
calls in a row (each call runs on the scratch the previous one left behind).  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1108_5882_gb300 import inputs

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    from paper_1108_5882_gb300 import build, pwa
    build.build()
    lib = pwa.load()
    f = lib.pwa_nll_grad_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, vp, vp, ctypes.c_double, vp, vp, vp]
    f.restype = ctypes.c_int
    return lib, f


def _call(f, A, K, n, ld, V, Psi, n_factor):
    """One call on the current stream; returns (nll, grad [2K]) after a synchronise."""
    nll = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros((1, 2 * K), dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    st = f(vp(A.data_ptr() if A is not None else None), K, n, ld, vp(V.data_ptr()), vp(Psi.data_ptr()), float(n_factor),
           vp(nll.data_ptr()), vp(g.data_ptr()), vp(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, nll.item(), g.cpu().numpy()[0]


def _problem(K, n, seed):
    ws = inputs.wave_set_spread(K, seed)
    kin = inputs.kinematics(n, seed, 4)
    A = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin).astype(np.complex64)
    kin_mc = inputs.kinematics(50_000, seed, 5)
    Psi = oracle.normint(oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin_mc).astype(np.complex64))
    ld = n + (n & 1)
    Ad = torch.zeros((K, ld), dtype=torch.complex64, device="cuda")
    Ad[:, :n] = torch.from_numpy(A)
    return A, Ad, ld, Psi, torch.from_numpy(Psi).cuda()


def _check_oracle(nll, g, A, V, Psi, n_factor):
    f_ref, g_ref, cf, cg, bad = oracle.nll_grad(A, V, Psi, n_factor=n_factor, with_cond=True)
    assert bad == 0
    assert abs(nll - f_ref[0]) <= 1e-5 * cf[0], (nll, f_ref[0])
    assert np.all(np.abs(g - g_ref[0]) <= 1e-4 * np.repeat(cg[0], 2))
    return cf[0], cg[0]


def test_noalloc_matches_oracle_and_handle_entry_point_on_two_calls():
    from paper_1108_5882_gb300 import pwa
    lib, f = _noalloc_fn()
    torch.cuda.set_device(0)
    K, n = 16, 150_001  # several blocks and an odd (ragged) tail
    A, Ad, ld, Psi, Psid = _problem(K, n, inputs.SEED_BASE + 42)
    h = pwa.Handle(0)
    Vs = inputs.starts(2, K, 7)
    for call in range(2):  # two calls in a row on the shared scratch
        V = torch.from_numpy(np.ascontiguousarray(Vs[call:call + 1])).cuda()
        nll_r = torch.zeros(1, dtype=torch.float64, device="cuda")
        g_r = torch.zeros((1, 2 * K), dtype=torch.float64, device="cuda")
        h.pwa_nll_grad(Ad, n, V, Psid, float(n), nll_r, g_r)
        st, nll_n, g_n = _call(f, Ad, K, n, ld, V, Psid, n)
        assert st == pwa.PWA_OK, lib.pwa_last_error(None)
        cf, cg = _check_oracle(nll_n, g_n, A, Vs[call:call + 1], Psi, n)
        assert abs(nll_n - nll_r.item()) <= 1e-5 * cf
        assert np.all(np.abs(g_n - g_r.cpu().numpy()[0]) <= 1e-4 * np.repeat(cg, 2))
    h.close()


@pytest.mark.parametrize("K,n", [(16, 4_000_001), (4, 4_000_000), (64, 30_001)])
def test_noalloc_large_and_wide_against_oracle(K, n):
    # n = 4e6 wants more blocks than the scratch holds partial sums for: the launch is capped
    # (at 1024 blocks, or fewer where the occupancy bound is lower) and every block strides over
    # the events; K = 64 fills the widest partial-sum rows.  Two calls in a row each.
    from paper_1108_5882_gb300 import pwa
    lib, f = _noalloc_fn()
    torch.cuda.set_device(0)
    A, Ad, ld, Psi, Psid = _problem(K, n, inputs.SEED_BASE + 43 + K)
    Vs = inputs.starts(2, K, 8 + K)
    for call in range(2):
        V = torch.from_numpy(np.ascontiguousarray(Vs[call:call + 1])).cuda()
        st, nll_n, g_n = _call(f, Ad, K, n, ld, V, Psid, n)
        assert st == pwa.PWA_OK, lib.pwa_last_error(None)
        _check_oracle(nll_n, g_n, A, Vs[call:call + 1], Psi, n)


def test_noalloc_flags_clear_between_calls_and_empty_sample():
    # A set with I_i = 0 everywhere (V = 0) gives nll = +inf and a zero gradient; the next call,
    # with a good V, must start from cleared flags and match the oracle.  n = 0 (A may be NULL)
    # leaves only the normalisation term: f = n_f S(V), g = 2 n_f Psi^T V.
    from paper_1108_5882_gb300 import pwa
    lib, f = _noalloc_fn()
    torch.cuda.set_device(0)
    K, n = 8, 10_001
    A, Ad, ld, Psi, Psid = _problem(K, n, inputs.SEED_BASE + 44)
    V0 = torch.zeros((1, K), dtype=torch.complex64, device="cuda")
    st, nll0, g0 = _call(f, Ad, K, n, ld, V0, Psid, n)
    assert st == pwa.PWA_OK and nll0 == float("inf") and np.all(g0 == 0)
    Vg = inputs.starts(1, K, 9)
    st, nll1, g1 = _call(f, Ad, K, n, ld, torch.from_numpy(Vg).cuda(), Psid, n)
    assert st == pwa.PWA_OK
    _check_oracle(nll1, g1, A, Vg, Psi, n)
    st, nll2, g2 = _call(f, None, K, 0, 0, torch.from_numpy(Vg).cuda(), Psid, 1000.0)
    assert st == pwa.PWA_OK
    v = Vg[0].astype(np.complex128)
    S = float(np.real(v @ Psi @ v.conj()))
    gc = 2 * 1000.0 * (Psi.T @ v)
    assert abs(nll2 - 1000.0 * S) <= 1e-10 * 1000.0 * S
    assert np.all(np.abs(g2[0::2] - gc.real) <= 1e-10 * np.abs(gc).max())
    assert np.all(np.abs(g2[1::2] - gc.imag) <= 1e-10 * np.abs(gc).max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1108_5882_gb300 import pwa
    lib, f = _noalloc_fn()
    st = f(None, 65, 0, 0, None, None, 1.0, None, None, None)
    assert st == pwa.PWA_ERR_INVALID_ARG
    assert b"K outside" in lib.pwa_last_error(None)
