"""The allocation-free entry point pwa_nll_grad_noalloc, called through the C ABI.

It exists for callers that cannot allocate device memory (inside a stream capture they do not
own, under a memory manager that forbids allocation after start-up, or as a plug-in of a
program that owns the device memory): it uses scratch compiled into the library instead of a
handle and its workspace.  Its results must agree with the handle-based pwa_nll_grad within
the tolerances the parity tests use, on two calls in a row (the second call runs on the
scratch the first one left behind).  This file is collected last on purpose.
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


def test_noalloc_matches_handle_entry_point_on_two_calls():
    from paper_1108_5882_gb300 import pwa
    lib, f = _noalloc_fn()
    torch.cuda.set_device(0)
    K, n = 16, 150_001  # several blocks and an odd (ragged) tail
    ws = inputs.wave_set_spread(K, inputs.SEED_BASE + 42)
    kin = inputs.kinematics(n, inputs.SEED_BASE + 42, 4)
    A = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin).astype(np.complex64)
    kin_mc = inputs.kinematics(100_000, inputs.SEED_BASE + 42, 5)
    Psi = oracle.normint(oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin_mc).astype(np.complex64))
    ld = n + 1
    Ad = torch.zeros((K, ld), dtype=torch.complex64, device="cuda")
    Ad[:, :n] = torch.from_numpy(A)
    Psid = torch.from_numpy(Psi).cuda()
    h = pwa.Handle(0)
    Vs = inputs.starts(2, K, 7)
    stream = torch.cuda.current_stream()
    for call in range(2):  # two calls in a row on the shared scratch
        V = torch.from_numpy(np.ascontiguousarray(Vs[call:call + 1])).cuda()
        nll_r = torch.zeros(1, dtype=torch.float64, device="cuda")
        g_r = torch.zeros((1, 2 * K), dtype=torch.float64, device="cuda")
        h.pwa_nll_grad(Ad, n, V, Psid, float(n), nll_r, g_r)
        nll_n = torch.zeros(1, dtype=torch.float64, device="cuda")
        g_n = torch.zeros((1, 2 * K), dtype=torch.float64, device="cuda")
        st = f(ctypes.c_void_p(Ad.data_ptr()), K, n, ld, ctypes.c_void_p(V.data_ptr()),
               ctypes.c_void_p(Psid.data_ptr()), float(n), ctypes.c_void_p(nll_n.data_ptr()),
               ctypes.c_void_p(g_n.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == pwa.PWA_OK, lib.pwa_last_error(None)
        torch.cuda.synchronize()
        _, _, cf, cg, _ = oracle.nll_grad(A, Vs[call:call + 1], Psi, with_cond=True)
        assert abs(nll_n.item() - nll_r.item()) <= 1e-5 * cf[0]
        assert np.all(np.abs(g_n.cpu().numpy()[0] - g_r.cpu().numpy()[0]) <= 1e-4 * np.repeat(cg[0], 2))
    h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1108_5882_gb300 import pwa
    lib, f = _noalloc_fn()
    st = f(None, 65, 0, 0, None, None, 1.0, None, None, None)
    assert st == pwa.PWA_ERR_INVALID_ARG
    assert b"K outside" in lib.pwa_last_error(None)
