"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads, and
exports every entry point include/pwa.h declares; calls that need no device behave as
documented; without a device pwa_create fails with PWA_ERR_NO_DEVICE (no CPU fallback)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1108_5882_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = pbuild.build()
    return ctypes.CDLL(path)


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^PWA_API[^(]*?\b(pwa_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pwa_amplitudes", "pwa_normint", "pwa_nll", "pwa_nll_grad", "pwa_create",
                     "pwa_destroy", "pwa_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    lib.pwa_status_string.restype = ctypes.c_char_p
    assert lib.pwa_status_string(0) == b"PWA_OK"
    assert lib.pwa_status_string(-4) == b"PWA_ERR_NONFINITE"
    assert lib.pwa_status_string(12345) == b"PWA_UNKNOWN_STATUS"
    assert lib.pwa_abi_version() >= 1


def test_create_without_device_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    h = ctypes.c_void_p()
    st = lib.pwa_create(ctypes.byref(h), 0)
    assert st == -2 and not h.value  # PWA_ERR_NO_DEVICE
    lib.pwa_last_error.restype = ctypes.c_char_p
    assert b"no CUDA device" in lib.pwa_last_error(None)


def test_binding_refuses_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_1108_5882_gb300 import pwa
    with pytest.raises(pwa.PWAError):
        pwa.Handle(0)


def test_null_handle_is_rejected(lib):
    assert lib.pwa_nll(None, None, 4, 0, 0, None, 1, None, ctypes.c_double(1.0), None, None) == -1
    lib.pwa_destroy(None)  # no-op


def test_envelope_host_matches_oracle():
    # the library's host-side accept-reject bound against the oracle's independent one
    import oracle
    from paper_1108_5882_gb300 import inputs, pwa
    ws = inputs.wave_set_spread(16, 5)
    V = inputs.production_amplitudes(16, 5)
    c_lib = pwa.pwa_envelope(pwa.waves_from(ws), V)
    c_orc = oracle.envelope(ws.M, ws.W, V.astype(np.complex128))
    assert abs(c_lib - c_orc) < 1e-6 * c_orc
    assert c_lib < float(np.sum(np.abs(V).astype(np.float64))) ** 2  # tighter than (sum |V|)^2


def test_fit_default_options_and_their_binding_layout():
    # pwa_fit_default_opts needs no device; the ctypes mirror of pwa_fit_opts must match the C
    # layout field by field (a missing or misordered field would shift every later one)
    from paper_1108_5882_gb300 import pwa
    o = pwa.fit_opts()
    assert (o.max_iter, o.history, o.gtol, o.check_every, o.gauge_fix, o.use_graph, o.polar) == \
        (1000, 10, 1e-6, 20, 1, 1, 0)
    src = open(os.path.join(ROOT, "include", "pwa.h")).read()
    body = re.search(r"typedef struct pwa_fit_opts \{(.*?)\} pwa_fit_opts;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    c_fields = re.findall(r"\b(\w+)\s*;", body)
    assert c_fields == [f for f, _ in pwa.pwa_fit_opts._fields_]
    assert pwa.fit_opts(polar=1).polar == 1


def test_barrier_recurrence_of_the_library_header_matches_the_oracle():
    # the host/device barrier factor of csrc/barrier.cuh (Hankel recurrence), compiled here as
    # plain C++ with g++, against the oracle's textbook polynomials for L = 0..4
    import shutil
    import subprocess
    import tempfile
    import oracle
    if not shutil.which("g++"):
        pytest.skip("no g++")
    src = open(os.path.join(ROOT, "paper_1108_5882_gb300", "csrc", "barrier.cuh")).read()
    fn = re.search(r"(__host__ __device__ inline double barrier2_host\(.*?\n\})", src, flags=re.S).group(1)
    fn = fn.replace("__host__ __device__ ", "")
    prog = "#include <cmath>\n#include <cstdio>\nusing std::sqrt;\n" + fn + """
int main() {
    const double zs[] = {1e-6, 0.01, 0.3, 1.0, 3.0, 10.0, 80.0, 1e4};
    for (int L = 0; L <= 4; ++L)
        for (double z : zs) std::printf("%d %.17g %.17g\\n", L, z, barrier2_host(L, z));
}
"""
    with tempfile.TemporaryDirectory() as d:
        cpp, exe = os.path.join(d, "b.cpp"), os.path.join(d, "b")
        open(cpp, "w").write(prog)
        subprocess.run(["g++", "-O1", "-o", exe, cpp], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    for line in out.strip().splitlines():
        L, z, v = line.split()
        ref = oracle.barrier2(int(L), float(z))
        assert abs(float(v) - ref) <= 1e-13 * ref + 1e-300, (L, z, v, ref)
