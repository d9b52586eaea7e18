"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances (relative 1e-5 on -lnL and 1e-4 per gradient component, read with condition-aware
denominators):
  -lnL:        |f_gpu - f_ref| <= 1e-5 * max(|f_ref|, sum_i |ln I_i|, n |S|)
  gradient:    |g_gpu - g_ref| <= 1e-4 * (2 sum_i |A_ic| s_i/I_i + 2 n sum_a |Psi_ac||V_a|)
               per real component, s_i = sum_a |V_a||A_ia| >= |u_i| (the forward-error scale of
               the single-precision sum u_i)
  amplitudes:  |A_gpu - A_ref| <= 4e-6 (|A| <= 1: unit-peak Breit-Wigner, |P_J| <= 1); with
               barrier factors 5e-6 * max(1, |A_ref|)
  dA/dM, dA/dG: per wave |err| <= 2e-5 * max_i |dA_ref|
  Psi:         |Psi_gpu - Psi_ref|_ab <= 1e-5 * sqrt(Psi_aa Psi_bb)
  Hessian:     |H_gpu - H_ref| <= 1e-5 * (the same sums of term magnitudes, per entry)
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1108_5882_gb300 import inputs
from problems import fp32_decision_band, make_problem, padded

pytestmark = pytest.mark.gpu

SEED = inputs.SEED_BASE


@pytest.fixture(scope="module")
def h():
    from paper_1108_5882_gb300 import build, pwa
    build.build()
    return pwa.Handle(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_nll_grad(h, A, n, V, Psi, n_factor=None, grad=True):
    from paper_1108_5882_gb300 import pwa  # noqa: F401
    K, ld = A.shape
    P = V.shape[0]
    n_factor = float(n if n_factor is None else n_factor)
    nll = torch.zeros(P, dtype=torch.float64, device="cuda")
    g = torch.zeros(P, 2 * K, dtype=torch.float64, device="cuda")
    if grad:
        h.pwa_nll_grad(dev(A), n, dev(V), dev(Psi), n_factor, nll, g)
    else:
        h.pwa_nll(dev(A), n, dev(V), dev(Psi), n_factor, nll)
    torch.cuda.synchronize()
    return nll.cpu().numpy(), g.cpu().numpy()


def check_nll(f_gpu, g_gpu, A, V, Psi, n_factor=None, check_grad=True):
    f_ref, g_ref, cf, cg, bad = oracle.nll_grad(A, V, Psi, n_factor=n_factor, with_cond=True)
    assert bad == 0
    err_f = np.abs(f_gpu - f_ref) / cf
    assert np.all(err_f <= 1e-5), (err_f.max(), f_gpu, f_ref)
    if check_grad:
        scale = np.repeat(cg, 2, axis=1)
        err_g = np.abs(g_gpu - g_ref) / scale
        assert np.all(err_g <= 1e-4), err_g.max()
    return f_ref, g_ref


def check_plain_gradient(g_gpu, A, V, Psi, n_factor=None):
    """At a random (non-stationary) V the gradient is O(N) and needs no condition-aware scale:
    every component with |g_ref| >= 1e-3 max|g_ref| within 1e-4 of itself, and max|g_gpu - g_ref|
    <= 1e-4 max|g_ref|.  Returns the ratio of the parity scale built from s_i = sum_a |V_a||A_ia|
    to the one built from |u_i| (the gradient tolerance's reading of the precision remark), per
    component, for the record."""
    n = A.shape[1]
    n_factor = float(n if n_factor is None else n_factor)
    f_ref, g_ref, cf, cg, bad = oracle.nll_grad(A, V, Psi, n_factor=n_factor, with_cond=True)
    err = np.abs(g_gpu - g_ref)
    big = np.abs(g_ref) >= 1e-3 * np.max(np.abs(g_ref), axis=1, keepdims=True)
    assert np.all(err[big] <= 1e-4 * np.abs(g_ref[big])), (err[big] / np.abs(g_ref[big])).max()
    assert np.all(np.max(err, axis=1) <= 1e-4 * np.max(np.abs(g_ref), axis=1))
    A64 = A.astype(np.complex128)
    ratios = []
    for p in range(V.shape[0]):
        u = V[p].astype(np.complex128) @ A64
        scale_u = 2 * (np.abs(A64) @ (1.0 / np.abs(u))) + 2 * n_factor * (np.abs(V[p]) @ np.abs(Psi))
        ratios.append(cg[p] / scale_u)
    return np.array(ratios)


# ------------------------------------------------------------------- amplitudes ---------

@pytest.mark.parametrize("K,n,ld", [(4, 10_000, 10_000), (16, 4099, 4352), (7, 1, 2), (48, 3001, 3002)])
def test_amplitudes_parity(h, K, n, ld):
    ws = inputs.wave_set_plain(SEED + 1) if K == 4 else inputs.wave_set_spread(K, SEED + K)
    kin = inputs.kinematics(n, SEED + K, 6)
    from paper_1108_5882_gb300 import pwa
    A = torch.full((K, ld), complex(7, 7), dtype=torch.complex64, device="cuda")
    dM = torch.zeros((K, ld), dtype=torch.complex64, device="cuda")
    dW = torch.zeros((K, ld), dtype=torch.complex64, device="cuda")
    h.pwa_amplitudes(pwa.waves_from(ws), dev(padded(kin, ld)), n, A, dM, dW)
    Ag, dMg, dWg = (x.cpu().numpy() for x in (A, dM, dW))
    Ar, dMr, dWr = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin, derivs=True)
    assert np.max(np.abs(Ag[:, :n] - Ar)) <= 4e-6
    assert np.all(Ag[:, n:] == 0)  # padding columns zeroed
    for a in range(K):
        assert np.max(np.abs(dMg[a, :n] - dMr[a])) <= 2e-5 * np.max(np.abs(dMr[a]))
        assert np.max(np.abs(dWg[a, :n] - dWr[a])) <= 2e-5 * np.max(np.abs(dWr[a]))


def test_amplitudes_peak_and_all_spins(h):
    # every (J, lambda) the kernel supports, at the resonance peak and elsewhere
    from paper_1108_5882_gb300 import pwa
    waves = [(J, lam, 1.0 + 0.1 * J + 0.01 * (lam + 8), 0.05 + 0.01 * J) for J in range(9) for lam in (-8, -3, 0, 1, 8)]
    waves = waves[:64]
    K = len(waves)
    n = 2048
    kin = inputs.kinematics(n, SEED, 8)
    A = torch.zeros((K, n), dtype=torch.complex64, device="cuda")
    h.pwa_amplitudes(waves, dev(kin), n, A)
    J = [w[0] for w in waves]
    lam = [w[1] for w in waves]
    M = [w[2] for w in waves]
    W = [w[3] for w in waves]
    Ar = oracle.amplitudes(J, lam, M, W, kin)
    assert np.max(np.abs(A.cpu().numpy() - Ar)) <= 4e-6


@pytest.mark.parametrize("K,n,ld,m1,m2,R", [(5, 10_001, 10_002, 0.4937, 0.4937, 3.0),
                                             (16, 65_537, 65_540, 0.1396, 0.4937, 5.0),
                                             (64, 3_001, 3_004, 0.0, 0.0, 1.0), (3, 1, 2, 0.4937, 0.4937, 0.2)])
def test_amplitudes_barrier_parity(h, K, n, ld, m1, m2, R):
    # mass-dependent widths and Blatt-Weisskopf barrier factors (L = J <= 4) against the oracle,
    # with events below, at and just above the decay threshold
    ws = inputs.wave_set_spread(K, SEED + 60 + K)
    J = np.arange(K) % 5  # every L = J the barrier factors support
    waves = [(int(j), int(l), float(M), float(W)) for j, l, M, W in zip(J, ws.lam, ws.M, ws.W)]
    kin = inputs.kinematics(n, SEED + 60 + K, 6)
    thr = np.float32(m1 + m2)
    edge = np.array([0.5 * thr, thr, np.nextafter(thr, np.float32(9)), thr + np.float32(1e-3)], dtype=np.float32)
    if m1 + m2 > 0:  # (with massless daughters the threshold is m = 0, outside any phase space)
        kin[0, :min(n, 4)] = edge[:min(n, 4)]
    A = torch.full((K, ld), complex(7, 7), dtype=torch.complex64, device="cuda")
    h.pwa_amplitudes_barrier(waves, m1, m2, R, dev(padded(kin, ld)), n, A)
    Ag = A.cpu().numpy()
    Ar = oracle.amplitudes_barrier(J, ws.lam, ws.M, ws.W, m1, m2, R, kin)
    err = np.abs(Ag[:, :n] - Ar) / np.maximum(1.0, np.abs(Ar))
    assert np.max(err) <= 5e-6, np.max(err)
    assert np.all(Ag[:, n:] == 0)  # padding columns zeroed
    if m1 + m2 > 0 and n >= 4:
        # below threshold q = 0: only the J = 0 waves survive; at it they vanish like q^J
        assert np.all(Ag[J > 0, 0] == 0) and np.all(Ag[J == 0, 0] != 0)
        assert np.all(np.abs(Ag[J > 0, 1:3]) < 1e-3)


def test_amplitudes_barrier_reduce_to_the_fixed_width_kernel(h):
    # L = 0 with massless daughters: Gamma(m) = Gamma_0 and B_0 = 1, so both kernels compute
    # the fixed-width Breit-Wigner (to FP32 rounding)
    from paper_1108_5882_gb300 import pwa
    n = 20_000
    waves = [(0, lam, 1.2 + 0.2 * a, 0.05 + 0.05 * a) for a, lam in enumerate((0, 1, -1, 2, 0, 1))]
    kin = dev(inputs.kinematics(n, SEED + 61, 6))
    A1 = torch.zeros((6, n), dtype=torch.complex64, device="cuda")
    A2 = torch.zeros((6, n), dtype=torch.complex64, device="cuda")
    h.pwa_amplitudes(waves, kin, n, A1)
    h.pwa_amplitudes_barrier(waves, 0.0, 0.0, 2.0, kin, n, A2)
    assert torch.max(torch.abs(A1 - A2)).item() <= 4e-6


# ------------------------------------------------------------------- normalisation ------

@pytest.mark.parametrize("K,n_mc,weighted", [(4, 50_000, False), (16, 30_001, False), (32, 9_999, True),
                                             (5, 1, False), (48, 7_000, True), (64, 3_000, False)])
def test_normint_parity(h, K, n_mc, weighted):
    g = np.random.default_rng(K + n_mc)
    A = (g.normal(size=(K, n_mc)) + 1j * g.normal(size=(K, n_mc))).astype(np.complex64)
    ld = n_mc + (n_mc % 2) + 2
    w = g.uniform(0, 2, n_mc).astype(np.float32) if weighted else None
    if weighted:
        w[::7] = 0.0
    Psi = torch.zeros((K, K), dtype=torch.complex128, device="cuda")
    h.pwa_normint(dev(padded(A, ld, fill=np.complex64(np.nan))), n_mc, Psi, w=None if w is None else dev(w),
                  n_gen=1.5 * n_mc)
    ref = oracle.normint(A, w, n_gen=1.5 * n_mc)
    got = Psi.cpu().numpy()
    d = np.sqrt(np.outer(np.diag(ref).real, np.diag(ref).real))
    assert np.all(np.abs(got - ref) <= 1e-5 * d + 1e-300)
    assert np.array_equal(got, got.conj().T)


@pytest.mark.parametrize("K,n_mc,from_kin", [(16, 30_001, False), (32, 20_003, False), (16, 30_001, True),
                                              (32, 20_003, True), (7, 5_000, True), (8, 4_001, False),
                                              (24, 9_001, True)])
def test_normint_simt_path_forced(h, K, n_mc, from_kin, monkeypatch):
    # unit weights and 16 < K <= 32 take the tensor-core kernel by default; PWA_NORMINT_TC=1 / 0
    # force the tensor-core / FP32 SIMT kernel for any K <= 32: both within the same bound
    from paper_1108_5882_gb300 import pwa
    ws = inputs.wave_set_spread(K, SEED + 1500 + K)
    kin = inputs.kinematics(n_mc, SEED + 1500 + K, 5, ld=n_mc + (n_mc & 1))
    A = torch.zeros((K, kin.shape[1]), dtype=torch.complex64, device="cuda")
    h.pwa_amplitudes(pwa.waves_from(ws), dev(kin), n_mc, A)
    out = {}
    for tc in ("1", "0"):
        monkeypatch.setenv("PWA_NORMINT_TC", tc)
        Psi = torch.zeros((K, K), dtype=torch.complex128, device="cuda")
        if from_kin:
            h.pwa_normint_from_kinematics(pwa.waves_from(ws), dev(kin), n_mc, Psi)
        else:
            h.pwa_normint(A, n_mc, Psi)
        out[tc] = Psi.cpu().numpy()
    A_np = A.cpu().numpy()[:, :n_mc]
    ref = oracle.normint(A_np)
    d = np.sqrt(np.outer(np.diag(ref).real, np.diag(ref).real))
    m = np.abs(A_np).sum(axis=1) / n_mc
    tol = 1e-5 * d + (4e-6 * (m[:, None] + m[None, :]) if from_kin else 0.0) + 1e-30
    for tc in ("1", "0"):
        assert np.all(np.abs(out[tc] - ref) <= tol), (tc, np.max(np.abs(out[tc] - ref) / tol))
        assert np.array_equal(out[tc], out[tc].conj().T)
    assert h.pwa_sync_status() == pwa.PWA_OK


def test_normint_on_amplitudes_of_the_plain_workload(h):
    p = make_problem(4, 100, 50_000, SEED + 1, accept_reject=False, plain=True)
    Psi = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    h.pwa_normint(dev(p.A_mc), p.A_mc.shape[1], Psi)
    d = np.sqrt(np.outer(np.diag(p.Psi).real, np.diag(p.Psi).real))
    assert np.all(np.abs(Psi.cpu().numpy() - p.Psi) <= 1e-5 * d)


# ------------------------------------------------------------------- likelihood ---------

@pytest.mark.parametrize("K", [1, 3, 4, 8, 13, 16, 24, 32, 48, 64])
def test_nll_grad_single_set(h, K):
    # several tiles of the stream kernel plus a ragged (odd) tail
    n = 20_001
    p = make_problem(K, n, 4 * n, SEED + 100 + K, accept_reject=(K <= 16))
    V = p.V_true[None, :]
    ld = n + 1
    f, g = gpu_nll_grad(h, padded(p.A, ld), n, V, p.Psi)
    check_nll(f, g, p.A, V, p.Psi)
    f2, _ = gpu_nll_grad(h, padded(p.A, ld), n, V, p.Psi, grad=False)
    assert f2[0] == f[0] or abs(f2[0] - f[0]) <= 1e-12 * abs(f[0])


@pytest.mark.parametrize("variant", ["PWA_STREAM_HOLD=0", "PWA_STREAM_FUSED=0", "PWA_STREAM_TMA=1",
                                     "PWA_STREAM_TMA=0", "PWA_STREAM_HOLD=0,PWA_STREAM_FUSED=0"])
@pytest.mark.parametrize("K", [4, 16, 32, 64])
def test_nll_grad_single_set_variants(h, K, variant, monkeypatch):
    # the single-set kernels besides the default, forced: the amplitudes reloaded for the
    # gradient pass instead of held in registers (HOLD=0), the grid reduction finalised by a
    # second launch instead of the last block (FUSED=0), the bulk-copy staged kernel (TMA=1, the
    # default for 16 < K <= 32) and the register kernel (TMA=0); ragged tail, NaN padding never
    # read, several blocks
    for kv in variant.split(","):
        k, v = kv.split("=")
        monkeypatch.setenv(k, v)
    n = 20_001
    p = make_problem(K, n, 2 * n, SEED + 200 + K, accept_reject=False)
    ld = n + 3
    for V in (p.V_true[None, :], inputs.starts(1, K, SEED + 201)):
        f, g = gpu_nll_grad(h, padded(p.A, ld, fill=np.complex64(np.nan)), n, V, p.Psi)
        check_nll(f, g, p.A, V, p.Psi)
        f2, _ = gpu_nll_grad(h, padded(p.A, ld, fill=np.complex64(np.nan)), n, V, p.Psi, grad=False)
        assert abs(f2[0] - f[0]) <= 1e-12 * abs(f[0])


def test_plain_workload_at_random_starts(h):
    # plain workload: K=4, N_data=1e4, N_MC=5e4, data by accept-reject, one set per launch
    p = make_problem(4, 10_000, 50_000, SEED + 1, plain=True)
    ratios = []
    for V in inputs.starts(8, 4, SEED + 1):
        f, g = gpu_nll_grad(h, p.A, p.n, V[None, :], p.Psi)
        check_nll(f, g, p.A, V[None, :], p.Psi)
        ratios.append(check_plain_gradient(g, p.A, V[None, :], p.Psi))
    r = np.concatenate(ratios).ravel()
    print(f"plain workload: s_i / |u_i| gradient scale ratio median {np.median(r):.2f}, max {r.max():.2f}")


@pytest.mark.parametrize("K,P", [(4, 2), (8, 33), (16, 64), (16, 100), (32, 7), (32, 256), (48, 40), (64, 65)])
def test_nll_grad_batched(h, K, P):
    n = 6_337
    p = make_problem(K, n, 2 * n, SEED + 200 + K, accept_reject=False)
    V = inputs.starts(P, K, SEED + P)
    V[0] = p.V_true
    f, g = gpu_nll_grad(h, padded(p.A, n + 1), n, V, p.Psi)
    check_nll(f, g, p.A, V, p.Psi)


@pytest.mark.parametrize("K,P,n", [(4, 3, 3001), (8, 64, 40_001), (13, 100, 9_999), (16, 64, 20_000),
                                   (32, 256, 200_001), (32, 7, 1)])
def test_nll_grad_batched_pipelined_shape(h, K, P, n, monkeypatch):
    # the pipelined batched kernel (shape 3: 128-event tiles staged by bulk copies, K <= 32)
    # forced by the tuning override: ragged odd tails (NaN in the padding column), several
    # chunks and tiles per block, more tiles than the G flush window, P not a multiple of 64
    monkeypatch.setenv("PWA_BATCHED_SHAPE", "3")
    p = make_problem(K, n, max(2 * n, 1000), SEED + 700 + K, accept_reject=False)
    V = inputs.starts(P, K, SEED + P + 1)
    V[0] = p.V_true
    ld = n + 1 if n % 2 else n + 2
    f, g = gpu_nll_grad(h, padded(p.A, ld, fill=np.complex64(np.nan)), n, V, p.Psi)
    check_nll(f, g, p.A, V, p.Psi)
    f2, g2 = gpu_nll_grad(h, padded(p.A, ld), n, V, p.Psi)
    assert np.array_equal(f, f2) and np.array_equal(g, g2)


@pytest.mark.parametrize("K,P,n", [(4, 3, 3001), (8, 64, 40_001), (13, 130, 9_999), (16, 64, 20_000),
                                   (32, 256, 200_001), (32, 7, 1), (29, 300, 70_001), (24, 129, 33),
                                   (16, 100, 14_500), (8, 90, 21_800), (16, 64, 6_400)])
def test_nll_grad_batched_tensor_core_shape(h, K, P, n, monkeypatch):
    # the tensor-core kernel (shape 4: 3xTF32 products accumulated in FP32 in tensor memory,
    # 48-event tiles over four rotating tensor-memory regions, 128 sets per block) forced by the
    # tuning override: ragged odd tails (NaN in the padding column), one, two, three and many
    # tiles per block (the pipeline's start-up and end), more tiles than the double-single flush
    # interval, several blocks of sets with a partial last one, K padded to 8, 16 or 32 waves, and
    # more event chunks than the SIMT shapes' geometry (the workspace is sized for both)
    monkeypatch.setenv("PWA_BATCHED_SHAPE", "4")
    p = make_problem(K, n, max(2 * n, 1000), SEED + 900 + K, accept_reject=False)
    V = inputs.starts(P, K, SEED + P + 2)
    V[0] = p.V_true
    ld = n + 1 if n % 2 else n + 2
    f, g = gpu_nll_grad(h, padded(p.A, ld, fill=np.complex64(np.nan)), n, V, p.Psi)
    check_nll(f, g, p.A, V, p.Psi)
    f2, g2 = gpu_nll_grad(h, padded(p.A, ld), n, V, p.Psi)
    assert np.array_equal(f, f2) and np.array_equal(g, g2)
    f3, _ = gpu_nll_grad(h, padded(p.A, ld), n, V, p.Psi, grad=False)
    assert np.array_equal(f3, f)  # the -lnL pass without the gradient GEMM gives the same bits
    assert h.pwa_batched_shape(K, n, P) == 4


@pytest.mark.parametrize("K,n,weighted", [(4, 3001, False), (16, 100_003, True), (13, 257, False), (48, 9_999, True),
                                        (7, 1, False)])
def test_normint_from_kinematics(h, K, n, weighted):
    # Psi straight from the kinematics vs the oracle's Psi of the oracle's amplitudes, and vs
    # pwa_amplitudes + pwa_normint, within the Psi tolerance widened by the amplitudes' bound
    from paper_1108_5882_gb300 import pwa
    ws = inputs.wave_set_plain(SEED + 3) if K == 4 else inputs.wave_set_spread(K, SEED + 1300 + K)
    ld = n + 1 if n % 2 else n + 2
    kin = padded(inputs.kinematics(n, SEED + 1400 + K, 5), ld)
    w = np.random.default_rng(K).uniform(0, 2, size=n).astype(np.float32) if weighted else None
    Psi_k = torch.zeros((K, K), dtype=torch.complex128, device="cuda")
    h.pwa_normint_from_kinematics(pwa.waves_from(ws), dev(kin), n, Psi_k, w=None if w is None else dev(w),
                                  n_gen=1.5 * n)
    A = torch.zeros((K, ld), dtype=torch.complex64, device="cuda")
    h.pwa_amplitudes(pwa.waves_from(ws), dev(kin), n, A)
    Psi_a = torch.zeros((K, K), dtype=torch.complex128, device="cuda")
    h.pwa_normint(A, n, Psi_a, w=None if w is None else dev(w), n_gen=1.5 * n)
    A_ref = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin[:, :n]).astype(np.complex64)
    ref = oracle.normint(A_ref, w=w, n_gen=1.5 * n)
    d = np.sqrt(np.outer(np.abs(np.diag(ref)), np.abs(np.diag(ref))))
    # the amplitudes' own bound, |A_gpu - A_ref| <= 4e-6, carried through the sum:
    # |dPsi_ab| <= 4e-6 (m_a + m_b) with m_a = (1/n_gen) sum_j w_j |A_a(j)|
    wv = np.ones(n) if w is None else w.astype(np.float64)
    m = (np.abs(A_ref) * wv).sum(axis=1) / (1.5 * n)
    tol = 1e-5 * d + 4e-6 * (m[:, None] + m[None, :]) + 1e-30
    assert np.all(np.abs(Psi_k.cpu().numpy() - ref) <= tol)
    assert np.all(np.abs(Psi_k.cpu().numpy() - Psi_a.cpu().numpy()) <= tol)  # the unfused path


# the last three run several FP32 windows per block (two blocks per SM over whole tiles)
@pytest.mark.parametrize("K,n", [(4, 3001), (13, 20_001), (16, 100_000), (32, 9_999), (1, 1),
                                 (16, 1_000_003), (32, 300_001), (4, 5_000_001)])
def test_hessian_fumili_and_exact(h, K, n):
    p = make_problem(K, n, min(max(2 * n, 1000), 2_000_000), SEED + 1500 + K, accept_reject=False)
    ld = n + 1 if n % 2 else n + 2
    Ad = dev(padded(p.A, ld, fill=np.complex64(np.nan)))
    V = inputs.starts(1, K, SEED + 1600 + K)[0]
    for exact in (False, True):
        H = torch.zeros((2 * K, 2 * K), dtype=torch.float64, device="cuda")
        h.pwa_hessian(Ad, n, dev(V), dev(p.Psi), float(n), H, exact=exact)
        ref, cond, bad = oracle.hessian(p.A, V, p.Psi, n_factor=float(n), exact=exact, with_cond=True)
        assert bad == 0
        err = np.abs(H.cpu().numpy() - ref) / (cond + 1e-300)
        assert np.all(err <= 1e-5), (exact, err.max())
    assert h.pwa_sync_status() == 0


def test_hessian_flags_a_vanishing_intensity(h):
    from paper_1108_5882_gb300 import pwa
    A = np.zeros((2, 8), dtype=np.complex64)  # u_i = 0 for every event
    H = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    h.pwa_hessian(dev(A), 8, dev(np.array([1.0 + 0j, 0.5j], dtype=np.complex64)),
                  dev(np.eye(2, dtype=np.complex128)), 8.0, H)
    assert np.all(np.isnan(H.cpu().numpy()))
    assert h.pwa_sync_status() == pwa.PWA_ERR_NONFINITE


def _incoherent_problem(K, H, n, n_mc, seed):
    # state h: the amplitude model of a wave set of its own (J, lambda, M, Gamma drawn per state),
    # on the same events: A [K][H][n] and the MC normalisation summed over the states
    kin = inputs.kinematics(n, seed, 4)
    kin_mc = inputs.kinematics(n_mc, seed, 5)
    A = np.empty((K, H, n), dtype=np.complex64)
    A_mc = np.empty((K, H, n_mc), dtype=np.complex64)
    for st in range(H):
        ws = inputs.wave_set_spread(K, seed + 17 * st)
        A[:, st, :] = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin)
        A_mc[:, st, :] = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin_mc)
    return A, oracle.normint_incoherent(A_mc, n_gen=float(n_mc))


@pytest.mark.parametrize("K,H,n,P", [(4, 2, 3001, 1), (13, 3, 9_999, 3), (16, 2, 20_000, 2), (32, 4, 5001, 1),
                                     (7, 1, 1, 1), (64, 2, 2001, 1), (16, 4, 70_001, 1)])
def test_nll_grad_incoherent(h, K, H, n, P):
    A, Psi = _incoherent_problem(K, H, n, max(2 * n, 1000), SEED + 1100 + K)
    V = inputs.starts(P, K, SEED + 1200 + K)
    ld = n + 1 if n % 2 else n + 2
    Ap = np.full((K, H, ld), np.complex64(np.nan), dtype=np.complex64)  # padding never read
    Ap[:, :, :n] = A
    nll = torch.zeros(P, dtype=torch.float64, device="cuda")
    g = torch.zeros(P, 2 * K, dtype=torch.float64, device="cuda")
    h.pwa_nll_grad_incoherent(dev(Ap), n, dev(V), dev(Psi), float(n), nll, g)
    nll2 = torch.zeros(P, dtype=torch.float64, device="cuda")
    h.pwa_nll_grad_incoherent(dev(Ap), n, dev(V), dev(Psi), float(n), nll2)
    torch.cuda.synchronize()
    f_ref, g_ref, cf, cg, bad = oracle.nll_grad_incoherent(A, V, Psi, n_factor=float(n), with_cond=True)
    assert bad == 0
    f_gpu, g_gpu = nll.cpu().numpy(), g.cpu().numpy()
    assert np.all(np.abs(f_gpu - f_ref) / cf <= 1e-5), (np.abs(f_gpu - f_ref) / cf).max()
    assert np.all(np.abs(g_gpu - g_ref) / np.repeat(cg, 2, axis=1) <= 1e-4)
    assert np.array_equal(nll2.cpu().numpy(), f_gpu)  # the pass without the gradient: the same bits
    if H == 1:
        # one state: the coherent kernels' arithmetic on the same events, within the tolerance
        f1, g1 = gpu_nll_grad(h, padded(A[:, 0, :], ld), n, V, Psi)
        assert np.all(np.abs(f1 - f_gpu) / cf <= 2e-5)


def test_batched_equals_separate_sets(h):
    # per-set independence: P sets in one launch vs each set alone (within tolerance), and
    # permuting the sets permutes the outputs exactly
    p = make_problem(16, 5000, 10000, SEED + 300, accept_reject=False)
    V = inputs.starts(37, 16, SEED + 301)
    f, g = gpu_nll_grad(h, p.A, p.n, V, p.Psi)
    perm = np.random.default_rng(0).permutation(37)
    fp, gp = gpu_nll_grad(h, p.A, p.n, V[perm], p.Psi)
    assert np.array_equal(fp, f[perm]) and np.array_equal(gp, g[perm])
    for q in (0, 17, 36):
        f1, g1 = gpu_nll_grad(h, p.A, p.n, V[q:q + 1], p.Psi)
        _, _, cf, cg, _ = oracle.nll_grad(p.A, V[q:q + 1], p.Psi, with_cond=True)
        assert abs(f1[0] - f[q]) <= 2e-5 * cf[0]
        assert np.all(np.abs(g1[0] - g[q]) <= 2e-4 * np.repeat(cg[0], 2))


def test_deterministic_bitwise(h):
    p = make_problem(16, 30_000, 30_000, SEED + 400, accept_reject=False)
    for V in (p.V_true[None, :], inputs.starts(50, 16, 3)):
        a = gpu_nll_grad(h, p.A, p.n, V, p.Psi)
        b = gpu_nll_grad(h, p.A, p.n, V, p.Psi)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_gradient_sums_in_the_coarse_fixed_point_tier(h):
    # One parameter set: the grid sums are exact fixed point in two tiers, trunc(|x| 2^64) for
    # warp sums |x| < 2^61 and |x| 2^-37 above.  |V| = 1e-18 makes every event's gradient term
    # 1e18, so the warp sums of this sample (>= 32 events each) land in the coarse tier.  The
    # result must agree with the oracle, and the words must be clean for the next evaluation.
    K, n = 2, 40_000
    A = np.zeros((K, n), np.complex64)
    A[0] = 1.0
    A[1] = 0.5j * np.exp(1j * np.linspace(0, 6, n)).astype(np.complex64)
    Psi = oracle.normint((np.random.default_rng(2).normal(size=(K, 64)) + 0j).astype(np.complex64))
    p = make_problem(16, 20_000, 20_000, SEED + 510, accept_reject=False)
    V16 = p.V_true[None, :]
    before = gpu_nll_grad(h, p.A, p.n, V16, p.Psi)
    V = np.array([[1e-18, 3e-19 - 2e-19j]], np.complex64)
    f, g = gpu_nll_grad(h, A, n, V, Psi)
    check_nll(f, g, A, V, Psi)
    assert np.abs(g).max() > 2.0 ** 61 * 32
    after = gpu_nll_grad(h, p.A, p.n, V16, p.Psi)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])


def test_padding_is_never_read_as_events(h):
    # NaN in every padding column must not change the result
    p = make_problem(16, 9_999, 9_999, SEED + 500, accept_reject=False)
    V = inputs.starts(5, 16, 4)
    ld = 10_240
    a = gpu_nll_grad(h, padded(p.A, ld, fill=np.complex64(np.nan)), p.n, V, p.Psi)
    b = gpu_nll_grad(h, padded(p.A, ld), p.n, V, p.Psi)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    a1 = gpu_nll_grad(h, padded(p.A, ld, fill=np.complex64(np.nan)), p.n, V[:1], p.Psi)
    b1 = gpu_nll_grad(h, padded(p.A, ld), p.n, V[:1], p.Psi)
    assert np.array_equal(a1[0], b1[0]) and np.array_equal(a1[1], b1[1])


def test_empty_data_sample(h):
    # n = 0: only the normalisation term remains
    K = 5
    Psi = oracle.normint((np.random.default_rng(1).normal(size=(K, 100)) + 0j).astype(np.complex64))
    V = inputs.starts(3, K, 5)
    for P in (1, 3):
        f, g = gpu_nll_grad(h, np.zeros((K, 2), np.complex64), 0, V[:P], Psi, n_factor=7.0)
        fr, gr = oracle.nll_grad(np.zeros((K, 0), np.complex64), V[:P], Psi, n_factor=7.0)
        assert np.allclose(f, fr, rtol=1e-14, atol=1e-14) and np.allclose(g, gr, rtol=1e-14, atol=1e-14)


def test_zero_intensity_flags_the_set(h):
    from paper_1108_5882_gb300 import pwa
    p = make_problem(4, 1000, 1000, SEED + 600, accept_reject=False)
    A = p.A.copy()
    A[:, 123] = 0
    for P in (1, 4):
        V = inputs.starts(P, 4, 6)
        f, g = gpu_nll_grad(h, A, p.n, V, p.Psi)
        assert np.all(np.isinf(f)) and np.all(g == 0)
        assert h.pwa_sync_status() == pwa.PWA_ERR_NONFINITE
        assert h.pwa_sync_status() == pwa.PWA_OK  # read-and-clear
        # the flag does not leak into the next evaluation
        f2, _ = gpu_nll_grad(h, p.A, p.n, V, p.Psi)
        assert np.all(np.isfinite(f2))


def test_invalid_arguments_are_rejected(h):
    from paper_1108_5882_gb300 import pwa
    A = torch.zeros((4, 10), dtype=torch.complex64, device="cuda")
    V = torch.zeros((1, 4), dtype=torch.complex64, device="cuda")
    Psi = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    nll = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pwa.PWAError, match="ld"):
        h.pwa_nll(A, 11, V, Psi, 1.0, nll)  # n > ld
    A9 = torch.zeros((4, 9), dtype=torch.complex64, device="cuda")
    with pytest.raises(pwa.PWAError, match="even"):
        h.pwa_nll(A9, 9, V, Psi, 1.0, nll)
    with pytest.raises(pwa.PWAError, match="n_gen"):
        h.pwa_normint(A, 10, Psi, n_gen=0.0)
    with pytest.raises(pwa.PWAError, match="mass"):
        h.pwa_amplitudes([(0, 0, -1.0, 0.1)] * 4, torch.zeros((3, 10), device="cuda"), 10, A)
    A5 = torch.zeros((4, 5, 10), dtype=torch.complex64, device="cuda")  # H = 5 states > PWA_MAX_STATES
    with pytest.raises(pwa.PWAError, match="H = 5"):
        h.pwa_nll_grad_incoherent(A5, 10, V, Psi, 1.0, nll)
    with pytest.raises(pwa.PWAError, match="n_gen"):
        h.pwa_normint_from_kinematics([(0, 0, 1.5, 0.1)] * 4, torch.zeros((3, 10), device="cuda"), 10, Psi, n_gen=0.0)
    kin10 = torch.zeros((3, 10), device="cuda")
    with pytest.raises(pwa.PWAError, match="J = 5"):
        h.pwa_amplitudes_barrier([(5, 0, 1.5, 0.1)] * 4, 0.14, 0.14, 3.0, kin10, 10, A)
    with pytest.raises(pwa.PWAError, match="threshold"):
        h.pwa_amplitudes_barrier([(2, 0, 0.9, 0.1)] * 4, 0.4937, 0.4937, 3.0, kin10, 10, A)
    with pytest.raises(pwa.PWAError, match="radius"):
        h.pwa_amplitudes_barrier([(2, 0, 1.5, 0.1)] * 4, 0.4937, 0.4937, 0.0, kin10, 10, A)


# ------------------------------------------------------------------- full sizes ---------

def test_scale_workload_full_size(h):
    # K=16, N_data=1e6 in the launch configuration the benchmark times (one set per launch)
    K, n = 16, 1_000_000
    ws = inputs.wave_set_spread(K, SEED + 2)
    kin = inputs.kinematics(n, SEED + 2, 4)
    A = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin).astype(np.complex64)
    kin_mc = inputs.kinematics(200_000, SEED + 2, 5)
    Psi = oracle.normint(oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin_mc).astype(np.complex64))
    V = inputs.production_amplitudes(K, SEED + 2)[None, :]
    f, g = gpu_nll_grad(h, A, n, V, Psi)
    check_nll(f, g, A, V, Psi)
    # a random start: plain relative gradient error, and the two gradient scales compared
    V = inputs.starts(1, K, SEED + 2)
    f, g = gpu_nll_grad(h, A, n, V, Psi)
    check_nll(f, g, A, V, Psi)
    r = check_plain_gradient(g, A, V, Psi).ravel()
    print(f"scale workload: s_i / |u_i| gradient scale ratio median {np.median(r):.2f}, max {r.max():.2f}")


def test_multistart_workload_full_size_sampled(h):
    # K=32, N_data=2e6, P=256 in one launch; the oracle checks a sample of the starts
    K, n, P = 32, 2_000_000, 256
    ws = inputs.wave_set_spread(K, SEED + 3)
    kin = inputs.kinematics(n, SEED + 3, 4)
    A = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin).astype(np.complex64)
    kin_mc = inputs.kinematics(50_000, SEED + 3, 5)
    Psi = oracle.normint(oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin_mc).astype(np.complex64))
    V = inputs.starts(P, K, SEED + 3)
    f, g = gpu_nll_grad(h, A, n, V, Psi)
    # the autotuner's choice at this size is the tensor-core shape (FP32 products as three TF32
    # products), the shape the benchmark times; the samples below check that shape
    assert h.pwa_batched_shape(K, n, P) == 4
    for q in (0, 101, 255):
        check_nll(f[q:q + 1], g[q:q + 1], A, V[q:q + 1], Psi)
    # the FP32 SIMT shape the fitter evaluates with, forced, at the same size
    os.environ["PWA_BATCHED_SHAPE"] = "3"
    try:
        f3, g3 = gpu_nll_grad(h, A, n, V, Psi)
    finally:
        del os.environ["PWA_BATCHED_SHAPE"]
    for q in (7, 128, 254):
        check_nll(f3[q:q + 1], g3[q:q + 1], A, V[q:q + 1], Psi)


# ------------------------------------------------------------------- generator ----------

def test_generator_matches_oracle(h):
    # Candidates are bit-identical (the same Philox4x32-10 counters); every accept decision the
    # kernel takes differently from the FP64 oracle must lie inside the FP32 error band of I at
    # that candidate (fp32_decision_band), decision by decision.
    from paper_1108_5882_gb300 import pwa
    K = 16
    ws = inputs.wave_set_spread(K, SEED + 2)
    V = inputs.production_amplitudes(K, SEED + 2)
    V128 = V.astype(np.complex128)
    C = pwa.pwa_envelope(pwa.waves_from(ws), V)
    n_cand = 300_000
    kin_c, u, I, s = oracle.candidates(ws.J, ws.lam, ws.M, ws.W, V128, 77, 3, 1000, n_cand)
    assert np.max(I) <= C
    acc_ref = u.astype(np.float64) * C < I
    kin = torch.zeros((3, n_cand), dtype=torch.float32, device="cuda")
    na = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.pwa_generate(pwa.waves_from(ws), dev(V), 77, 3, 1000, n_cand, C, kin, n_cand, na)
    got_n = int(na.item())
    got = kin[:, :got_n].cpu().numpy()
    # every accepted event is one of the candidates, in candidate order
    index = {t: j for j, t in enumerate(map(tuple, kin_c.T.view(np.uint32).tolist()))}
    idx = np.array([index[t] for t in map(tuple, got.T.view(np.uint32).tolist())], dtype=np.int64)
    assert np.all(np.diff(idx) > 0)
    acc_gpu = np.zeros(n_cand, dtype=bool)
    acc_gpu[idx] = True
    differ = np.flatnonzero(acc_gpu != acc_ref)
    band = fp32_decision_band(V128, C, u, I, s, K)
    margin = np.abs(u.astype(np.float64) * C - I)
    assert np.all(margin[differ] <= band[differ]), (len(differ), (margin[differ] / band[differ]).max())
    # order: candidate order, identical geometry-independent prefix
    kin2 = torch.zeros((3, 100), dtype=torch.float32, device="cuda")
    h.pwa_generate(pwa.waves_from(ws), dev(V), 77, 3, 1000, n_cand, C, kin2, 100, na)
    assert torch.equal(kin2, kin[:, :100])