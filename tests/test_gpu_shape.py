"""Floating masses and widths (Sec. 2: amplitudes recomputed each iteration, streamed MC
normalisation): pwa_nll_grad_shape against the FP64 oracle, and pwa_fit_shape_batch fits of
several uneven channels whose results are oracle-stationary points in (V, M, Gamma)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1108_5882_gb300 import inputs
from problems import accept_reject_data

pytestmark = pytest.mark.gpu
SEED = inputs.SEED_BASE + 4


@pytest.fixture(scope="module")
def h():
    from paper_1108_5882_gb300 import build, pwa
    build.build()
    return pwa.Handle(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _scales(A, dA, Am, dAm, fwave, V, n_f, n_gen, w):
    """Condition scales (sums of magnitudes of the terms) of f, grad_V and grad_shape."""
    A, dA, Am, dAm = (x.astype(np.complex128) for x in (A, dA, Am, dAm))
    u, um = V @ A, V @ Am
    I, Im = np.abs(u) ** 2, np.abs(um) ** 2
    w = np.ones(Am.shape[1]) if w is None else w.astype(np.float64)
    sc = n_f / n_gen
    cf = max(np.sum(np.abs(np.log(I))), sc * np.sum(w * Im))
    cgV = 2 * (np.abs(A) @ (np.abs(u) / I)) + 2 * sc * (np.abs(Am) @ (w * np.abs(um)))
    cgS = np.array([2 * np.abs(V[r]) * (np.abs(dA[q]) @ (np.abs(u) / I)) + 2 * sc * np.abs(V[r]) * (np.abs(dAm[q]) @ (w * np.abs(um)))
                    for q, r in enumerate(fwave)])
    return cf, cgV, cgS


@pytest.mark.parametrize("K,weighted", [(6, False), (24, True), (48, False)])
def test_nll_grad_shape_parity(h, K, weighted):
    ws = inputs.wave_set_spread(K, SEED + K)
    n, n_mc = 20_001, 50_000
    kin, kin_mc = inputs.kinematics(n, SEED + K, 4), inputs.kinematics(n_mc, SEED + K, 5)
    A, dM, dW = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin, derivs=True)
    Am, dMm, dWm = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin_mc, derivs=True)
    fwave = [1, 3, 1, 3]
    dA = np.stack([dM[1], dM[3], dW[1], dW[3]]).astype(np.complex64)
    dAm = np.stack([dMm[1], dMm[3], dWm[1], dWm[3]]).astype(np.complex64)
    A, Am = A.astype(np.complex64), Am.astype(np.complex64)
    w = np.random.default_rng(K).uniform(0, 2, n_mc).astype(np.float32) if weighted else None
    V = inputs.production_amplitudes(K, SEED + K)
    ld = n + 1
    nll = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(2 * K + 4, dtype=torch.float64, device="cuda")
    pad = lambda x: np.concatenate([x, np.full((x.shape[0], ld - n), np.nan, np.complex64)], axis=1)
    h.pwa_nll_grad_shape(dev(pad(A)), dev(pad(dA)), n, dev(Am), dev(dAm), n_mc, fwave, dev(V), float(n), nll, grad,
                         w_mc=None if w is None else dev(w), n_gen=1.2 * n_mc)
    torch.cuda.synchronize()
    f, gV, gS, bad = oracle.nll_grad_shape(A, dA, Am, dAm, fwave, V, n_factor=n, w_mc=w, n_gen=1.2 * n_mc)
    assert bad == 0
    cf, cgV, cgS = _scales(A, dA, Am, dAm, fwave, V.astype(np.complex128), n, 1.2 * n_mc, w)
    g = grad.cpu().numpy()
    assert abs(nll.item() - f) <= 1e-5 * max(abs(f), cf)
    assert np.all(np.abs(g[:2 * K] - gV) <= 1e-4 * np.repeat(cgV, 2))
    assert np.all(np.abs(g[2 * K:] - gS) <= 1e-4 * cgS)


def _channel(K, n, seed):
    ws = inputs.wave_set_plain(seed) if K == 4 else inputs.wave_set_spread(K, seed)
    V = inputs.production_amplitudes(K, seed)
    kin = accept_reject_data(ws, V, n, seed)
    kin_mc = inputs.kinematics(4 * n, seed, 5)
    return ws, V, kin, kin_mc


@pytest.mark.parametrize("polar", [0, 1])
def test_shape_fits_of_uneven_channels(h, polar):
    from paper_1108_5882_gb300 import pwa
    chans = []
    meta = []
    for i, (K, n) in enumerate(((4, 20_000), (6, 40_000), (8, 15_000))):
        ws, V, kin, kin_mc = _channel(K, n, SEED + 100 + i)
        fwave, fkind = [0, 1, 0, 1], [0, 0, 1, 1]  # masses and widths of waves 0 and 1
        waves = pwa.waves_from(ws)
        start = [list(w) for w in waves]
        for r in (0, 1):
            start[r][2] *= 1.01  # mass +1 %
            start[r][3] *= 0.95  # width -5 %
        x_out = torch.zeros(2 * K + 4, dtype=torch.float64, device="cuda")
        chans.append(dict(waves=[tuple(s) for s in start], kin=dev(kin), n=n, kin_mc=dev(kin_mc), n_mc=4 * n,
                          n_gen=4 * n, n_factor=n, float_wave=fwave, float_kind=fkind,
                          V0=dev(V * 1.1), x_out=x_out))
        meta.append((ws, V, kin, kin_mc, fwave, fkind, x_out))
    res = h.pwa_fit_shape_batch(chans, pwa.fit_opts(max_iter=2000, polar=polar))
    for r, (ws, V, kin, kin_mc, fwave, fkind, x_out) in zip(res, meta):
        assert r["status"] == 0, r
        x = x_out.cpu().numpy()
        K = ws.K
        Vh = x[0:2 * K:2] + 1j * x[1:2 * K:2]
        M, W = ws.M.copy(), ws.W.copy()
        for q, (wv, kd) in enumerate(zip(fwave, fkind)):
            (M if kd == 0 else W)[wv] = x[2 * K + q]
        # oracle stationarity in (V, M, Gamma) from FP64 amplitudes recomputed at the result
        A, dM, dW = oracle.amplitudes(ws.J, ws.lam, M, W, kin, derivs=True)
        Am, dMm, dWm = oracle.amplitudes(ws.J, ws.lam, M, W, kin_mc, derivs=True)
        dA = np.stack([(dM if kd == 0 else dW)[wv] for wv, kd in zip(fwave, fkind)])
        dAm = np.stack([(dMm if kd == 0 else dWm)[wv] for wv, kd in zip(fwave, fkind)])
        f, gV, gS, bad = oracle.nll_grad_shape(A.astype(np.complex64), dA.astype(np.complex64),
                                               Am.astype(np.complex64), dAm.astype(np.complex64), fwave,
                                               Vh.astype(np.complex64), n_factor=kin.shape[1])
        n = kin.shape[1]
        gV[1] = 0.0
        assert np.max(np.abs(gV)) < 1e-4 * n and np.max(np.abs(gS)) < 1e-4 * n, (np.max(np.abs(gV)), gS)
        # the floating masses move back towards the truth (data drawn at the true masses)
        for q, (wv, kd) in enumerate(zip(fwave, fkind)):
            if kd == 0:
                assert abs(x[2 * K + q] - ws.M[wv]) < abs(1.01 * ws.M[wv] - ws.M[wv])


def test_shape_gradient_against_gpu_finite_differences(h):
    # d f / d M_r and d f / d Gamma_r from pwa_nll_grad_shape vs central differences of the GPU
    # objective itself, with the amplitudes recomputed by pwa_amplitudes at theta +- h
    from paper_1108_5882_gb300 import pwa
    K, n, n_mc = 6, 30_000, 60_000
    ws = inputs.wave_set_spread(K, SEED + 500)
    V = inputs.production_amplitudes(K, SEED + 500)
    kin = dev(inputs.kinematics(n, SEED + 500, 4))
    kin_mc = dev(inputs.kinematics(n_mc, SEED + 500, 5))
    Vd = dev(V)
    nll = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(2 * K + 2, dtype=torch.float64, device="cuda")

    def objective(waves, with_grad=False):
        A = torch.zeros((K, n), dtype=torch.complex64, device="cuda")
        Am = torch.zeros((K, n_mc), dtype=torch.complex64, device="cuda")
        dM = torch.zeros((K, n), dtype=torch.complex64, device="cuda")
        dW = torch.zeros((K, n), dtype=torch.complex64, device="cuda")
        dMm = torch.zeros((K, n_mc), dtype=torch.complex64, device="cuda")
        dWm = torch.zeros((K, n_mc), dtype=torch.complex64, device="cuda")
        h.pwa_amplitudes(waves, kin, n, A, dM, dW)
        h.pwa_amplitudes(waves, kin_mc, n_mc, Am, dMm, dWm)
        dA = torch.stack([dM[2], dW[2]]).contiguous()
        dAm = torch.stack([dMm[2], dWm[2]]).contiguous()
        h.pwa_nll_grad_shape(A, dA, n, Am, dAm, n_mc, [2, 2], Vd, float(n), nll, grad)
        torch.cuda.synchronize()
        return nll.item(), grad.cpu().numpy().copy()

    waves = pwa.waves_from(ws)
    f0, g0 = objective(waves)
    for q, field in ((0, 2), (1, 3)):  # mass, width of wave 2
        step = 1e-4
        wp = [list(w) for w in waves]
        wm = [list(w) for w in waves]
        wp[2][field] += step
        wm[2][field] -= step
        fp, _ = objective([tuple(w) for w in wp])
        fm, _ = objective([tuple(w) for w in wm])
        fd = (fp - fm) / (2 * step)
        analytic = g0[2 * K + q]
        # f ~ 1e5 is evaluated in FP32 per event: its rounding noise (~1e-3 absolute) / step
        # bounds the FD error, far below the gradient's scale
        assert abs(fd - analytic) <= 2e-3 * max(abs(analytic), 1e3) + 50.0, (q, fd, analytic)
