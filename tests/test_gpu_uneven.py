"""Many channels of uneven wave and event counts with floating masses and widths in one
persistent launch (pwa_nll_grad_uneven) and the multi-channel fitter built on it
(pwa_fit_shape_batch), against the FP64 oracle.

Parity per channel: f within 1e-5 and every gradient component (V and the floating masses and
widths) within 1e-4 of the sums of the magnitudes of their terms, the tolerances of the other
floating-shape tests; the kernel recomputes every amplitude from the kinematics, the oracle gets
its own FP64 amplitudes rounded to complex64.  Fits: every channel converges to a point where
the oracle's gradient in (V, M, Gamma) vanishes, and the kernel's gradient there matches FP64
central differences of the oracle objective computed straight from the kinematics."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1108_5882_gb300 import inputs
from problems import accept_reject_data
from test_gpu_shape import _scales

pytestmark = pytest.mark.gpu
SEED = inputs.SEED_BASE + 6


@pytest.fixture(scope="module")
def h():
    from paper_1108_5882_gb300 import build, pwa
    build.build()
    return pwa.Handle(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _oracle_channel(ws, M, W, kin, kin_mc, fwave, fkind, V, n_factor, n_gen, w_mc=None):
    """Oracle f, grad_V [2K], grad_theta [F] and their scales at masses M and widths W."""
    A, dM, dW = oracle.amplitudes(ws.J, ws.lam, M, W, kin, derivs=True)
    Am, dMm, dWm = oracle.amplitudes(ws.J, ws.lam, M, W, kin_mc, derivs=True)
    F = len(fwave)
    n, n_mc = kin.shape[1], kin_mc.shape[1]
    if F:
        dA = np.stack([(dM if k == 0 else dW)[r] for r, k in zip(fwave, fkind)]).astype(np.complex64)
        dAm = np.stack([(dMm if k == 0 else dWm)[r] for r, k in zip(fwave, fkind)]).astype(np.complex64)
    else:
        dA, dAm = np.zeros((0, n), np.complex64), np.zeros((0, n_mc), np.complex64)
    A, Am = A.astype(np.complex64), Am.astype(np.complex64)
    f, gV, gS, bad = oracle.nll_grad_shape(A, dA, Am, dAm, list(fwave), V, n_factor=n_factor, w_mc=w_mc, n_gen=n_gen)
    assert bad == 0
    if F:
        cf, cgV, cgS = _scales(A, dA, Am, dAm, fwave, V.astype(np.complex128), n_factor, n_gen, w_mc)
    else:
        cf, cgV, _ = _scales(A, np.zeros((1, n), np.complex64), Am, np.zeros((1, n_mc), np.complex64), [0],
                             V.astype(np.complex128), n_factor, n_gen, w_mc)
        cgS = np.zeros(0)
    return f, gV, gS, cf, cgV, cgS


# (K, n_data, n_mc, floating (wave, kind) pairs, MC weights, padding)
CHANNELS = [
    (4, 3_001, 9_001, [(0, 0), (1, 0), (0, 1), (1, 1)], False, 1),
    (7, 12_345, 30_000, [(2, 0), (5, 1)], True, 3),
    (13, 20_001, 41_000, [(0, 0), (3, 0), (0, 1), (3, 1)], False, 1),
    (16, 4_097, 12_288, [], False, 0),
    (21, 9_000, 27_001, [(20, 0), (20, 1)], False, 7),
    (33, 15_000, 30_000, [(1, 0), (8, 0), (1, 1), (8, 1)], True, 1),
    (40, 7_777, 20_000, [(39, 0), (0, 1)], False, 2),
    (48, 11_000, 33_000, [(10, 0), (11, 0), (10, 1), (11, 1)], False, 0),
]


def _build_channels(specs, seed):
    out = []
    for c, (K, n, n_mc, fl, weighted, pad) in enumerate(specs):
        ws = inputs.wave_set_spread(K, seed + c)
        kin = inputs.kinematics(n, seed + c, 4)
        kin_mc = inputs.kinematics(n_mc, seed + c, 5)
        ld, ld_mc = n + pad + ((n + pad) & 1), n_mc + ((n_mc) & 1)
        kin_p = np.full((3, ld), np.nan, np.float32)
        kin_p[:, :n] = kin
        kin_mc_p = np.full((3, ld_mc), np.nan, np.float32)
        kin_mc_p[:, :n_mc] = kin_mc
        w = np.random.default_rng(seed + c).uniform(0, 2, n_mc).astype(np.float32) if weighted else None
        fwave = [r for r, _ in fl]
        fkind = [k for _, k in fl]
        # theta: the floating masses and widths moved off the wave set's values
        theta = np.array([(ws.M[r] * 1.01 if k == 0 else ws.W[r] * 0.95) for r, k in fl], dtype=np.float64)
        V = inputs.production_amplitudes(K, seed + c)
        out.append(dict(ws=ws, kin=kin, kin_mc=kin_mc, kin_p=kin_p, kin_mc_p=kin_mc_p, w=w, fwave=fwave, fkind=fkind,
                        theta=theta, V=V, n=n, n_mc=n_mc, n_gen=1.25 * n_mc))
    return out


def _descs(chs):
    from paper_1108_5882_gb300 import pwa
    return [dict(waves=pwa.waves_from(c["ws"]), kin=dev(c["kin_p"]), n=c["n"], kin_mc=dev(c["kin_mc_p"]), n_mc=c["n_mc"],
                 n_gen=c["n_gen"], n_factor=float(c["n"]), w_mc=None if c["w"] is None else dev(c["w"]),
                 float_wave=c["fwave"], float_kind=c["fkind"]) for c in chs]


def _eval(h, descs, chs):
    V = dev(np.concatenate([c["V"] for c in chs]))
    th = np.concatenate([c["theta"] for c in chs])
    theta = dev(th) if th.size else None
    nll = torch.zeros(len(chs), dtype=torch.float64, device="cuda")
    ng = sum(2 * len(c["V"]) + len(c["fwave"]) for c in chs)
    grad = torch.zeros(ng, dtype=torch.float64, device="cuda")
    h.pwa_nll_grad_uneven(descs, V, theta, nll, grad)
    torch.cuda.synchronize()
    return nll.cpu().numpy(), grad.cpu().numpy()


def test_uneven_channels_match_the_oracle(h):
    chs = _build_channels(CHANNELS, SEED)
    descs = _descs(chs)
    f, g = _eval(h, descs, chs)
    f2, g2 = _eval(h, descs, chs)
    assert np.array_equal(f, f2) and np.array_equal(g, g2)  # deterministic: per-item slots, fixed order
    off = 0
    for i, c in enumerate(chs):
        K, F = len(c["V"]), len(c["fwave"])
        M, W = c["ws"].M.copy(), c["ws"].W.copy()
        for q, (r, k) in enumerate(zip(c["fwave"], c["fkind"])):
            (M if k == 0 else W)[r] = c["theta"][q]
        fr, gV, gS, cf, cgV, cgS = _oracle_channel(c["ws"], M, W, c["kin"], c["kin_mc"], c["fwave"], c["fkind"],
                                                   c["V"], float(c["n"]), c["n_gen"], c["w"])
        assert abs(f[i] - fr) <= 1e-5 * max(abs(fr), cf), (K, f[i], fr)
        gc = g[off:off + 2 * K + F]
        assert np.all(np.abs(gc[:2 * K] - gV) <= 1e-4 * np.repeat(cgV, 2)), (K, np.max(np.abs(gc[:2 * K] - gV) / np.repeat(cgV, 2)))
        assert np.all(np.abs(gc[2 * K:] - gS) <= 1e-4 * cgS), (K, gc[2 * K:], gS)
        off += 2 * K + F


def test_uneven_large_channel_and_a_vanishing_intensity(h):
    # a channel of 1e6 data events (many items, the final fixed-order sum over all of them) next
    # to a channel whose V is zero (I = 0: f = +inf, gradient zero, the others unaffected)
    from paper_1108_5882_gb300 import pwa
    specs = [(12, 1_000_000, 2_000_000, [(0, 0), (1, 0), (0, 1), (1, 1)], False, 0),
             (5, 2_000, 4_000, [(0, 0)], False, 0)]
    chs = _build_channels(specs, SEED + 50)
    chs[1]["V"] = np.zeros(5, np.complex64)
    f, g = _eval(h, _descs(chs), chs)
    assert f[1] == np.inf and np.all(g[2 * 12 + 4:] == 0)
    c = chs[0]
    M, W = c["ws"].M.copy(), c["ws"].W.copy()
    for q, (r, k) in enumerate(zip(c["fwave"], c["fkind"])):
        (M if k == 0 else W)[r] = c["theta"][q]
    fr, gV, gS, cf, cgV, cgS = _oracle_channel(c["ws"], M, W, c["kin"], c["kin_mc"], c["fwave"], c["fkind"], c["V"],
                                               float(c["n"]), c["n_gen"])
    assert abs(f[0] - fr) <= 1e-5 * max(abs(fr), cf)
    assert np.all(np.abs(g[:24] - gV) <= 1e-4 * np.repeat(cgV, 2))
    assert np.all(np.abs(g[24:28] - gS) <= 1e-4 * cgS)
    assert h.pwa_sync_status() == pwa.PWA_ERR_NONFINITE


def test_uneven_fits_reach_oracle_stationary_points(h):
    # eight channels, K from 4 to 48, one with 1e6 data events (the widest ones with enough events
    # for their ~100 parameters to be determined); each floats the masses and widths of two waves,
    # started 1 % (mass) and 5 % (width) off the values the data were drawn with;
    # one iteration of all channels is two launches (the persistent evaluation, the L-BFGS step)
    from paper_1108_5882_gb300 import pwa
    specs = [(4, 20_000), (9, 15_000), (16, 1_000_000), (21, 12_000), (27, 10_000), (34, 10_000), (41, 30_000),
             (48, 100_000)]
    chans, meta = [], []
    for i, (K, n) in enumerate(specs):
        seed = SEED + 300 + i
        ws = inputs.wave_set_spread(K, seed)
        V = inputs.production_amplitudes(K, seed)
        kin = accept_reject_data(ws, V, n, seed)
        n_mc = 2 * n
        kin_mc = inputs.kinematics(n_mc, seed, 5)
        # the masses and widths of the two interior resonances with the largest couplings; a weakly
        # produced wave, or one whose (J, lambda) neighbours can take over its shape, lets the fit
        # run into the narrow-spike direction of the likelihood (width -> 0 with |V| growing), a
        # property of the model, not of the fit
        inner = np.arange(K // 4, K - K // 4) if K >= 8 else np.arange(K)
        r0, r1 = sorted(inner[np.argsort(-np.abs(V[inner]))[:2]].tolist())
        fwave, fkind = [r0, r1, r0, r1], [0, 0, 1, 1]
        start = [list(w) for w in pwa.waves_from(ws)]
        for r in (r0, r1):
            start[r][2] *= 1.01
            start[r][3] *= 0.95
        x_out = torch.zeros(2 * K + 4, dtype=torch.float64, device="cuda")
        chans.append(dict(waves=[tuple(s) for s in start], kin=dev(kin), n=n, kin_mc=dev(kin_mc), n_mc=n_mc,
                          n_gen=n_mc, n_factor=n, float_wave=fwave, float_kind=fkind, V0=dev(V * 1.1), x_out=x_out))
        meta.append((ws, kin, kin_mc, fwave, fkind, x_out, [tuple(s) for s in start]))
    res = h.pwa_fit_shape_batch(chans, pwa.fit_opts(max_iter=20000, history=20))
    for r, (ws, kin, kin_mc, fwave, fkind, x_out, start) in zip(res, meta):
        print(f"K={ws.K} n={kin.shape[1]}: {r}")
    for r, (ws, kin, kin_mc, fwave, fkind, x_out, start) in zip(res, meta):
        assert r["status"] == 0, (ws.K, r)
        K, n = ws.K, kin.shape[1]
        x = x_out.cpu().numpy()
        Vh = (x[0:2 * K:2] + 1j * x[1:2 * K:2]).astype(np.complex64)
        M, W = ws.M.copy(), ws.W.copy()
        for q, (wv, kd) in enumerate(zip(fwave, fkind)):
            (M if kd == 0 else W)[wv] = x[2 * K + q]
        f, gV, gS, cf, cgV, cgS = _oracle_channel(ws, M, W, kin, kin_mc, fwave, fkind, Vh, float(n), float(2 * n))
        gV[1] = 0.0  # the frozen phase of V_0
        assert np.max(np.abs(gV)) < 1e-4 * n and np.max(np.abs(gS)) < 1e-4 * n, (K, np.max(np.abs(gV)), gS)
        # the kernel's gradient at the result against FP64 central differences of the oracle
        # objective (amplitudes recomputed from the kinematics at every point)
        desc = dict(waves=start, kin=dev(kin), n=n, kin_mc=dev(kin_mc), n_mc=2 * n, n_gen=float(2 * n), n_factor=float(n),
                    float_wave=fwave, float_kind=fkind)
        nll = torch.zeros(1, dtype=torch.float64, device="cuda")
        grad = torch.zeros(2 * K + 4, dtype=torch.float64, device="cuda")
        h.pwa_nll_grad_uneven([desc], dev(Vh), dev(x[2 * K:]), nll, grad)
        gk = grad.cpu().numpy()

        def obj(Mx, Wx, Vx):
            return oracle.nll_shape_from_kin(ws.J, ws.lam, Mx, Wx, kin, kin_mc, Vx.astype(np.complex128),
                                             n_factor=float(n), n_gen=float(2 * n))

        for q, (wv, kd) in enumerate(zip(fwave, fkind)):
            hq = 1e-6 * x[2 * K + q]
            Mp, Wp, Mm, Wm = M.copy(), W.copy(), M.copy(), W.copy()
            (Mp if kd == 0 else Wp)[wv] += hq
            (Mm if kd == 0 else Wm)[wv] -= hq
            fd = (obj(Mp, Wp, Vh) - obj(Mm, Wm, Vh)) / (2 * hq)
            assert abs(gk[2 * K + q] - fd) <= 1e-4 * cgS[q], (K, q, gk[2 * K + q], fd)
        for a in (0, K - 1):
            for unit, comp in ((1.0, 2 * a), (1j, 2 * a + 1)):
                Vp, Vm = Vh.astype(np.complex128), Vh.astype(np.complex128)
                Vp[a] += 1e-6 * unit
                Vm[a] -= 1e-6 * unit
                fd = (obj(M, W, Vp) - obj(M, W, Vm)) / 2e-6
                assert abs(gk[comp] - fd) <= 1e-4 * cgV[a], (K, a, gk[comp], fd)
