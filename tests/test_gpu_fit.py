"""Batched device-side fits (pwa_fit_batch) checked against the FP64 oracle.

A converged start must be a stationary point of the oracle's -lnL (oracle gradient small,
and S(V) = V^T Psi V* = 1, which the Euler identity forces at any stationary point); the best
minimum over the starts must match an independent minimiser (scipy L-BFGS-B on the oracle);
and a toy fit must recover the seeded production amplitudes within statistical error.  The
polar coordinates of V (Sec. 4, "Fits with complex parameters") must reach the same minima.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1108_5882_gb300 import inputs
from problems import accept_reject_data, make_problem, polar_gradient

pytestmark = pytest.mark.gpu
SEED = inputs.SEED_BASE


@pytest.fixture(scope="module")
def h():
    from paper_1108_5882_gb300 import build, pwa
    build.build()
    return pwa.Handle(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_fits(h, problems_and_starts, **opt):
    from paper_1108_5882_gb300 import pwa
    fits = []
    outs = []
    for p, V0 in problems_and_starts:
        out = torch.zeros(V0.shape, dtype=torch.complex128, device="cuda")
        outs.append(out)
        fits.append(dict(A=dev(p.A), n=p.n, Psi=dev(p.Psi), n_factor=float(p.n), V0=dev(V0), V_out=out))
    res = h.pwa_fit_batch(fits, pwa.fit_opts(**opt) if opt else None)
    torch.cuda.synchronize()
    return res, [o.cpu().numpy() for o in outs]


def stationary(p, V, gtol_rel=1e-5):
    Vf = V.astype(np.complex64)
    f, g = oracle.nll_grad(p.A, Vf[None, :], p.Psi)
    gc = g[0].copy()
    gc[1] = 0.0  # gauge component (Im V_0 frozen)
    S = float(np.real(Vf.astype(np.complex128) @ p.Psi @ np.conj(Vf.astype(np.complex128))))
    return f[0], np.max(np.abs(gc)) / p.n, S


def test_fit_plain_workload_starts(h):
    p = make_problem(4, 10_000, 50_000, SEED + 1, plain=True)
    V0 = inputs.starts(16, 4, SEED + 1)
    res, (V,) = run_fits(h, [(p, V0)])
    conv = [i for i, r in enumerate(res) if r["status"] == 0]
    assert len(conv) >= 12, [r["status"] for r in res]
    for i in conv:
        r = res[i]
        assert r["grad_max"] < 1e-6 * p.n
        f, gmax, S = stationary(p, V[i])
        assert gmax < 1e-5, gmax
        assert abs(S - 1.0) < 1e-4, S
        assert abs(f - r["nll"]) <= 1e-5 * max(abs(f), p.n)
        assert abs(V[i][0].imag) == 0.0 and V[i][0].real >= 0.0  # gauge fixed
    # independent minimiser on the oracle from a few of the same starts
    from scipy.optimize import minimize

    def fg(x):
        V = (x[0::2] + 1j * x[1::2])[None, :]
        f, g = oracle.nll_grad(p.A, V, p.Psi)
        return f[0], g[0]

    best_scipy = math.inf
    for i in range(4):
        x0 = np.empty(8)
        x0[0::2], x0[1::2] = V0[i].real, V0[i].imag
        r = minimize(fg, x0, jac=True, method="L-BFGS-B", options=dict(maxiter=5000, gtol=1e-9, ftol=1e-15))
        best_scipy = min(best_scipy, r.fun)
    best_gpu = min(res[i]["nll"] for i in conv)
    assert best_gpu <= best_scipy + 1e-6 * abs(best_scipy)


@pytest.mark.parametrize("shape", ["3", "4"])
def test_multistart_fit_with_each_batched_shape(h, shape, monkeypatch):
    # K = 32, 2e5 events, 64 starts per launch, with the pipelined FP32 SIMT shape and with the
    # tensor-core shape (FP32 products as three TF32 products, the sums drained from tensor memory
    # every 64 events) forced: the starts converge to oracle-stationary points with S = 1
    monkeypatch.setenv("PWA_BATCHED_SHAPE", shape)
    p = make_problem(32, 200_000, 400_000, SEED + 31, accept_reject=False)
    V0 = inputs.starts(64, 32, SEED + 31)
    res, (V,) = run_fits(h, [(p, V0)], max_iter=3000)
    bad = [(i, r) for i, r in enumerate(res) if r["status"] != 0]
    # the tensor-core shape's gradient error at a minimum (~4e-8 of the gradient scale) lets an
    # occasional start in a flat valley stall above the threshold (1 of these 64 at 2e5 events);
    # at the multistart size (2e6 events, 256 starts) every start converges with it
    assert len(bad) <= (0 if shape == "3" else 2), (len(bad), bad[:4])
    for i, r in enumerate(res):
        if r["status"] != 0:
            continue
        f, gmax, S = stationary(p, V[i])
        assert gmax < 1e-5, (i, gmax)
        assert abs(S - 1.0) < 1e-4, S
        assert abs(f - r["nll"]) <= 1e-5 * max(abs(f), p.n)


def test_toy_fit_recovers_seeded_amplitudes(h):
    # N = 1e5 events drawn from I under V_true; the fit from V_true's neighbourhood must land
    # within statistical error of V_true rescaled to S = 1 (the extended-likelihood scale) and
    # rotated to the gauge V_0 >= 0 real.
    K, N = 4, 100_000
    ws = inputs.wave_set_plain(SEED + 9)
    V_true = inputs.production_amplitudes(K, SEED + 9)
    kin = accept_reject_data(ws, V_true, N, SEED + 9)
    A = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin).astype(np.complex64)
    A_mc = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, inputs.kinematics(400_000, SEED + 9, 5)).astype(np.complex64)
    Psi = oracle.normint(A_mc)

    class Pr:
        pass
    p = Pr()
    p.A, p.Psi, p.n = A, Psi, N
    Vt = V_true.astype(np.complex128)
    Vt = Vt / math.sqrt(np.real(Vt @ Psi @ Vt.conj()))
    Vt = Vt * np.exp(-1j * np.angle(Vt[0]))
    starts = (Vt * (1 + 0.2 * inputs.starts(4, K, 3) / 2)).astype(np.complex64)
    res, (V,) = run_fits(h, [(p, starts)])
    best = int(np.argmin([r["nll"] for r in res]))
    assert res[best]["status"] == 0
    Vh = V[best]
    # covariance from the oracle Hessian (central differences of the analytic gradient) in the
    # real coordinates without the frozen gauge component Im V_0
    x = np.empty(2 * K)
    x[0::2], x[1::2] = Vh.real, Vh.imag
    free = [i for i in range(2 * K) if i != 1]
    H = np.zeros((len(free), len(free)))
    for a, i in enumerate(free):
        e = 1e-5 * max(1.0, abs(x[i]))
        xp, xm = x.copy(), x.copy()
        xp[i] += e
        xm[i] -= e
        gp = oracle.nll_grad(A, (xp[0::2] + 1j * xp[1::2])[None, :], Psi)[1][0]
        gm = oracle.nll_grad(A, (xm[0::2] + 1j * xm[1::2])[None, :], Psi)[1][0]
        H[a] = (gp - gm)[free] / (2 * e)
    H = 0.5 * (H + H.T)
    xt = np.empty(2 * K)
    xt[0::2], xt[1::2] = Vt.real, Vt.imag
    dx = (x - xt)[free]
    chi2 = float(dx @ H @ dx)  # ~ chi^2 with 7 degrees of freedom
    assert chi2 < 30.0, chi2
    pulls = dx / np.sqrt(np.diag(np.linalg.inv(H)))
    assert np.all(np.abs(pulls) < 5.0), pulls


def test_fit_scale_workload_single_start(h):
    p = make_problem(16, 200_000, 400_000, SEED + 2, accept_reject=False)
    V0 = inputs.starts(1, 16, SEED + 2)
    res, (V,) = run_fits(h, [(p, V0)])
    r = res[0]
    assert r["status"] == 0, r
    f, gmax, S = stationary(p, V[0])
    assert gmax < 1e-5 and abs(S - 1) < 1e-4


def test_multistart_and_uneven_fits_in_one_call(h):
    pa = make_problem(4, 5_000, 20_000, SEED + 20, accept_reject=True, plain=True)
    pb = make_problem(8, 20_000, 40_000, SEED + 21, accept_reject=False)
    pc = make_problem(32, 30_000, 60_000, SEED + 22, accept_reject=False)
    jobs = [(pa, inputs.starts(3, 4, 1)), (pb, inputs.starts(17, 8, 2)), (pc, inputs.starts(40, 32, 3))]
    res, Vs = run_fits(h, jobs, max_iter=3000)
    q = 0
    for (p, V0), V in zip(jobs, Vs):
        for i in range(V0.shape[0]):
            r = res[q]
            q += 1
            assert r["status"] in (0, 1), r
            if r["status"] == 0 and i % 5 == 0:
                f, gmax, S = stationary(p, V[i])
                assert gmax < 1e-5 and abs(S - 1) < 1e-4


def test_paused_starts_resume_as_a_dense_batch(h, monkeypatch):
    # a start pauses after its first backtrack (PWA_FIT_PAUSE_BACKTRACKS=1 instead of 10), so most
    # starts of three fits (tensor-core shape forced for the K=16 and K=32 fits) finish in the
    # precise phase, where only the resumed starts are evaluated: gathered from the fits' rows into
    # one dense batch per fit, on the FP32 SIMT shapes, and scattered back.  Every start must still
    # end at an oracle-stationary point with S = 1, the other fits' rows untouched by the batch.
    monkeypatch.setenv("PWA_FIT_PAUSE_BACKTRACKS", "1")
    monkeypatch.setenv("PWA_BATCHED_SHAPE", "4")
    pa = make_problem(4, 5_000, 20_000, SEED + 50, accept_reject=True, plain=True)
    pb = make_problem(16, 40_000, 80_000, SEED + 51, accept_reject=False)
    pc = make_problem(32, 60_000, 120_000, SEED + 52, accept_reject=False)
    jobs = [(pa, inputs.starts(5, 4, 11)), (pb, inputs.starts(23, 16, 12)), (pc, inputs.starts(70, 32, 13))]
    res, Vs = run_fits(h, jobs, max_iter=3000)
    q = 0
    for (p, V0), V in zip(jobs, Vs):
        for i in range(V0.shape[0]):
            r = res[q]
            q += 1
            assert r["status"] == 0, (q, r)
            f, gmax, S = stationary(p, V[i])
            assert gmax < 1e-5 and abs(S - 1) < 1e-4, (q, gmax, S)
            assert abs(f - r["nll"]) <= 1e-5 * max(abs(f), p.n)


def test_graph_and_eager_are_identical(h):
    p = make_problem(8, 8_000, 16_000, SEED + 30, accept_reject=False)
    V0 = inputs.starts(5, 8, 9)
    r1, (V1,) = run_fits(h, [(p, V0)], use_graph=1)
    r2, (V2,) = run_fits(h, [(p, V0)], use_graph=0)
    assert [r["nll"] for r in r1] == [r["nll"] for r in r2]
    assert np.array_equal(V1, V2)



@pytest.mark.parametrize("K,n,n_mc,P", [(4, 10_000, 50_000, 16), (16, 50_000, 100_000, 8)])
def test_polar_fits_end_at_minima_of_f(h, K, n, n_mc, P):
    p = make_problem(K, n, n_mc, SEED + 41 + K, plain=(K == 4), accept_reject=(K == 4))
    V0 = inputs.starts(P, K, SEED + 41 + K)
    rc, (Vc,) = run_fits(h, [(p, V0)], max_iter=3000)
    rp, (Vp,) = run_fits(h, [(p, V0)], max_iter=3000, polar=1)
    conv = [i for i, r in enumerate(rp) if r["status"] == 0]
    assert len(conv) >= P // 2, [r["status"] for r in rp]
    for i in conv:
        r = rp[i]
        assert r["grad_max"] < 1e-6 * p.n
        Vf = Vp[i].astype(np.complex64)
        f, g = oracle.nll_grad(p.A, Vf[None, :], p.Psi)
        gr, gp = polar_gradient(g[0], Vp[i])
        gp[0] = 0.0  # phi_0 frozen by the gauge
        assert max(np.max(np.abs(gr)), np.max(np.abs(gp))) < 1e-5 * p.n
        # a minimum of f itself, not only of its polar map (which is singular at rho_a = 0):
        # the Cartesian gradient of wave a is (gr_a, gp_a / rho_a) rotated by phi_a
        gc = g[0].copy()
        gc[1] = 0.0  # Im V_0, the same frozen direction at V_0 > 0
        ga = np.hypot(gc[0::2], gc[1::2])
        assert np.all(ga < 1e-5 * p.n * np.maximum(1.0, 1.0 / np.abs(Vp[i]))), ga
        S = float(np.real(Vf.astype(np.complex128) @ p.Psi @ np.conj(Vf.astype(np.complex128))))
        assert abs(S - 1.0) < 1e-4, S  # stationarity along every rho_a forces S = 1
        assert abs(f[0] - r["nll"]) <= 1e-5 * max(abs(f[0]), p.n)
        assert abs(Vp[i][0].imag) == 0.0 and Vp[i][0].real >= 0.0
    if K == 4:
        # few waves, data drawn from the model: the best start reaches the global minimum
        # (Delta lnL < 0.01) in both coordinate systems
        best_c = min(r["nll"] for r in rc if r["status"] == 0)
        best_p = min(rp[i]["nll"] for i in conv)
        assert abs(best_p - best_c) < 0.01, (best_p, best_c)
    # K = 16 on flat data has many local minima (Sec. 4, "Fits with large numbers of
    # parameters"): from the same start the two coordinate systems may end in different ones
    # (so do scipy's L-BFGS-B runs on the oracle in each system), so only minimality is checked.
