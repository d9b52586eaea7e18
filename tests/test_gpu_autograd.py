"""The autograd.Function around the hand-written adjoint: its gradient must equal PyTorch's own
autograd of a plain FP64 torch expression of Eq. 3 (checks the complex-gradient convention),
for one and for several parameter sets, through a downstream chain rule."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1108_5882_gb300 import inputs
from problems import make_problem

pytestmark = pytest.mark.gpu


def _torch_nll(V64, A64, Psi, n_factor):
    u = V64 @ A64  # [P][n]
    I = u.real ** 2 + u.imag ** 2
    S = torch.real(torch.einsum("pa,ab,pb->p", V64, Psi, V64.conj()))
    return -torch.log(I).sum(dim=1) + n_factor * S


@pytest.mark.parametrize("K,P", [(4, 1), (16, 1), (8, 5)])
def test_autograd_gradient_matches_torch_fp64(K, P):
    from paper_1108_5882_gb300 import autograd, build
    build.build()
    n = 3000
    p = make_problem(K, n, 2 * n, inputs.SEED_BASE + 70 + K, accept_reject=False, plain=(K == 4))
    A = torch.from_numpy(p.A).cuda()
    Psi = torch.from_numpy(p.Psi).cuda()
    V0 = inputs.starts(P, K, 11)
    V = torch.from_numpy(V0).cuda().requires_grad_(True)
    w = torch.arange(1, P + 1, dtype=torch.float64, device="cuda")  # downstream chain rule
    f = autograd.nll(V if P > 1 else V[0], A, n, Psi)
    loss = (w * f).sum() if P > 1 else 3.0 * f
    loss.backward()
    V64 = torch.from_numpy(V0.astype(np.complex128)).cuda().requires_grad_(True)
    f_ref = _torch_nll(V64, A.to(torch.complex128), Psi, float(n))
    loss_ref = (w * f_ref).sum() if P > 1 else 3.0 * f_ref[0]
    loss_ref.backward()
    _, _, cf, cg, _ = oracle.nll_grad(p.A, V0, p.Psi, with_cond=True)
    fr = f.detach().reshape(-1).cpu().numpy()
    assert np.all(np.abs(fr - f_ref.detach().cpu().numpy()) <= 1e-5 * cf)
    gg = V.grad.cpu().numpy().astype(np.complex128)
    gr = V64.grad.cpu().numpy()
    wts = w.cpu().numpy()[:, None] if P > 1 else 3.0
    scale = cg * wts
    assert np.all(np.abs(gg.real - gr.real) <= 1e-4 * scale)
    assert np.all(np.abs(gg.imag - gr.imag) <= 1e-4 * scale)


def test_shape_autograd_matches_oracle_and_finite_differences():
    # ShapeNLLFunction: -lnL with the masses and widths of two waves floating (Sec. 2), its
    # gradient in V and theta = (M_1, M_3, G_1, G_3) through a downstream chain rule, against
    # the oracle's analytic (V, theta) gradient (the parity tolerances of the shape tests) and
    # against FP64 central differences of the oracle objective computed from the kinematics.
    from test_gpu_shape import _scales

    from paper_1108_5882_gb300 import autograd, build, pwa
    build.build()
    K, n, n_mc = 6, 20_001, 40_000
    seed = inputs.SEED_BASE + 77
    ws = inputs.wave_set_spread(K, seed)
    kin = inputs.kinematics(n, seed, 4, ld=n + 1)
    kin_mc = inputs.kinematics(n_mc, seed, 5)
    fwave, fkind = [1, 3, 1, 3], [0, 0, 1, 1]
    theta0 = np.array([ws.M[1] * 1.01, ws.M[3] * 0.99, ws.W[1] * 1.05, ws.W[3] * 0.97])
    ev = autograd.ShapeEvaluator(pwa.waves_from(ws), torch.from_numpy(kin).cuda(), n, torch.from_numpy(kin_mc).cuda(),
                                 n_mc, fwave, fkind)
    V0 = inputs.production_amplitudes(K, seed)
    V = torch.from_numpy(V0).cuda().requires_grad_(True)
    theta = torch.from_numpy(theta0).cuda().requires_grad_(True)
    f = autograd.nll_shape(V, theta, ev)
    (2.5 * f).backward()
    # oracle at the same theta, from its own FP64 amplitudes rounded to complex64
    M, W = ws.M.copy(), ws.W.copy()
    for q, (r, k) in enumerate(zip(fwave, fkind)):
        (M if k == 0 else W)[r] = theta0[q]
    kin_n = np.ascontiguousarray(kin[:, :n])
    A, dM, dW = oracle.amplitudes(ws.J, ws.lam, M, W, kin_n, derivs=True)
    Am, dMm, dWm = oracle.amplitudes(ws.J, ws.lam, M, W, kin_mc, derivs=True)
    dA = np.stack([(dM if k == 0 else dW)[r] for r, k in zip(fwave, fkind)]).astype(np.complex64)
    dAm = np.stack([(dMm if k == 0 else dWm)[r] for r, k in zip(fwave, fkind)]).astype(np.complex64)
    A, Am = A.astype(np.complex64), Am.astype(np.complex64)
    f_ref, gV, gS, bad = oracle.nll_grad_shape(A, dA, Am, dAm, fwave, V0, n_factor=n)
    assert bad == 0
    cf, cgV, cgS = _scales(A, dA, Am, dAm, fwave, V0.astype(np.complex128), n, n_mc, None)
    assert abs(f.item() - f_ref) <= 1e-5 * max(abs(f_ref), cf)
    gv = V.grad.cpu().numpy().astype(np.complex128) / 2.5
    assert np.all(np.abs(gv.real - gV[0::2]) <= 1e-4 * cgV) and np.all(np.abs(gv.imag - gV[1::2]) <= 1e-4 * cgV)
    gt = theta.grad.cpu().numpy() / 2.5
    assert np.all(np.abs(gt - gS) <= 1e-4 * cgS)

    # central differences of the FP64 objective straight from the kinematics
    def obj(Mx, Wx, Vx):
        return oracle.nll_shape_from_kin(ws.J, ws.lam, Mx, Wx, kin_n, kin_mc, Vx.astype(np.complex128), n_factor=n)

    for q, (r, k) in enumerate(zip(fwave, fkind)):
        hq = 1e-6 * theta0[q]
        Mp, Wp, Mm, Wm = M.copy(), W.copy(), M.copy(), W.copy()
        (Mp if k == 0 else Wp)[r] += hq
        (Mm if k == 0 else Wm)[r] -= hq
        fd = (obj(Mp, Wp, V0) - obj(Mm, Wm, V0)) / (2 * hq)
        assert abs(gt[q] - fd) <= 1e-4 * cgS[q], (q, gt[q], fd)
    for a in (0, 4):
        for unit, comp in ((1.0, gv.real), (1j, gv.imag)):
            hv = 1e-6
            Vp, Vm = V0.astype(np.complex128).copy(), V0.astype(np.complex128).copy()
            Vp[a] += hv * unit
            Vm[a] -= hv * unit
            fd = (obj(M, W, Vp) - obj(M, W, Vm)) / (2 * hv)
            assert abs(comp[a] - fd) <= 1e-4 * cgV[a], (a, comp[a], fd)
