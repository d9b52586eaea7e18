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
