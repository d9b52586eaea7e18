"""torch.autograd.Function around the hand-written adjoint of -lnL (pwa_nll_grad).

Forward evaluates the extended -lnL of Eq. 3 (Sec. 2; footnote 2) for P parameter sets on the
GPU; backward returns the analytic gradient the same launch produced.  PyTorch's convention for
a real loss of a complex leaf is grad = dL/dRe V + i dL/dIm V, which is exactly
g_c = 2 dF/dconj(V_c) as returned by the library, so backward is grad_out * g (no conjugation).
"""
from __future__ import annotations

import torch

from . import pwa


class NLLFunction(torch.autograd.Function):
    """nll = NLLFunction.apply(V, A, n, Psi, n_factor, handle)

    V: complex64 [P][K] (requires_grad), A: complex64 [K][ld], Psi: complex128 [K][K].
    Returns float64 [P]."""

    @staticmethod
    def forward(ctx, V, A, n, Psi, n_factor, handle):
        Vc = V.detach().contiguous()
        P, K = Vc.shape
        nll = torch.empty(P, dtype=torch.float64, device=V.device)
        g = torch.empty((P, 2 * K), dtype=torch.float64, device=V.device)
        handle.pwa_nll_grad(A, n, Vc, Psi, float(n_factor), nll, g)
        ctx.save_for_backward(torch.view_as_complex(g.view(P, K, 2)))
        return nll

    @staticmethod
    def backward(ctx, gout):
        (gc,) = ctx.saved_tensors
        gV = (gc * gout[:, None].to(gc.dtype)).to(torch.complex64)
        return gV, None, None, None, None, None


def nll(V, A, n, Psi, n_factor=None, handle=None):
    """-lnL for V [P][K] or [K] (complex64 CUDA tensor), differentiable in V."""
    h = handle if handle is not None else _default_handle(V.device)
    squeeze = V.dim() == 1
    V2 = V.unsqueeze(0) if squeeze else V
    out = NLLFunction.apply(V2, A, n, Psi, float(n if n_factor is None else n_factor), h)
    return out[0] if squeeze else out


_handles: dict[int, pwa.Handle] = {}


def _default_handle(device) -> pwa.Handle:
    idx = device.index if device.index is not None else torch.cuda.current_device()
    if idx not in _handles:
        _handles[idx] = pwa.Handle(idx)
    return _handles[idx]
