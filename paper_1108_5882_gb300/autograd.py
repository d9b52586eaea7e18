"""torch.autograd.Function wrappers around the hand-written adjoints of -lnL.

NLLFunction (pwa_nll_grad): forward evaluates the extended -lnL of Eq. 3 (Sec. 2; footnote 2)
for P parameter sets on the GPU; backward returns the analytic gradient the same launch
produced.  PyTorch's convention for a real loss of a complex leaf is grad = dL/dRe V +
i dL/dIm V, which is exactly g_c = 2 dF/dconj(V_c) as returned by the library, so backward is
grad_out * g (no conjugation).

ShapeNLLFunction (pwa_amplitudes + pwa_nll_grad_shape): the same objective when resonance
masses and widths float (Sec. 2: the amplitudes are recomputed for every (M, Gamma) and the MC
normalisation is summed anew), differentiable in V and in the floating masses and widths theta.
Forward recomputes every amplitude of data and MC at the current theta, and the derivative rows
dA/dtheta_q of the floating ones, then evaluates -lnL with its gradient in (V, theta) in one
call; backward scales that gradient by grad_out.
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


class ShapeNLLFunction(torch.autograd.Function):
    """nll = ShapeNLLFunction.apply(V, theta, ev, handle)

    V: complex64 [K] (requires_grad); theta: float64 [F] (requires_grad), the current value of
    floating parameter q (a mass if float_kind[q] == 0, else a width) of wave float_wave[q];
    ev: a ShapeEvaluator holding the kinematics and work buffers.  Returns a float64 scalar."""

    @staticmethod
    def forward(ctx, V, theta, ev, handle):
        g = ev.evaluate(handle, V.detach().contiguous(), theta.detach())
        K = ev.K
        ctx.save_for_backward(torch.view_as_complex(g[:2 * K].view(K, 2)), g[2 * K:])
        return ev.nll[0].clone()

    @staticmethod
    def backward(ctx, gout):
        gc, gt = ctx.saved_tensors
        gV = (gc * gout.to(gc.dtype)).to(torch.complex64)
        return gV, gt * gout, None, None


class ShapeEvaluator:
    """Data and MC kinematics of one channel with floating masses and widths, and the amplitude
    buffers the floating-shape evaluation recomputes (device memory owned here).

    waves: [(J, lambda, M, Gamma)] starting table (the values of floating parameters are replaced
    by theta at every evaluation); kin, kin_mc: float32 [3][ld] CUDA; float_wave, float_kind: per
    floating parameter its wave and kind (0 mass, 1 width); w_mc optional float32 [n_mc]."""

    def __init__(self, waves, kin, n, kin_mc, n_mc, float_wave, float_kind, n_factor=None, n_gen=None, w_mc=None):
        self.waves = [tuple(w) for w in waves]
        self.K = len(self.waves)
        self.F = len(float_wave)
        assert len(float_kind) == self.F
        self.float_wave = [int(r) for r in float_wave]
        self.float_kind = [int(k) for k in float_kind]
        self.kin, self.kin_mc, self.n, self.n_mc = kin, kin_mc, int(n), int(n_mc)
        self.n_factor = float(n if n_factor is None else n_factor)
        self.n_gen = float(n_mc if n_gen is None else n_gen)
        self.w_mc = w_mc
        dev = kin.device
        ld, ld_mc = kin.shape[1], kin_mc.shape[1]
        F1 = max(self.F, 1)
        self.A = torch.zeros((self.K, ld), dtype=torch.complex64, device=dev)
        self.A_mc = torch.zeros((self.K, ld_mc), dtype=torch.complex64, device=dev)
        self.dA = torch.zeros((F1, ld), dtype=torch.complex64, device=dev)
        self.dA_mc = torch.zeros((F1, ld_mc), dtype=torch.complex64, device=dev)
        # a wave's derivative in the parameter that does not float lands in a scratch row
        self._spare = torch.zeros((1, ld), dtype=torch.complex64, device=dev)
        self._spare_mc = torch.zeros((1, ld_mc), dtype=torch.complex64, device=dev)
        self.nll = torch.zeros(1, dtype=torch.float64, device=dev)
        self.grad = torch.zeros(2 * self.K + self.F, dtype=torch.float64, device=dev)

    def table(self, theta_host):
        w = [list(x) for x in self.waves]
        for q, (r, k) in enumerate(zip(self.float_wave, self.float_kind)):
            w[r][2 + k] = float(theta_host[q])
        return [tuple(x) for x in w]

    def evaluate(self, handle, V, theta):
        """Amplitudes and derivative rows at theta, then -lnL and its gradient [2K + F] at V."""
        waves = self.table(theta.cpu().tolist())
        handle.pwa_amplitudes(waves, self.kin, self.n, self.A)
        handle.pwa_amplitudes(waves, self.kin_mc, self.n_mc, self.A_mc)
        for r in sorted(set(self.float_wave)):
            rows = {k: q for q, (rr, k) in enumerate(zip(self.float_wave, self.float_kind)) if rr == r}
            for A, dA, spare, kin, n in ((self.A, self.dA, self._spare, self.kin, self.n),
                                         (self.A_mc, self.dA_mc, self._spare_mc, self.kin_mc, self.n_mc)):
                dM = dA[rows[0]:rows[0] + 1] if 0 in rows else spare
                dW = dA[rows[1]:rows[1] + 1] if 1 in rows else spare
                handle.pwa_amplitudes([waves[r]], kin, n, A[r:r + 1], dM, dW)
        handle.pwa_nll_grad_shape(self.A, self.dA, self.n, self.A_mc, self.dA_mc, self.n_mc, self.float_wave, V,
                                  self.n_factor, self.nll, self.grad, w_mc=self.w_mc, n_gen=self.n_gen)
        return self.grad.clone()


def nll_shape(V, theta, ev, handle=None):
    """-lnL with floating masses and widths, differentiable in V (complex64 [K]) and theta
    (float64 [F]); ev a ShapeEvaluator."""
    h = handle if handle is not None else _default_handle(V.device)
    return ShapeNLLFunction.apply(V, theta, ev, h)


_handles: dict[int, pwa.Handle] = {}


def _default_handle(device) -> pwa.Handle:
    idx = device.index if device.index is not None else torch.cuda.current_device()
    if idx not in _handles:
        _handles[idx] = pwa.Handle(idx)
    return _handles[idx]
