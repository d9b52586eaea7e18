"""FP64 reference of the learned start proposer's MLP pieces (plain numpy).

TEST INFRASTRUCTURE ONLY (tests, smoke, the benchmark's CPU leg).  Inputs in bfloat16 arrive as
uint16 bit patterns and are widened exactly to float64; every product and sum here is FP64 in
the order the formula states.

  linear(X, W, b, relu)          Y = X W^T + b (ReLU)
  linear_backward(...)           dX = (dY o mask) W, dW = (dY o mask)^T X, db = sum_b (dY o mask)
  wta_loss(out, target, C, K)    winner-takes-all phase-aligned distance and its gradient
  adam(p, g, m, v, ...)          one bias-corrected Adam step (Kingma and Ba)
"""
import numpy as np


def bf16_to_f64(u):
    u = np.ascontiguousarray(u, dtype=np.uint16)
    return (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def linear(X, W, b=None, relu=False):
    Y = X @ W.T
    if b is not None:
        Y = Y + b
    return np.maximum(Y, 0.0) if relu else Y


def linear_backward(X, W, Y, dY, relu=False):
    g = dY * (Y > 0) if relu else dY
    return g @ W, g.T @ X, g.sum(axis=0)


def wta_loss(out, target, C, K, eps):
    """out [B][C*2K], target [B][2K] (re, im pairs) -> loss [B], dout [B][C*2K], winner [B].
    d_c = |V_c|^2 + |T|^2 - 2 |sum_a conj(V_ca) T_a|; loss = (1-eps) min_c d_c + eps mean_c d_c;
    dout = gradient of mean_b loss."""
    B = target.shape[0]
    V = out.reshape(B, C, K, 2)
    Vc = V[..., 0] + 1j * V[..., 1]
    T = target.reshape(B, K, 2)
    Tc = T[..., 0] + 1j * T[..., 1]
    z = np.einsum("bca,ba->bc", np.conj(Vc), Tc)
    d = np.sum(np.abs(Vc) ** 2, axis=2) + np.sum(np.abs(Tc) ** 2, axis=1)[:, None] - 2 * np.abs(z)
    win = np.argmin(d, axis=1)
    loss = (1 - eps) * d[np.arange(B), win] + eps * d.mean(axis=1)
    w = np.full((B, C), eps / C)
    w[np.arange(B), win] += 1 - eps
    ph = np.where(np.abs(z) > 0, np.conj(z) / np.where(np.abs(z) > 0, np.abs(z), 1.0), 1.0)  # exp(-i arg z)
    g = 2 * (Vc - ph[:, :, None] * Tc[:, None, :]) * (w / B)[:, :, None]
    dout = np.stack([g.real, g.imag], axis=-1).reshape(B, C * 2 * K)
    return loss, dout, win


def adam(p, g, m, v, lr, b1, b2, eps, step):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
