"""Seeded problem instances for the parity tests (test infrastructure).

Inputs come from paper_1108_5882_gb300.inputs; where the method itself is needed to build an
input (amplitudes, the accept-reject data sample, Psi), it is computed by the FP64 oracle and
rounded to the single-precision layout the GPU consumes, so the CUDA path never supplies an
oracle input.
"""
from dataclasses import dataclass

import numpy as np

import oracle
from paper_1108_5882_gb300 import inputs


@dataclass
class Problem:
    ws: inputs.WaveSet
    V_true: np.ndarray      # complex64 [K]
    kin_data: np.ndarray    # float32 [3][n]
    kin_mc: np.ndarray      # float32 [3][n_mc]
    A: np.ndarray           # complex64 [K][n]   (oracle amplitudes rounded to complex64)
    A_mc: np.ndarray        # complex64 [K][n_mc]
    Psi: np.ndarray         # complex128 [K][K]  (oracle normint of A_mc)

    @property
    def K(self):
        return self.ws.K

    @property
    def n(self):
        return self.A.shape[1]


def accept_reject_data(ws, V, n, seed, stream=11):
    """n events drawn by the oracle's accept-reject from I under V (Eq. 1)."""
    C = oracle.envelope(ws.M, ws.W, V.astype(np.complex128))
    out = []
    got = 0
    cand0 = 0
    step = max(4096, 40 * n)
    while got < n:
        kin, na, mr = oracle.generate(ws.J, ws.lam, ws.M, ws.W, V.astype(np.complex128), seed, stream, cand0, step,
                                      C, n - got)
        assert mr <= 1.0
        out.append(kin)
        got += kin.shape[1]
        cand0 += step
    return np.ascontiguousarray(np.concatenate(out, axis=1)[:, :n])


def make_problem(K, n, n_mc, seed, accept_reject=True, plain=False):
    ws = inputs.wave_set_plain(seed) if plain else inputs.wave_set_spread(K, seed)
    V = inputs.production_amplitudes(ws.K, seed)
    if accept_reject:
        kin = accept_reject_data(ws, V, n, seed)
    else:
        kin = inputs.kinematics(n, seed, 4)
    kin_mc = inputs.kinematics(n_mc, seed, 5)
    A = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin).astype(np.complex64)
    A_mc = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin_mc).astype(np.complex64)
    Psi = oracle.normint(A_mc)
    return Problem(ws, V, kin, kin_mc, A, A_mc, Psi)


def padded(a, ld, fill=0.0):
    """[rows][n] -> [rows][ld] with the padding columns set to `fill`."""
    out = np.full((a.shape[0], ld), fill, dtype=a.dtype)
    out[:, :a.shape[1]] = a
    return out


def polar_gradient(g, V):
    """d f / d rho_a, d f / d phi_a at V_a = rho_a exp(i phi_a) from the Cartesian gradient g
    (Re, Im interleaved).  Their magnitudes do not depend on which of the two polar
    representations (rho, phi), (-rho, phi + pi) of V_a is taken."""
    gre, gim = g[0::2], g[1::2]
    rho, phi = np.abs(V), np.angle(V)
    gr = gre * np.cos(phi) + gim * np.sin(phi)
    gp = rho * (gim * np.cos(phi) - gre * np.sin(phi))
    return gr, gp


def fp32_decision_band(V, C, unif, I, s, K):
    """Half-width of the band around the decision boundary unif * C = I inside which a single-
    precision generator may decide either way, per candidate (unif: the accept uniforms).  The
    kernel evaluates I from FP32 amplitudes (each within 4e-6 of the FP64 value, |A| <= 1: the
    amplitude parity bound), sums u = sum_a V_a A_a in FP32 (<= 2K + 2 roundings of terms bounded
    by s = sum_a |V_a||A_a|), squares it in FP32, and compares with unif * C in FP32 (C rounded to
    float, one rounding of the product)."""
    eps = 2.0 ** -24
    du = np.sum(np.abs(V)) * 4e-6 + (2 * K + 2) * eps * s
    dI = 2 * s * du + du * du + 2 * eps * s * s
    return dI + 2 * eps * unif.astype(np.float64) * C
