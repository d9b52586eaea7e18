"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds none of the likelihood arithmetic: it only draws the phase-space points,
wave sets, production amplitudes and starting values that the five workloads are defined on,
so that the CUDA library and the FP64 oracle can be fed identical inputs.  Every draw is keyed
by (seed, stream) through numpy's SeedSequence, so a given (seed, stream) gives the same
numbers on every machine.

Workloads (sizes and distributions; m_KK in GeV):
  plain       K=4  (J,lambda) = (0,0),(0,1),(2,0),(2,1); N_data=1e4, N_MC=5e4
  scale       K=16 J in {0,2,4} x lambda in {0,1}; masses spread over 1.3-2.8; N_data=1e6, N_MC=5e6
  multistart  K=32, N_data=2e6, N_MC=1e7, P=256 starts, |V0| U[0,2], arg V0 U[0,2pi)
  uneven      64 channels, K ~ U{4..48}, N_data log-U[1e4, 4e6], N_MC = 5 N_data
Phase space is flat: m_KK U[0.99, 3.0], cos(theta) U[-1, 1], phi U[0, 2pi).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

M_LO, M_HI = 0.99, 3.0
SEED_BASE = 11085882  # seed of workload k is SEED_BASE + k (k = 1..5)


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


@dataclass
class WaveSet:
    """K partial waves: spin J, helicity-like index lambda, resonance mass and width (GeV)."""
    J: np.ndarray      # int32 [K]
    lam: np.ndarray    # int32 [K]
    M: np.ndarray      # float64 [K]
    W: np.ndarray      # float64 [K]

    @property
    def K(self) -> int:
        return int(self.J.shape[0])


def wave_set_plain(seed: int) -> WaveSet:
    """K=4, J = 0,0,2,2 with lambda alternating 0,1 inside each equal-J pair; M U[1.3,2.3],
    Gamma U[0.05,0.3]."""
    g = rng(seed, 1)
    J = np.array([0, 0, 2, 2], dtype=np.int32)
    lam = np.array([0, 1, 0, 1], dtype=np.int32)
    M = g.uniform(1.3, 2.3, size=4)
    W = g.uniform(0.05, 0.3, size=4)
    return WaveSet(J, lam, M, W)


def wave_set_spread(K: int, seed: int, stream: int = 1) -> WaveSet:
    """(J, lambda) cycles over {0,2,4} x {0,1}; masses evenly spaced over [1.3, 2.8] with
    +-0.05 jitter; widths U[0.05, 0.3]."""
    g = rng(seed, stream)
    combos = [(j, l) for j in (0, 2, 4) for l in (0, 1)]
    J = np.array([combos[a % 6][0] for a in range(K)], dtype=np.int32)
    lam = np.array([combos[a % 6][1] for a in range(K)], dtype=np.int32)
    base = np.linspace(1.3, 2.8, K) if K > 1 else np.array([2.0])
    M = base + g.uniform(-0.05, 0.05, size=K)
    W = g.uniform(0.05, 0.3, size=K)
    return WaveSet(J, lam, M, W)


def kinematics(n: int, seed: int, stream: int, ld: int | None = None) -> np.ndarray:
    """Flat phase-space points as float32 SoA [3][ld] (m, cos theta, phi); columns >= n are
    zero padding."""
    g = rng(seed, stream)
    ld = n if ld is None else ld
    kin = np.zeros((3, ld), dtype=np.float32)
    kin[0, :n] = g.uniform(M_LO, M_HI, size=n)
    kin[1, :n] = g.uniform(-1.0, 1.0, size=n)
    kin[2, :n] = g.uniform(0.0, 2.0 * math.pi, size=n)
    # uniform() can round up to the open end in float32; keep phi in [0, 2pi)
    np.minimum(kin[2, :n], np.nextafter(np.float32(2.0 * math.pi), np.float32(0)), out=kin[2, :n])
    return kin


def accept_uniforms(n: int, seed: int, stream: int) -> np.ndarray:
    """float64 U[0,1) numbers for the accept-reject test of n candidate events."""
    return rng(seed, stream).random(n)


def production_amplitudes(K: int, seed: int, stream: int = 2, lo: float = 0.2,
                          hi: float = 2.0) -> np.ndarray:
    """A true V: |V_a| U[lo, hi], arg V_a U[0, 2pi), complex64 [K]."""
    g = rng(seed, stream)
    mod = g.uniform(lo, hi, size=K)
    ph = g.uniform(0.0, 2.0 * math.pi, size=K)
    return (mod * np.exp(1j * ph)).astype(np.complex64)


def starts(P: int, K: int, seed: int, stream: int = 3, hi: float = 2.0) -> np.ndarray:
    """P random starting vectors: |V| U[0, hi], arg V U[0, 2pi), complex64 [P][K]."""
    g = rng(seed, stream)
    mod = g.uniform(0.0, hi, size=(P, K))
    ph = g.uniform(0.0, 2.0 * math.pi, size=(P, K))
    return (mod * np.exp(1j * ph)).astype(np.complex64)


def uneven_channels(n_channels: int, seed: int, kmin: int = 4, kmax: int = 48,
                    nmin: float = 1e4, nmax: float = 4e6, mc_factor: int = 5):
    """(K_c, N_data_c, N_MC_c) for the uneven multi-fit workload: K ~ U{kmin..kmax},
    N_data log-uniform on [nmin, nmax], N_MC = mc_factor * N_data."""
    g = rng(seed, 7)
    K = g.integers(kmin, kmax + 1, size=n_channels)
    N = np.exp(g.uniform(math.log(nmin), math.log(nmax), size=n_channels)).astype(np.int64)
    return [(int(k), int(n), int(mc_factor * n)) for k, n in zip(K, N)]


def pad_to(n: int, mult: int = 256) -> int:
    return ((n + mult - 1) // mult) * mult


def bf16_bits(x) -> np.ndarray:
    """float32 values -> bfloat16 bit patterns (uint16), rounding to nearest even."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    return ((b + 0x7FFF + lsb) >> 16).astype(np.uint16)


def mlp_weights(dims, seed: int, stream: int = 21):
    """He-initialised weights W_l [out][in] (float32) and zero biases for layer sizes dims."""
    g = rng(seed, stream)
    Ws, bs = [], []
    for i in range(len(dims) - 1):
        Ws.append((g.normal(size=(dims[i + 1], dims[i])) * math.sqrt(2.0 / dims[i])).astype(np.float32))
        bs.append(np.zeros(dims[i + 1], dtype=np.float32))
    return Ws, bs
