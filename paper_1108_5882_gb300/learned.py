"""Learned start proposer: an MLP maps the angular moments of a data sample to C candidate
production-amplitude vectors, used as fit starts instead of (or before) random ones.

The paper has no such part; it motivates it.  Fits are repeated from many random starts to gain
confidence in the global minimum, which is "excessively time consuming" for many parameters
(Sec. 2, and Sec. 4 "Fits with large numbers of parameters").  The plain method (random
multi-start) stays the fallback and the judge.

Everything runs in the library's kernels:
  features    pwa_moments (data) / pwa_toy_moments (toys drawn on the fly, never stored)
  network     1000 -> 256 -> 256 -> 256 -> C*2K, BF16 weights and activations, FP32 accumulate
              (pwa_mlp_gemm forward and backward, pwa_mlp_relu_backward, pwa_mlp_bias_grad)
  loss        pwa_mlp_wta_loss: winner-takes-all over the C candidates of the distance after the
              optimal global phase, to targets V / sqrt(S(V)) (the scale a fit converges to)
  optimiser   pwa_mlp_adam
  evaluation  pwa_fit_batch from the proposed starts and from random starts on the same data
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import inputs, pwa

FEAT_SCALE = 100.0  # features (event averages of Y_LM per bin, ~1e-2) -> O(1) network inputs


class Proposer:
    """MLP with FP32 master weights, BF16 working copies and Adam state on the device."""

    def __init__(self, handle: pwa.Handle, K: int = 16, C: int = 32, hidden=(256, 256, 256), n_feat: int = 1000,
                 seed: int = inputs.SEED_BASE + 5):
        self.h, self.K, self.C = handle, K, C
        self.dims = [n_feat, *hidden, C * 2 * K]
        Ws, bs = inputs.mlp_weights(self.dims, seed)
        self.W = [torch.from_numpy(w).cuda() for w in Ws]
        self.b = [torch.from_numpy(b).cuda() for b in bs]
        self.Wb = [w.to(torch.bfloat16) for w in self.W]
        self.mW = [torch.zeros_like(w) for w in self.W]
        self.vW = [torch.zeros_like(w) for w in self.W]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.step = 0

    # ---------------------------------------------------------------- forward / backward
    def forward(self, X):
        """X bf16 [B][n_feat] -> (hidden activations bf16, output fp32 [B][C*2K])."""
        B = X.shape[0]
        acts = [X]
        L = len(self.W)
        out = None
        for i in range(L):
            n_in, n_out = self.dims[i], self.dims[i + 1]
            if i < L - 1:
                Y = torch.empty((B, n_out), dtype=torch.bfloat16, device="cuda")
                self.h.pwa_mlp_gemm(B, n_out, n_in, acts[-1], (n_in, 1), self.Wb[i], (n_in, 1), C_bf16=Y,
                                    bias=self.b[i], relu=True)
                acts.append(Y)
            else:
                out = torch.empty((B, n_out), dtype=torch.float32, device="cuda")
                self.h.pwa_mlp_gemm(B, n_out, n_in, acts[-1], (n_in, 1), self.Wb[i], (n_in, 1), C=out,
                                    bias=self.b[i], relu=False)
        return acts, out

    def backward(self, acts, dout):
        """Weight and bias gradients from d loss / d output (fp32 [B][C*2K])."""
        B = dout.shape[0]
        L = len(self.W)
        gW = [None] * L
        gb = [None] * L
        dY = dout
        for i in reversed(range(L)):
            n_in, n_out = self.dims[i], self.dims[i + 1]
            if i < L - 1:
                self.h.pwa_mlp_relu_backward(acts[i + 1], dY)
            gW[i] = torch.empty((n_out, n_in), dtype=torch.float32, device="cuda")
            gb[i] = torch.empty(n_out, dtype=torch.float32, device="cuda")
            # dW[o][k] = sum_b dY[b][o] X[b][k]
            self.h.pwa_mlp_gemm(n_out, n_in, B, dY, (1, n_out), acts[i], (1, n_in), C=gW[i])
            self.h.pwa_mlp_bias_grad(dY, gb[i])
            if i > 0:
                dX = torch.empty((B, n_in), dtype=torch.float32, device="cuda")
                # dX[b][k] = sum_o dY[b][o] W[o][k]
                self.h.pwa_mlp_gemm(B, n_in, n_out, dY, (n_out, 1), self.Wb[i], (1, n_in), C=dX)
                dY = dX
        return gW, gb

    def train_step(self, X, target, lr=1e-3, eps=0.05):
        acts, out = self.forward(X)
        B = X.shape[0]
        loss = torch.empty(B, dtype=torch.float32, device="cuda")
        dout = torch.empty_like(out)
        self.h.pwa_mlp_wta_loss(out, target, self.C, self.K, eps, loss, dout)
        gW, gb = self.backward(acts, dout)
        self.step += 1
        for i in range(len(self.W)):
            self.h.pwa_mlp_adam(self.W[i], gW[i], self.mW[i], self.vW[i], self.Wb[i], lr, self.step)
            self.h.pwa_mlp_adam(self.b[i], gb[i], self.mb[i], self.vb[i], None, lr, self.step)
        return loss

    def propose(self, feat):
        """feat float64 [B][1000] (device) -> candidate V complex64 [B][C][K]."""
        B = feat.shape[0]
        X = torch.empty((B, self.dims[0]), dtype=torch.bfloat16, device="cuda")
        self.h.pwa_mlp_to_bf16(feat.contiguous(), X, FEAT_SCALE)
        _, out = self.forward(X)
        return torch.view_as_complex(out.view(B, self.C, self.K, 2).contiguous())


# ---------------------------------------------------------------- training data
def flat_psi(h, waves, n_mc=2_000_000, seed=inputs.SEED_BASE + 5):
    """Psi over the flat phase space (the mean intensity S(V) = V^T Psi V* of pwa_toy_moments)."""
    K = len(waves)
    kin = torch.from_numpy(inputs.kinematics(n_mc, seed, 31)).cuda()
    A = torch.empty((K, n_mc), dtype=torch.complex64, device="cuda")
    h.pwa_amplitudes(waves, kin, n_mc, A)
    Psi = torch.empty((K, K), dtype=torch.complex128, device="cuda")
    h.pwa_normint(A, n_mc, Psi)
    return Psi


def random_truths(T, K, seed, stream=41):
    """Production amplitudes of the training/held-out toys: |V| U[0.2, 2], arg V U[0, 2pi)."""
    g = inputs.rng(seed, stream)
    mod = g.uniform(0.2, 2.0, size=(T, K))
    ph = g.uniform(0.0, 2.0 * math.pi, size=(T, K))
    return (mod * np.exp(1j * ph)).astype(np.complex64)


def normalised_targets(h, V, Psi):
    """V / sqrt(S(V)) as float32 [T][2K]: the scale an extended-likelihood fit converges to."""
    Vd = torch.from_numpy(V).cuda()
    T, K = V.shape
    # S(V) through the library: -lnL with no data events is exactly n_factor * S(V)
    nll = torch.empty(T, dtype=torch.float64, device="cuda")
    A0 = torch.zeros((K, 2), dtype=torch.complex64, device="cuda")
    h.pwa_nll(A0, 0, Vd, Psi, 1.0, nll)
    S = nll.cpu().numpy()
    Vn = V / np.sqrt(S)[:, None]
    return torch.from_numpy(np.stack([Vn.real, Vn.imag], axis=-1).reshape(T, 2 * K).astype(np.float32)).cuda()


def make_training_set(h, waves, Psi, T, n_events, seed, chunk=4096):
    """Features (float64 [T][1000]) and normalised targets of T toys of ~n_events each."""
    K = len(waves)
    V = random_truths(T, K, seed)
    feats = torch.empty((T, 1000), dtype=torch.float64, device="cuda")
    nacc = torch.empty(T, dtype=torch.int64, device="cuda")
    for t0 in range(0, T, chunk):
        t1 = min(T, t0 + chunk)
        h.pwa_toy_moments(waves, torch.from_numpy(V[t0:t1]).cuda(), Psi, n_events, seed, 100_000 + t0,
                          feats[t0:t1], nacc[t0:t1])
    return feats, normalised_targets(h, V, Psi), V, nacc


def train(prop, feats, targets, epochs=20, batch=256, lr=1e-3, seed=0, log=None):
    T = feats.shape[0]
    X = torch.empty((T, 1000), dtype=torch.bfloat16, device="cuda")
    prop.h.pwa_mlp_to_bf16(feats.contiguous(), X, FEAT_SCALE)
    g = np.random.default_rng(seed)
    history = []
    for ep in range(epochs):
        perm = torch.from_numpy(g.permutation(T)).cuda()
        tot = 0.0
        nb = 0
        for b0 in range(0, T - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            loss = prop.train_step(X[idx].contiguous(), targets[idx].contiguous(), lr=lr)
            tot += float(loss.mean())
            nb += 1
        history.append(tot / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4f}")
    return history


# ---------------------------------------------------------------- evaluation
def gauge(V):
    """Rotate so that V_0 is real and non-negative (the likelihood ignores a global phase)."""
    V = np.asarray(V, dtype=np.complex128)
    ph = np.angle(V[..., :1])
    return V * np.exp(-1j * ph)


def cluster_minima(Vs, fs, ok, tol=1e-4):
    """Group converged solutions by gauge-fixed V (max-norm distance < tol * max |V|).
    Returns representative indices ordered by f and the cluster id of every solution."""
    Vg = gauge(Vs)
    order = [i for i in np.argsort(fs) if ok[i]]
    reps, cid = [], np.full(len(fs), -1)
    for i in order:
        for c, r in enumerate(reps):
            if np.max(np.abs(Vg[i] - Vg[r])) < tol * np.max(np.abs(Vg[r])):
                cid[i] = c
                break
        else:
            cid[i] = len(reps)
            reps.append(i)
    return reps, cid


def evaluate_toy(h, waves, Psi, prop, V_true, n_events, seed, stream, P_rand=256):
    """One held-out toy: fits from the proposed starts and from P_rand random starts.
    Returns a dict with per-method outcomes, times and the converged solutions."""
    K = len(waves)
    C = pwa.pwa_envelope(waves, V_true)
    kin = torch.zeros((3, n_events), dtype=torch.float32, device="cuda")
    na = torch.zeros(1, dtype=torch.int64, device="cuda")
    got, cand0, step = 0, 0, 1 << 25
    Vd = torch.from_numpy(V_true).cuda()
    while got < n_events:
        tmp = torch.zeros((3, n_events - got), dtype=torch.float32, device="cuda")
        h.pwa_generate(waves, Vd, seed, stream, cand0, step, C, tmp, n_events - got, na)
        k = min(int(na.item()), n_events - got)
        kin[:, got:got + k] = tmp[:, :k]
        got += k
        cand0 += step
    A = torch.empty((K, n_events), dtype=torch.complex64, device="cuda")
    h.pwa_amplitudes(waves, kin, n_events, A)
    feat = torch.empty((1, 1000), dtype=torch.float64, device="cuda")
    h.pwa_moments(kin, n_events, feat)
    torch.cuda.synchronize()
    out = {}
    t0 = time.perf_counter()
    cand = prop.propose(feat)[0].contiguous()
    V_out = torch.empty((prop.C, K), dtype=torch.complex128, device="cuda")
    res_l = h.pwa_fit_batch([dict(A=A, n=n_events, Psi=Psi, n_factor=n_events, V0=cand, V_out=V_out)])
    torch.cuda.synchronize()
    out["t_learned"] = time.perf_counter() - t0
    Vl = V_out.cpu().numpy()
    starts = torch.from_numpy(inputs.starts(P_rand, K, seed, 50 + stream)).cuda()
    V_out2 = torch.empty((P_rand, K), dtype=torch.complex128, device="cuda")
    t0 = time.perf_counter()
    res_r = h.pwa_fit_batch([dict(A=A, n=n_events, Psi=Psi, n_factor=n_events, V0=starts, V_out=V_out2)])
    torch.cuda.synchronize()
    out["t_random"] = time.perf_counter() - t0
    Vr = V_out2.cpu().numpy()
    # the plain method: one random start per fit (the stream kernel path), timed per fit
    V_out3 = torch.empty((1, K), dtype=torch.complex128, device="cuda")
    t0 = time.perf_counter()
    res_1 = h.pwa_fit_batch([dict(A=A, n=n_events, Psi=Psi, n_factor=n_events, V0=starts[:1].contiguous(),
                                  V_out=V_out3)])
    torch.cuda.synchronize()
    out["t_single"] = time.perf_counter() - t0
    out["single_status"] = res_1[0]["status"]
    Vs = np.concatenate([Vl, Vr])
    fs = np.array([r["nll"] for r in res_l + res_r])
    ok = np.array([r["status"] == 0 for r in res_l + res_r])
    reps, cid = cluster_minima(Vs, fs, ok)
    out.update(Vs=Vs, fs=fs, ok=ok, reps=reps, cid=cid, n_learned=prop.C, n_random=P_rand, A=A, kin=kin,
               evals_learned=sum(r["evaluations"] for r in res_l), evals_random=sum(r["evaluations"] for r in res_r))
    return out


def summarize(outs):
    """Per method: fraction of toys whose best start reached the global minimum (the best
    cluster of all converged starts) and per-start success rates."""
    hit_l, hit_r, q_l, q_r, tl, tr, ts = [], [], [], [], [], [], []
    for o in outs:
        if not o["reps"]:
            continue
        g = o["cid"] == 0
        nl = o["n_learned"]
        hit_l.append(bool(np.any(g[:nl])))
        hit_r.append(bool(np.any(g[nl:])))
        q_l.append(float(np.mean(g[:nl])))
        q_r.append(float(np.mean(g[nl:])))
        tl.append(o["t_learned"])
        tr.append(o["t_random"])
        ts.append(o.get("t_single", float("nan")))
    qr = float(np.mean(q_r))
    t1 = float(np.mean(ts))
    # plain method: one random start at a time until one reaches the global minimum; the
    # expected number of fits is 1/q for a per-start success rate q
    t_plain = t1 / qr if qr > 0 else float("inf")
    t_l, t_r = float(np.mean(tl)), float(np.mean(tr))
    ql = float(np.mean(q_l))
    # learned candidates used one at a time, like the plain method but in the network's order
    t_learned_seq = t1 / ql if ql > 0 else float("inf")
    return dict(toys=len(hit_l), learned_reaches_global=float(np.mean(hit_l)), random_reaches_global=float(np.mean(hit_r)),
                per_start_success_learned=float(np.mean(q_l)), per_start_success_random=qr,
                wall_s_per_fit_learned=t_l, wall_s_per_fit_random=t_r, wall_s_single_start_fit=t1,
                time_to_global_plain_s=t_plain, time_to_global_batched_s=t_r, time_to_global_learned_s=t_l,
                speedup_batched_vs_plain=t_plain / t_r, speedup_learned_vs_plain=t_plain / t_l,
                time_to_global_learned_sequential_s=t_learned_seq,
                speedup_learned_sequential_vs_plain=t_plain / t_learned_seq)


def main():
    ap = argparse.ArgumentParser(description="train the start proposer and compare with random starts")
    ap.add_argument("--train-toys", type=int, default=100_000)
    ap.add_argument("--train-events", type=int, default=200_000)
    ap.add_argument("--eval-toys", type=int, default=100)
    ap.add_argument("--eval-events", type=int, default=1_000_000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--random-starts", type=int, default=256)
    args = ap.parse_args()
    from . import build
    build.build()
    h = pwa.Handle(0)
    seed = inputs.SEED_BASE + 5
    ws = inputs.wave_set_spread(16, seed)
    waves = pwa.waves_from(ws)
    t0 = time.perf_counter()
    Psi = flat_psi(h, waves)
    feats, targets, _, _ = make_training_set(h, waves, Psi, args.train_toys, args.train_events, seed)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    prop = Proposer(h)
    t0 = time.perf_counter()
    hist = train(prop, feats, targets, epochs=args.epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    Vh = random_truths(args.eval_toys, 16, seed + 1)
    outs = []
    for t in range(args.eval_toys):
        o = evaluate_toy(h, waves, Psi, prop, Vh[t], args.eval_events, seed + 1, 7 + t, args.random_starts)
        for k in ("A", "kin"):
            o.pop(k)
        outs.append(o)
    summ = summarize(outs)
    summ.update(train_toys=args.train_toys, train_events=args.train_events, eval_events=args.eval_events,
                epochs=args.epochs, loss_first=hist[0], loss_last=hist[-1], t_generate_s=t_gen, t_train_s=t_train)
    print(json.dumps(summ))


if __name__ == "__main__":
    main()
