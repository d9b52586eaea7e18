"""Learned start proposer: an MLP maps the angular moments of a data sample to C candidate
production-amplitude vectors, used as fit starts instead of (or before) random ones.

The paper has no such part; it motivates it.  Fits are rerun from many random starts until
the lowest minimum is trusted to be global, and that grows costly as the parameter count rises
(Sec. 2, and Sec. 4 "Fits with large numbers of parameters").  The plain method (random
multi-start) stays the fallback and decides which minimum is global.

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
    """MLP with FP32 master weights, BF16 working copies and Adam state on the device.

    All parameters live in one flat FP32 buffer (weights and biases of every layer are views
    into it), and so do their gradients, the Adam moments and the BF16 copies, so one Adam
    launch updates the whole network.  train_step replays the forward pass, the loss and the
    backward pass as one captured CUDA graph (static input/target buffers of the batch size it
    was captured for), then takes the Adam step."""

    def __init__(self, handle: pwa.Handle, K: int = 16, C: int = 32, hidden=(256, 256, 256), n_feat: int = 1000,
                 seed: int = inputs.SEED_BASE + 5):
        self.h, self.K, self.C = handle, K, C
        self.dims = [n_feat, *hidden, C * 2 * K]
        Ws, bs = inputs.mlp_weights(self.dims, seed)
        sizes = []
        for w, b in zip(Ws, bs):
            sizes += [w.size, b.size]
        n = int(sum(sizes))
        self.P = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.G = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.M1 = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.M2 = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.Pb = torch.zeros(n, dtype=torch.bfloat16, device="cuda")
        self.W, self.b, self.Wb, self.gW, self.gb = [], [], [], [], []
        off = 0
        for w, b in zip(Ws, bs):
            shp = w.shape
            self.W.append(self.P[off:off + w.size].view(shp))
            self.Wb.append(self.Pb[off:off + w.size].view(shp))
            self.gW.append(self.G[off:off + w.size].view(shp))
            self.W[-1].copy_(torch.from_numpy(w))
            off += w.size
            self.b.append(self.P[off:off + b.size])
            self.gb.append(self.G[off:off + b.size])
            self.b[-1].copy_(torch.from_numpy(b))
            off += b.size
        self.Pb.copy_(self.P.to(torch.bfloat16))
        self.step = 0
        self._graph = None

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
        """Weight and bias gradients (into the flat gradient buffer) from d loss / d output."""
        B = dout.shape[0]
        L = len(self.W)
        dY = dout
        for i in reversed(range(L)):
            n_in, n_out = self.dims[i], self.dims[i + 1]
            if i < L - 1:
                self.h.pwa_mlp_relu_backward(acts[i + 1], dY)
            # dW[o][k] = sum_b dY[b][o] X[b][k]
            self.h.pwa_mlp_gemm(n_out, n_in, B, dY, (1, n_out), acts[i], (1, n_in), C=self.gW[i])
            self.h.pwa_mlp_bias_grad(dY, self.gb[i])
            if i > 0:
                dX = torch.empty((B, n_in), dtype=torch.float32, device="cuda")
                # dX[b][k] = sum_o dY[b][o] W[o][k]
                self.h.pwa_mlp_gemm(B, n_in, n_out, dY, (n_out, 1), self.Wb[i], (1, n_in), C=dX)
                dY = dX
        return self.gW, self.gb

    def _loss_and_grads(self, X, target, eps):
        acts, out = self.forward(X)
        B = X.shape[0]
        loss = torch.empty(B, dtype=torch.float32, device="cuda")
        dout = torch.empty_like(out)
        self.h.pwa_mlp_wta_loss(out, target, self.C, self.K, eps, loss, dout)
        self.backward(acts, dout)
        return loss

    def train_step(self, X, target, lr=1e-3, eps=0.05, graph=True):
        """One Adam step on the batch (X bf16 [B][n_feat], target fp32 [B][2K]); returns the
        per-sample loss (a view of a static buffer when graph=True)."""
        if graph:
            B = X.shape[0]
            if self._graph is None or self._graph_key != (B, eps):
                self._sX = torch.empty_like(X)
                self._sT = torch.empty_like(target)
                self._sX.copy_(X)
                self._sT.copy_(target)
                side = torch.cuda.Stream()
                side.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(side):  # warm-up outside the capture
                    self._loss_and_grads(self._sX, self._sT, eps)
                torch.cuda.current_stream().wait_stream(side)
                self._graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self._graph):
                    self._sLoss = self._loss_and_grads(self._sX, self._sT, eps)
                self._graph_key = (B, eps)
            self._sX.copy_(X)
            self._sT.copy_(target)
            self._graph.replay()
            loss = self._sLoss
        else:
            loss = self._loss_and_grads(X, target, eps)
        self.step += 1
        self.h.pwa_mlp_adam(self.P, self.G, self.M1, self.M2, self.Pb, lr, self.step)
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
        tot = torch.zeros((), dtype=torch.float64, device="cuda")
        nb = 0
        for b0 in range(0, T - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            loss = prop.train_step(X[idx].contiguous(), targets[idx].contiguous(), lr=lr)
            tot += loss.sum(dtype=torch.float64)  # stays on the device: no sync per step
            nb += 1
        history.append(float(tot) / max(nb * batch, 1))
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


def _single_fit(h, A, n_events, Psi, V0):
    """One start fitted alone (the stream-kernel path), timed; returns (result, seconds, V)."""
    K = A.shape[0]
    V_out = torch.empty((1, K), dtype=torch.complex128, device="cuda")
    t0 = time.perf_counter()
    r = h.pwa_fit_batch([dict(A=A, n=n_events, Psi=Psi, n_factor=n_events, V0=V0, V_out=V_out)])[0]
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0, V_out[0].cpu().numpy()


def _exact_f(h, A, n_events, Psi, V):
    """-lnL at V (complex [K]) by the single-set kernel, whose event sums are exact fixed point:
    the values a comparison at the 0.01 level needs from every fit alike (the batched tensor-core
    shape carries an offset of order n * 1e-6 common to all starts, harmless to its own fits)."""
    Vc = torch.from_numpy(np.asarray(V).astype(np.complex64)[None, :]).cuda()
    f = torch.empty(1, dtype=torch.float64, device="cuda")
    h.pwa_nll(A, n_events, Vc, Psi, float(n_events), f)
    return float(f.item())


def evaluate_toy(h, waves, Psi, prop, V_true, n_events, seed, stream, P_rand=256, max_seq=64, dlnl=0.01):
    """One held-out toy, four ways on the same data:
      batched random   P_rand random starts in one batched fit
      batched learned  the C proposed starts in one batched fit
      plain            random starts fitted one at a time until one reaches the global minimum
      learned ranked   the proposed starts ranked by -lnL at the start (one batched evaluation),
                       fitted one at a time in that order until one reaches the global minimum,
                       then random starts (the plain method as fallback)
    The global minimum is the lowest -lnL over every converged fit of the toy; a fit reaches it
    when its -lnL is within dlnl (Delta lnL < 0.01).  Every -lnL compared comes from the single-
    set kernel (the batched results are re-evaluated there once per distinct minimum).  The sequential methods stop on that
    criterion, so their times are measured, not modelled; the batched times are those of the
    whole batch."""
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
    # ---- batched learned and batched random
    t0 = time.perf_counter()
    cand = prop.propose(feat)[0].contiguous()
    V_out = torch.empty((prop.C, K), dtype=torch.complex128, device="cuda")
    res_l = h.pwa_fit_batch([dict(A=A, n=n_events, Psi=Psi, n_factor=n_events, V0=cand, V_out=V_out)])
    torch.cuda.synchronize()
    out["t_learned"] = time.perf_counter() - t0
    Vl = V_out.cpu().numpy()
    starts = torch.from_numpy(inputs.starts(P_rand + max_seq, K, seed, 50 + stream)).cuda()
    V_out2 = torch.empty((P_rand, K), dtype=torch.complex128, device="cuda")
    t0 = time.perf_counter()
    res_r = h.pwa_fit_batch([dict(A=A, n=n_events, Psi=Psi, n_factor=n_events, V0=starts[:P_rand].contiguous(),
                                  V_out=V_out2)])
    torch.cuda.synchronize()
    out["t_random"] = time.perf_counter() - t0
    Vr = V_out2.cpu().numpy()
    fs = [r["nll"] for r in res_l + res_r]
    oks = [r["status"] == 0 for r in res_l + res_r]
    Vs = [v for v in Vl] + [v for v in Vr]
    # the batched results' -lnL on the single-set kernel, once per distinct minimum, so that they
    # compare with the one-at-a-time fits below (bookkeeping of the decisions, not timed)
    reps, cid = cluster_minima(np.array(Vs), np.array(fs), np.array(oks))
    f_rep = [_exact_f(h, A, n_events, Psi, Vs[r]) for r in reps]
    fs = [f_rep[cid[i]] if oks[i] else fs[i] for i in range(len(fs))]
    f_best = min((f for f, o in zip(fs, oks) if o), default=float("inf"))

    # ---- plain: fresh random starts (not among the batched ones), one at a time
    seq_rand = starts[P_rand:]
    t_plain, n_plain, plain_hit = 0.0, 0, False
    iters_rand = []
    plain_stop = -1  # index into the solutions of the fit the plain method stopped on
    for j in range(max_seq):
        r, dt, V = _single_fit(h, A, n_events, Psi, seq_rand[j:j + 1].contiguous())
        t_plain += dt
        n_plain += 1
        iters_rand.append(r["iterations"])
        if r["status"] == 0:
            fs.append(r["nll"]); oks.append(True); Vs.append(V)
            f_best = min(f_best, r["nll"])
            if r["nll"] < f_best + dlnl:
                plain_hit = True
                plain_stop = len(fs) - 1
                break
    # ---- learned ranked: -lnL of every candidate in one batched evaluation, then in order
    t0 = time.perf_counter()
    cand = prop.propose(feat)[0].contiguous()
    f0 = torch.empty(prop.C, dtype=torch.float64, device="cuda")
    h.pwa_nll(A, n_events, cand, Psi, float(n_events), f0)
    order = torch.argsort(f0).cpu().numpy()
    t_rank = time.perf_counter() - t0
    t_lseq, n_lseq, lseq_hit, iters_learned, lseq_stop = t_rank, 0, False, [], -1
    queue = [cand[o:o + 1].contiguous() for o in order] + [seq_rand[j:j + 1].contiguous() for j in range(max_seq)]
    for V0 in queue[:prop.C + max_seq]:
        r, dt, V = _single_fit(h, A, n_events, Psi, V0)
        t_lseq += dt
        n_lseq += 1
        if n_lseq <= prop.C:
            iters_learned.append(r["iterations"])
        if r["status"] == 0:
            fs.append(r["nll"]); oks.append(True); Vs.append(V)
            f_best = min(f_best, r["nll"])
            if r["nll"] < f_best + dlnl:
                lseq_hit = True
                lseq_stop = len(fs) - 1
                break
    nl = prop.C
    fs_a, ok_a = np.array(fs), np.array(oks)
    reached = ok_a & (fs_a < f_best + dlnl)
    out.update(f_best=f_best, reached_learned=reached[:nl], reached_random=reached[nl:nl + P_rand],
               t_plain=t_plain, n_plain=n_plain, plain_hit=plain_hit,
               t_learned_seq=t_lseq, t_rank=t_rank, n_learned_seq=n_lseq, learned_seq_hit=lseq_hit,
               iters_first_random=iters_rand[0] if iters_rand else 0,
               iters_first_learned=iters_learned[0] if iters_learned else 0,
               plain_stop=plain_stop, learned_seq_stop=lseq_stop,
               n_learned=nl, n_random=P_rand, Vs=np.array(Vs), fs=fs_a, ok=ok_a, A=A, kin=kin,
               evals_learned=sum(r["evaluations"] for r in res_l), evals_random=sum(r["evaluations"] for r in res_r),
               iters_max_random=max(r["iterations"] for r in res_r),
               unconverged_random=sum(1 for r in res_r if r["status"] != 0))
    return out


def summarize(outs):
    """Per method: fraction of toys that reached the global minimum, per-start success rates,
    and the measured wall time to the global minimum per fit (mean over toys, and the median and
    maximum of the one-at-a-time methods, whose means a few slow toys can carry; the learned
    ranking step, the network's forward pass and the 32-set evaluation, is also given alone)."""
    m = lambda k: float(np.mean([o[k] for o in outs]))
    t_plain = m("t_plain")
    res = dict(toys=len(outs),
               learned_reaches_global=float(np.mean([np.any(o["reached_learned"]) for o in outs])),
               random_reaches_global=float(np.mean([np.any(o["reached_random"]) for o in outs])),
               per_start_success_learned=float(np.mean([np.mean(o["reached_learned"]) for o in outs])),
               per_start_success_random=float(np.mean([np.mean(o["reached_random"]) for o in outs])),
               plain_reached=m("plain_hit"), learned_sequential_reached=m("learned_seq_hit"),
               fits_to_global_plain=m("n_plain"), fits_to_global_learned_sequential=m("n_learned_seq"),
               iterations_first_start_random=m("iters_first_random"),
               iterations_first_start_learned=m("iters_first_learned"),
               time_to_global_plain_s=t_plain,
               time_to_global_learned_sequential_s=m("t_learned_seq"),
               time_to_global_batched_random_s=m("t_random"),
               time_to_global_batched_learned_s=m("t_learned"),
               time_to_global_plain_median_s=float(np.median([o["t_plain"] for o in outs])),
               time_to_global_learned_sequential_median_s=float(np.median([o["t_learned_seq"] for o in outs])),
               learned_ranking_time_mean_s=m("t_rank"),
               learned_ranking_time_max_s=float(np.max([o["t_rank"] for o in outs])),
               learned_sequential_time_max_s=float(np.max([o["t_learned_seq"] for o in outs])),
               plain_time_max_s=float(np.max([o["t_plain"] for o in outs])),
               batched_random_time_median_s=float(np.median([o["t_random"] for o in outs])),
               batched_random_time_max_s=float(np.max([o["t_random"] for o in outs])),
               batched_random_iterations_max=int(np.max([o["iters_max_random"] for o in outs])),
               toys_with_unconverged_random_start=int(sum(o["unconverged_random"] > 0 for o in outs)))
    for k in ("learned_sequential", "batched_random", "batched_learned"):
        res[f"speedup_{k}_vs_plain"] = t_plain / res[f"time_to_global_{k}_s"]
    return res


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
        o.pop("A")
        o.pop("kin")
        outs.append(o)
    summ = summarize(outs)
    summ.update(train_toys=args.train_toys, train_events=args.train_events, eval_events=args.eval_events,
                epochs=args.epochs, loss_first=hist[0], loss_last=hist[-1], t_generate_s=t_gen, t_train_s=t_train)
    print(json.dumps(summ))


if __name__ == "__main__":
    main()
