"""The learned-start comparison judged by the FP64 oracle (test infrastructure).

The learned part's figure of merit is the fraction of fits that reach the global minimum of a
toy (Delta lnL < 0.01) and the time to get there.  While it runs, the comparison (learned.py)
decides "reached" from the -lnL the GPU fits report, evaluated in single precision: at 1e6
events that value is only bounded to a few units, far above 0.01.  This module re-decides every
such decision with the oracle: for each held-out toy it takes the toy's events, computes the
oracle's own FP64 amplitudes and its normalisation integral over the same flat MC events the
GPU's Psi used, re-evaluates -lnL of every distinct converged minimum (solutions clustered by
gauge-fixed V) whose GPU value lies within F_MARGIN of the GPU's best, defines the global
minimum as the best oracle value, and marks a solution as reaching it when its oracle value is
within 0.01.  Minima farther than F_MARGIN (several times the FP32 evaluation's error bound) can
neither be the global minimum nor within 0.01 of it, so they are not re-evaluated.  The fits
stop at |grad|_inf < 1e-6 N, where the decrease left to a polish step is ~g^2 / H << 0.01, so
the minima are re-evaluated, not polished.

    python tests/learned_oracle_judge.py [--train-toys T] [--eval-toys E] [--json out.json]

runs the whole comparison (training included) and prints the GPU-decided and the
oracle-decided summaries side by side with the number of decisions that changed.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1108_5882_gb300 import inputs, learned  # noqa: E402

F_MARGIN = 10.0


def oracle_psi(ws, n_mc=2_000_000, seed=inputs.SEED_BASE + 5):
    """The oracle's Psi over the same flat MC events as learned.flat_psi."""
    kin = inputs.kinematics(n_mc, seed, 31)
    return oracle.normint(oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin).astype(np.complex64))


def judge_toy(o, ws, Psi_or, dlnl=0.01):
    """Oracle decisions for one toy of learned.evaluate_toy (which must keep "kin")."""
    kin = np.ascontiguousarray(o["kin"].cpu().numpy())
    n = kin.shape[1]
    A = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin).astype(np.complex64)
    Vs, fs, ok = o["Vs"], o["fs"], o["ok"]
    reps, cid = learned.cluster_minima(Vs, fs, ok)
    f_gpu_best = min(fs[r] for r in reps)
    close = [c for c, r in enumerate(reps) if fs[r] <= f_gpu_best + F_MARGIN]
    f_or, _ = oracle.nll_grad(A, np.stack([Vs[reps[c]] for c in close]), Psi_or, n_factor=float(n))
    f_rep = np.full(len(reps), np.inf)
    f_rep[close] = f_or
    f_best = float(np.min(f_or))
    reached = np.array([bool(ok[i]) and cid[i] >= 0 and f_rep[cid[i]] < f_best + dlnl for i in range(len(fs))])
    nl, nr = o["n_learned"], o["n_random"]
    gpu_choice = int(np.argmin([fs[r] for r in reps]))
    j = dict(f_best_oracle=f_best, f_best_gpu=float(o["f_best"]), n_minima=len(reps), n_reevaluated=len(close),
             global_cluster_same=bool(int(np.argmin(f_rep)) == gpu_choice),
             gpu_choice_is_global=bool(f_rep[gpu_choice] < f_best + dlnl),
             reached_learned=reached[:nl], reached_random=reached[nl:nl + nr],
             plain_hit=bool(o["plain_stop"] >= 0 and reached[o["plain_stop"]]),
             learned_seq_hit=bool(o["learned_seq_stop"] >= 0 and reached[o["learned_seq_stop"]]))
    j["changed_starts"] = int(np.sum(j["reached_learned"] != o["reached_learned"]) +
                              np.sum(j["reached_random"] != o["reached_random"]))
    j["changed_stops"] = int((j["plain_hit"] != o["plain_hit"]) + (j["learned_seq_hit"] != o["learned_seq_hit"]))
    return j


def summarize_judged(outs, judged):
    """The summary of learned.summarize with every "reached" decided by the oracle; a sequential
    method whose stopping fit the oracle does not place at the global minimum counts as a miss."""
    mod = []
    for o, j in zip(outs, judged):
        m = dict(o)
        m.update(reached_learned=j["reached_learned"], reached_random=j["reached_random"], plain_hit=j["plain_hit"],
                 learned_seq_hit=j["learned_seq_hit"])
        mod.append(m)
    s = learned.summarize(mod)
    s.update(changed_start_decisions=int(sum(j["changed_starts"] for j in judged)),
             start_decisions=int(sum(len(j["reached_learned"]) + len(j["reached_random"]) for j in judged)),
             changed_sequential_stops=int(sum(j["changed_stops"] for j in judged)),
             toys_global_minimum_differs=int(sum(not j["global_cluster_same"] for j in judged)),
             toys_gpu_choice_not_global=int(sum(not j["gpu_choice_is_global"] for j in judged)),
             max_abs_f_gpu_minus_oracle=float(max(abs(j["f_best_gpu"] - j["f_best_oracle"]) for j in judged)),
             minima_per_toy=float(np.mean([j["n_minima"] for j in judged])),
             reevaluated_per_toy=float(np.mean([j["n_reevaluated"] for j in judged])))
    return s


def main():
    import time

    import torch

    from paper_1108_5882_gb300 import build, pwa
    ap = argparse.ArgumentParser(description="learned-vs-random comparison, every decision judged by the oracle")
    ap.add_argument("--train-toys", type=int, default=100_000)
    ap.add_argument("--train-events", type=int, default=200_000)
    ap.add_argument("--eval-toys", type=int, default=100)
    ap.add_argument("--eval-events", type=int, default=1_000_000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--random-starts", type=int, default=256)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    build.build()
    h = pwa.Handle(0)
    seed = inputs.SEED_BASE + 5
    ws = inputs.wave_set_spread(16, seed)
    waves = pwa.waves_from(ws)
    t0 = time.perf_counter()
    Psi = learned.flat_psi(h, waves)
    feats, targets, _, _ = learned.make_training_set(h, waves, Psi, args.train_toys, args.train_events, seed)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    prop = learned.Proposer(h)
    t0 = time.perf_counter()
    hist = learned.train(prop, feats, targets, epochs=args.epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    Psi_or = oracle_psi(ws)
    Vh = learned.random_truths(args.eval_toys, 16, seed + 1)
    outs, judged = [], []
    t0 = time.perf_counter()
    for t in range(args.eval_toys):
        o = learned.evaluate_toy(h, waves, Psi, prop, Vh[t], args.eval_events, seed + 1, 7 + t, args.random_starts)
        judged.append(judge_toy(o, ws, Psi_or))
        o.pop("A")
        o.pop("kin")
        outs.append(o)
    t_eval = time.perf_counter() - t0
    gpu = learned.summarize(outs)
    orc = summarize_judged(outs, judged)
    per_toy = {k: [float(o[k]) for o in outs] for k in ("t_plain", "t_learned_seq", "t_rank", "t_random", "t_learned",
                                                         "n_plain", "n_learned_seq", "iters_first_learned")}
    res = dict(gpu_decided=gpu, oracle_decided=orc, per_toy=per_toy, train_toys=args.train_toys,
               train_events=args.train_events,
               eval_toys=args.eval_toys, eval_events=args.eval_events, epochs=args.epochs, loss_first=hist[0],
               loss_last=hist[-1], t_generate_s=t_gen, t_train_s=t_train, t_eval_and_judge_s=t_eval)
    print(json.dumps(res))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
