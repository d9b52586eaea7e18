"""Per-step measurement of the hot path: every kernel family at its workload size, timed with
CUDA events on the launching stream after warm-up, with the L2 flushed (a 512 MiB read) before
every timed launch, and compared with the roofline that bounds it.

    python -m paper_1108_5882_gb300.rowbench [--reps R] [--rows a1,a3,...] [--json out.json]

Peaks: HBM = the measured copy bandwidth of MEASURED_PEAKS.json; FP32 = the FFMA rate measured
now by libpwa_peaks.so (the library's microbenchmark).  For a kernel bound by both, the roofline
time is max(bytes / HBM, flop / FP32), and frac = roofline time / measured time.  Inputs are the
seeded synthetic workloads of paper_1108_5882_gb300.inputs (flat phase space; Sec. 2 of the
paper for the quantities).  Prints one line per measurement and, with --json, writes them all.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import time

import numpy as np
import torch

from . import build, inputs, learned, pwa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def hbm_peak() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except Exception:
        return 6800.0


def ffma_peak(sm_count: int) -> float:
    lib = ctypes.CDLL(build.PEAKS_LIB)
    lib.pwa_peak_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    best = 0.0
    for _ in range(3):
        ms, fl = ctypes.c_float(0), ctypes.c_double(0)
        if lib.pwa_peak_fma(0, 4 * sm_count, 2048, 20, ctypes.byref(ms), ctypes.byref(fl), None) != 0:
            raise RuntimeError("pwa_peak_fma failed")
        best = max(best, fl.value / (ms.value * 1e-3) / 1e12)
    return best


class Timer:
    def __init__(self, single=False):
        self.single = single
        self.flush = torch.ones(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        self.out = torch.empty((), dtype=torch.float32, device="cuda")

    def __call__(self, fn, reps=20, warmup=3, flush=True):
        st = torch.cuda.current_stream()
        if self.single:
            reps, warmup = 1, 1
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        if not self.single:
            torch.cuda._sleep(int(2e9 * 0.02))
        for i in range(reps):
            if flush:
                torch.sum(self.flush, dim=0, out=self.out)
            ev[i][0].record(st)
            fn()
            ev[i][1].record(st)
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ev])) * 1e-3  # seconds


def line(row, what, sec, nbytes=0.0, flops=0.0, hbm=6800.0, f32=80.0, extra=None):
    t_roof = max(nbytes / (hbm * 1e9), flops / (f32 * 1e12))
    bound = "hbm" if nbytes / (hbm * 1e9) >= flops / (f32 * 1e12) else "fp32"
    d = {"row": row, "what": what, "us": sec * 1e6, "GB/s": nbytes / sec / 1e9 if nbytes else None,
         "TFLOP/s": flops / sec / 1e12 if flops else None, "bound": bound, "frac": t_roof / sec}
    if extra:
        d.update(extra)
    gbs = f"{d['GB/s']:8.1f} GB/s" if d["GB/s"] else " " * 13
    tfs = f"{d['TFLOP/s']:7.2f} TF/s" if d["TFLOP/s"] else " " * 12
    print(f"{row:3s} {what:58s} {sec * 1e6:10.1f} us {gbs} {tfs}  {bound:4s} frac {d['frac']:.3f}", flush=True)
    return d


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--rows", default="a1,a1b,a2,a3,a3i,a4,a4u,a5,a7,a7p,a7h,a8,a9")
    ap.add_argument("--json", default=None)
    ap.add_argument("--profile", action="store_true",
                    help="one warm-up and one timed launch per kernel, no peak microbenchmark and 64 toys "
                         "in a8: a short run for a profiler to capture single launches")
    args = ap.parse_args()
    rows = set(args.rows.split(","))
    build.build()
    torch.cuda.set_device(0)
    h = pwa.Handle(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    HBM = hbm_peak()
    F32 = sms * 4 * 32 * 2 * 2.07e9 / 1e12 if args.profile else ffma_peak(sms)
    print(f"peaks: HBM {HBM:.1f} GB/s (measured copy), FP32 {F32:.2f} TFLOP/s "
          f"({'derived at 2.07 GHz' if args.profile else 'FFMA microbenchmark, now'})", flush=True)
    T = Timer(single=args.profile)
    out = {"peaks": {"hbm_gbs": HBM, "fp32_tflops": F32}, "rows": []}
    R = args.reps

    def add(*a, **k):
        out["rows"].append(line(*a, hbm=HBM, f32=F32, **k))

    seed = inputs.SEED_BASE + 2
    ws16 = inputs.wave_set_spread(16, seed)
    w16 = pwa.waves_from(ws16)
    if rows & {"a1", "a1b", "a2", "a3", "a5"}:
        n_mc = 5_000_000
        kin_mc = torch.from_numpy(inputs.kinematics(n_mc, seed, 5)).cuda()
        A_mc = torch.empty((16, n_mc), dtype=torch.complex64, device="cuda")
    if "a1" in rows:
        sec = T(lambda: h.pwa_amplitudes(w16, kin_mc, n_mc, A_mc), R)
        add("a1", "amplitudes K=16, 5e6 events", sec, nbytes=n_mc * (12 + 8 * 16),
            flops=n_mc * 16 * 30.0)
        dM = torch.empty_like(A_mc)
        dG = torch.empty_like(A_mc)
        sec = T(lambda: h.pwa_amplitudes(w16, kin_mc, n_mc, A_mc, dM, dG), R)
        add("a1", "amplitudes + dA/dM + dA/dG, K=16, 5e6 events", sec, nbytes=n_mc * (12 + 3 * 8 * 16),
            flops=n_mc * 16 * 50.0)
        del dM, dG
    if "a1b" in rows:
        # mass-dependent widths and barrier factors (L = J, K+K- daughters, R = 3 GeV^-1)
        wb = [(min(j, 4), l, m, w) for (j, l, m, w) in w16]
        sec = T(lambda: h.pwa_amplitudes_barrier(wb, 0.4937, 0.4937, 3.0, kin_mc, n_mc, A_mc), R)
        add("a1b", "amplitudes with mass-dependent widths and barrier factors, K=16, 5e6 events", sec,
            nbytes=n_mc * (12 + 8 * 16), flops=n_mc * 16 * 40.0)
    Psi16 = torch.empty((16, 16), dtype=torch.complex128, device="cuda")
    if rows & {"a2", "a3", "a5"}:
        h.pwa_amplitudes(w16, kin_mc, n_mc, A_mc)
        h.pwa_normint(A_mc, n_mc, Psi16)
    if "a2" in rows:
        # the tensor-core kernel (default: unit weights, K <= 32) and the FP32 SIMT one
        for tc in ("1", "0"):
            os.environ["PWA_NORMINT_TC"] = tc
            kind = "tcgen05" if tc == "1" else "SIMT"
            sec = T(lambda: h.pwa_normint(A_mc, n_mc, Psi16), R)
            add("a2", f"normint K=16, 5e6 MC events ({kind})", sec, nbytes=n_mc * 8 * 16, flops=n_mc * 8.0 * 16 * 17 / 2)
            sec = T(lambda: h.pwa_normint_from_kinematics(w16, kin_mc, n_mc, Psi16), R)
            add("a2", f"normint from kinematics K=16, 5e6 ({kind})", sec, nbytes=n_mc * 12.0,
                flops=n_mc * (30.0 * 16 + 8.0 * 16 * 17 / 2))
        os.environ.pop("PWA_NORMINT_TC")
        # the multistart workload's Psi: K=32, 1e7 MC events straight from the kinematics
        ws32n = inputs.wave_set_spread(32, seed + 1)
        kin32 = torch.from_numpy(inputs.kinematics(10_000_000, seed + 1, 5)).cuda()
        Psi32 = torch.empty((32, 32), dtype=torch.complex128, device="cuda")
        for tc in ("1", "0"):
            os.environ["PWA_NORMINT_TC"] = tc
            sec = T(lambda: h.pwa_normint_from_kinematics(pwa.waves_from(ws32n), kin32, 10_000_000, Psi32), max(5, R // 2))
            add("a2", f"normint from kinematics K=32, 1e7 ({'tcgen05' if tc == '1' else 'SIMT'})", sec,
                nbytes=1e7 * 12.0, flops=1e7 * (30.0 * 32 + 8.0 * 32 * 33 / 2))
        os.environ.pop("PWA_NORMINT_TC")
        del kin32
    if "a3" in rows:
        for K, N in ((4, 1_000_000), (16, 1_000_000), (16, 4_000_000), (32, 1_000_000)):
            wsK = inputs.wave_set_spread(K, seed)
            kin = torch.from_numpy(inputs.kinematics(N, seed, 4)).cuda()
            A = torch.empty((K, N), dtype=torch.complex64, device="cuda")
            h.pwa_amplitudes(pwa.waves_from(wsK), kin, N, A)
            V = torch.from_numpy(inputs.production_amplitudes(K, seed)[None, :]).cuda()
            Psi = torch.eye(K, dtype=torch.complex128, device="cuda")
            nll = torch.empty(1, dtype=torch.float64, device="cuda")
            g = torch.empty((1, 2 * K), dtype=torch.float64, device="cuda")
            sec = T(lambda: h.pwa_nll_grad(A, N, V, Psi, float(N), nll, g), R)
            add("a3", f"-lnL+grad one set (stream, a5+a6 fused), K={K}, N={N:.0e}", sec, nbytes=N * K * 8,
                flops=N * (16 * K + 12.0))
            del A, kin
    if "a3i" in rows:
        # incoherent sum over H = 2 states (two wave sets on the same events), K = 16, N = 1e6
        K, N, H = 16, 1_000_000, 2
        kin = torch.from_numpy(inputs.kinematics(N, seed, 4)).cuda()
        A = torch.empty((K, H, N), dtype=torch.complex64, device="cuda")
        for st in range(H):
            A_st = torch.empty((K, N), dtype=torch.complex64, device="cuda")
            h.pwa_amplitudes(pwa.waves_from(inputs.wave_set_spread(K, seed + 17 * st)), kin, N, A_st)
            A[:, st, :] = A_st
        V = torch.from_numpy(inputs.production_amplitudes(K, seed)[None, :]).cuda()
        Psi = torch.eye(K, dtype=torch.complex128, device="cuda")
        nll = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty((1, 2 * K), dtype=torch.float64, device="cuda")
        sec = T(lambda: h.pwa_nll_grad_incoherent(A, N, V, Psi, float(N), nll, g), R)
        add("a3i", f"incoherent -lnL+grad (H={H} states), K={K}, N={N:.0e}", sec, nbytes=N * K * H * 8,
            flops=N * H * (16 * K + 4.0))
        del A, kin
    if "a7h" in rows:
        # Hessian of -lnL for one set, K = 16, N = 1e6 (Fumili: one fused pass; exact: + the
        # weighted normalisation-integral pass)
        K, N = 16, 1_000_000
        kin = torch.from_numpy(inputs.kinematics(N, seed, 4)).cuda()
        A = torch.empty((K, N), dtype=torch.complex64, device="cuda")
        h.pwa_amplitudes(w16, kin, N, A)
        V = torch.from_numpy(inputs.production_amplitudes(K, seed)).cuda()
        Psi = torch.eye(K, dtype=torch.complex128, device="cuda")
        Hm = torch.empty((2 * K, 2 * K), dtype=torch.float64, device="cuda")
        for exact in (False, True):
            sec = T(lambda: h.pwa_hessian(A, N, V, Psi, float(N), Hm, exact=exact), R)
            D = 2 * K
            # algorithmic bytes: A read once (Fumili); exact: A read again by the weighted Gram
            # pass, and 1/I written and read.  flops: r_i (~14K + 4), the symmetric rank-1
            # update D(D+1), exact: + the complex Gram 4K(K+1)
            nb = N * K * 8 * (2 if exact else 1) + (8 * N if exact else 0)
            fl = N * (14.0 * K + 4 + D * (D + 1)) + (N * 4.0 * K * (K + 1) if exact else 0.0)
            add("a7h", f"Hessian of -lnL ({'exact' if exact else 'Fumili'}), K={K}, N={N:.0e}", sec, nbytes=nb, flops=fl)
        del A, kin
    if "a5" in rows:
        # floating shape: data 1e6 + MC 5e6 events, 4 floating parameters (2 masses, 2 widths)
        K, N, F = 16, 1_000_000, 4
        kin = torch.from_numpy(inputs.kinematics(N, seed, 4)).cuda()
        A = torch.empty((K, N), dtype=torch.complex64, device="cuda")
        h.pwa_amplitudes(w16, kin, N, A)
        dA = torch.zeros((F, N), dtype=torch.complex64, device="cuda")
        dAm = torch.zeros((F, n_mc), dtype=torch.complex64, device="cuda")
        V = torch.from_numpy(inputs.production_amplitudes(K, seed)).cuda()
        nll = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty(2 * K + F, dtype=torch.float64, device="cuda")
        fw = [3, 3, 9, 9]
        sec = T(lambda: h.pwa_nll_grad_shape(A, dA, N, A_mc, dAm, n_mc, fw, V, float(N), nll, g), R)
        add("a5", "streamed-normalisation -lnL + V and (M,G) gradient, K=16, 1e6+5e6", sec,
            nbytes=(N + n_mc) * (K + F) * 8, flops=(N + n_mc) * (16 * K + 4 * F + 12.0))
        del A, dA, dAm, kin
    if rows & {"a1", "a1b", "a2", "a3", "a5"}:
        del A_mc, kin_mc
    if rows & {"a4", "a7", "a7p"}:
        K, N, P = 32, 2_000_000, 256
        ws32 = inputs.wave_set_spread(K, seed + 1)
        kin = torch.from_numpy(inputs.kinematics(N, seed + 1, 4)).cuda()
        A = torch.empty((K, N), dtype=torch.complex64, device="cuda")
        h.pwa_amplitudes(pwa.waves_from(ws32), kin, N, A)
        del kin
        kin_mc = torch.from_numpy(inputs.kinematics(2_000_000, seed + 1, 5)).cuda()
        A_mc = torch.empty((K, 2_000_000), dtype=torch.complex64, device="cuda")
        h.pwa_amplitudes(pwa.waves_from(ws32), kin_mc, 2_000_000, A_mc)
        Psi = torch.empty((K, K), dtype=torch.complex128, device="cuda")
        h.pwa_normint(A_mc, 2_000_000, Psi)
        del A_mc, kin_mc
        V = torch.from_numpy(inputs.starts(P, K, seed + 1)).cuda()
        nll = torch.empty(P, dtype=torch.float64, device="cuda")
        g = torch.empty((P, 2 * K), dtype=torch.float64, device="cuda")
        h.pwa_reserve(K, N, P)
        if "a4" in rows:
            sec = T(lambda: h.pwa_nll_grad(A, N, V, Psi, float(N), nll, g), max(5, R // 2))
            shape = h.pwa_batched_shape(K, N, P)
            extra = {"shape": shape}
            if shape == 4:
                # tensor cores: FP32 products emulated by three TF32 products; peak = TF32 dense
                # (measured bf16 burst x 1.1 / 2.25) / 3
                with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                    tpeak = float(json.load(fh)["bf16_tflops"]) * (1.1 / 2.25) / 3.0
                extra.update({"tensor_emulated_fp32_peak": tpeak,
                              "frac_tensor": N * P * (16 * K + 12.0) / sec / 1e12 / tpeak})
            add("a4", f"batched -lnL+grad, K={K}, N={N:.0e}, P={P} (autotuned shape {shape})", sec, nbytes=N * K * 8,
                flops=N * P * (16 * K + 12.0), extra=extra)
            if shape == 4:
                print(f"      tensor-core shape: {extra['frac_tensor']:.3f} of the 3xTF32 emulated-FP32 peak "
                      f"({tpeak:.1f} TFLOP/s)", flush=True)
        for tag, polar in (("a7", 0), ("a7p", 1)):
            if tag not in rows:
                continue
            Vout = torch.empty((P, K), dtype=torch.complex128, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = h.pwa_fit_batch([dict(A=A, n=N, Psi=Psi, n_factor=N, V0=V, V_out=Vout)], pwa.fit_opts(polar=polar))
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            iters = max(r["iterations"] for r in res)
            evals = sum(r["evaluations"] for r in res) / P
            conv = sum(r["status"] == 0 for r in res)
            best = min(r["nll"] for r in res)
            coords = "polar (rho, phi)" if polar else "Cartesian (Re V, Im V)"
            out["rows"].append({"row": tag, "what": f"batched L-BFGS fit K={K}, N={N:.0e}, P={P}, {coords}",
                                "wall_s": wall, "iterations_max": iters, "evaluations_per_start": evals,
                                "converged": conv, "best_nll": best})
            print(f"{tag:3s} batched L-BFGS fit K={K}, N={N:.0e}, P={P}, {coords}: {wall:.3f} s, {iters} iterations "
                  f"(max), {evals:.1f} evaluations/start, {conv}/{P} converged, best -lnL {best:.3f}", flush=True)
        del A
    if "a4u" in rows:
        # many channels with floating masses and widths in one persistent launch: the uneven
        # workload's 64 channels at 1/8 of its event counts (N_data log-U[1e4, 5e5], N_MC = 5 N_data),
        # flat events; masses and widths of waves 0 and K/2 float
        sdu = inputs.SEED_BASE + 6
        descs, Vs, ths, flops, n_data, n_ev = [], [], [], 0.0, 0, 0
        for c, (K, N, NMC) in enumerate(inputs.uneven_channels(64, sdu, nmax=5e5)):
            wsu = inputs.wave_set_spread(K, sdu, stream=100 + c)
            ld, ldm = N + (N & 1), NMC + (NMC & 1)
            fl = [0, K // 2]
            descs.append(dict(waves=pwa.waves_from(wsu), kin=torch.from_numpy(inputs.kinematics(N, sdu, 300 + c, ld=ld)).cuda(),
                              n=N, kin_mc=torch.from_numpy(inputs.kinematics(NMC, sdu, 400 + c, ld=ldm)).cuda(),
                              n_mc=NMC, n_gen=float(NMC), n_factor=float(N), float_wave=[fl[0], fl[1], fl[0], fl[1]],
                              float_kind=[0, 0, 1, 1]))
            Vs.append(inputs.production_amplitudes(K, sdu, stream=200 + c))
            ths.append([wsu.M[fl[0]], wsu.M[fl[1]], wsu.W[fl[0]], wsu.W[fl[1]]])
            # per event: per wave one Breit-Wigner (11 flop) and the complex multiply-adds into u and
            # the gradient (16); per floating parameter 10; |u|^2, ln I and w 12
            flops += (N + NMC) * (27.0 * K + 10 * 4 + 12)
            n_data += N
            n_ev += N + NMC
        Vu = torch.from_numpy(np.concatenate(Vs)).cuda()
        thu = torch.tensor(np.concatenate(ths), dtype=torch.float64, device="cuda")
        nllu = torch.empty(len(descs), dtype=torch.float64, device="cuda")
        gu = torch.empty(sum(2 * len(d["waves"]) + 4 for d in descs), dtype=torch.float64, device="cuda")
        sec = T(lambda: h.pwa_nll_grad_uneven(descs, Vu, thu, nllu, gu), max(5, R // 2), flush=False)
        add("a4u", f"64 channels, floating (M,G), {n_data:.2e} data + {n_ev - n_data:.2e} MC events", sec,
            nbytes=12.0 * n_ev, flops=flops)
        del descs, Vu, thu
    if "a8" in rows:
        sd = inputs.SEED_BASE + 5
        wsl = inputs.wave_set_spread(16, sd)
        wl = pwa.waves_from(wsl)
        Psi_flat = learned.flat_psi(h, wl)
        Tt, n_t = (64 if args.profile else 1024), 200_000
        V = learned.random_truths(Tt, 16, sd)
        Vd = torch.from_numpy(V).cuda()
        feats = torch.empty((Tt, 1000), dtype=torch.float64, device="cuda")
        nacc = torch.empty(Tt, dtype=torch.int64, device="cuda")
        sec = T(lambda: h.pwa_toy_moments(wl, Vd, Psi_flat, n_t, sd, 100_000, feats, nacc), 3, warmup=1, flush=False)
        s_nll = torch.empty(Tt, dtype=torch.float64, device="cuda")
        h.pwa_nll(torch.zeros((16, 2), dtype=torch.complex64, device="cuda"), 0, Vd, Psi_flat, 1.0, s_nll)
        S = s_nll.cpu().numpy()
        C = np.array([pwa.pwa_envelope(wl, V[t]) for t in range(Tt)])
        n_cand = float(np.sum(np.ceil(n_t * C / S)))
        acc = float(nacc.sum())
        # flop estimate per candidate: K waves x ~24 (Breit-Wigner, angular factor, complex
        # products) + ~40 angles; Philox integer work not counted
        add("a8", f"toy generation + moments, {Tt} toys x {n_t:.0e} events, K=16", sec,
            flops=n_cand * (16 * 24 + 40.0),
            extra={"accepted_per_s": acc / sec, "candidates_per_s": n_cand / sec, "candidates_per_accepted": n_cand / acc})
        print(f"      {acc / sec / 1e9:.3f} G accepted events/s, {n_cand / sec / 1e9:.2f} G candidates/s, "
              f"{n_cand / acc:.1f} candidates per event", flush=True)
    if "a9" in rows:
        prop = learned.Proposer(h)
        B = 256
        X = torch.randn((B, 1000), device="cuda").to(torch.bfloat16)
        tgt = torch.randn((B, 32), device="cuda")
        sec = T(lambda: prop.train_step(X, tgt), R, flush=False)
        macs = sum(prop.dims[i] * prop.dims[i + 1] for i in range(len(prop.dims) - 1))
        flops = 2.0 * B * macs * 3  # forward, input gradient, weight gradient
        add("a9", f"MLP training step (fwd+bwd+WTA+Adam), batch {B}", sec, flops=flops,
            nbytes=4.0 * macs * 5)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(out, fh, indent=1)
    h.close()


if __name__ == "__main__":
    main()
