#!/usr/bin/env python3
"""Benchmark of the PWA likelihood hot path on GB300 (one JSON line on rank 0).

Workload (default "multistart", the largest single-GPU configuration): K=32 waves (J in
{0,2,4} x lambda in {0,1}, masses spread over 1.3-2.8 GeV), N_data = 2e6 events drawn on the GPU
by accept-reject from I under a seeded V, N_MC = 1e7 flat phase-space events, complex64
amplitudes, P = 256 parameter sets (|V| U[0,2], arg V U[0,2pi)) evaluated together.
Amplitudes and Psi are computed once (masses and widths fixed: Sec. 2 of the paper, the
bracket and per-event terms can be pre-calculated); one step is one multistart-iteration
evaluation of -lnL and its gradient at all P sets (the batched event x wave x set contraction,
the normalisation term and the fixed-order reduction).  "scale" (K=16, N=1e6, P=1) and
"plain" (K=4, N=1e4, P=1) give the other configurations' lines.

Metric: event x parameter-set NLL+grad evaluations per second = N_data * P / step time.
  value     device time of the steps (CUDA events on the launching stream), inputs resident in
            HBM, L2 flushed (a 512 MiB read) before every step, outside the events.
  e2e       the same metric through the C ABI from HOST buffers: each step copies the data and MC
            kinematics from pinned host memory, recomputes amplitudes and Psi, evaluates -lnL
            and its gradient, and reads nll and the gradient back.
  roofline  the dominant kernel against its roof: P = 1, the streaming kernel against the
            measured HBM copy bandwidth (N_data * K * 8 bytes per launch); P > 1, the batched
            contraction's (16K + 12) flop per (event, set) against the FFMA rate measured in the
            same run (FP32 SIMT shapes) or against the emulated-FP32 tensor peak (tensor-core shape).
  cpu_baseline  the FP64 oracle (single-threaded C) on all N_data events of the workload and a
            stated fraction of its parameter sets, extrapolated linearly to a full iteration.

--impl reference times the oracle as the reference arm on a bounded sample of this workload.
Under torchrun (N > 1) every rank evaluates its own replica (independent fits, no collective
on the data path): weak scaling, value = all ranks' units / max time over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "event x param-set NLL+grad evals/s"
UNIT = "event-evals/s"

WORKLOADS = {
    # name: (K, N_data, N_MC, P, seed)
    "plain": (4, 10_000, 50_000, 1, 11085883),
    "scale": (16, 1_000_000, 5_000_000, 1, 11085884),
    "multistart": (32, 2_000_000, 10_000_000, 256, 11085885),
}
# uneven: 64 channels, K ~ U{4..48}, N_data log-U[1e4, 4e6], N_MC = 5 N_data, 2 floating masses and
# 2 floating widths per channel
UNEVEN = (64, 11085886)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Polls SM clock and clock-event reasons through NVML (read-only queries) while running."""

    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
               0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}

    def __init__(self, device_index: int, period_s: float = 0.002):
        self.samples = []
        self.reasons = 0
        self.max_mhz = None
        self.ok = False
        self.period = period_s
        self._stop = threading.Event()
        try:
            import torch
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            p = torch.cuda.get_device_properties(device_index)
            bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0".encode()
            self.dev = ctypes.c_void_p()
            if self.nvml.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(self.dev)) != 0:
                return
            mx = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(mx)) == 0:  # 1 = SM clock
                self.max_mhz = int(mx.value)
            self.ok = True
        except Exception:
            self.ok = False

    def _run(self):
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        get_reasons = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(self.nvml, "nvmlDeviceGetCurrentClocksThrottleReasons")
        while not self._stop.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(clk)) == 0:
                self.samples.append(int(clk.value))
            if get_reasons(self.dev, ctypes.byref(rs)) == 0:
                self.reasons |= int(rs.value)
            time.sleep(self.period)

    def __enter__(self):
        if self.ok:
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()
        return self

    def __exit__(self, *a):
        if self.ok:
            self._stop.set()
            self.t.join()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"]}
        names = [v for k, v in self.REASONS.items() if self.reasons & k]
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz, "reasons": names,
                "samples": len(self.samples)}


def measured_traffic(kernel_tag):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None when
    the kernel's sources changed since that capture (their sha256 no longer matches)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        hsh = hashlib.sha256()
        for f in d["sources"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                hsh.update(fh.read())
        if hsh.hexdigest() != d["sources_sha256"]:
            return None
        return float(d["dram_bytes_read"]) + float(d["dram_bytes_write"])
    except Exception:
        return None


def fma_peak_tflops(sm_count, fp64=False, launches=20):
    """FMA rate of this GPU's SIMT pipes in TFLOP/s, measured now by the library's own
    microbenchmark (libpwa_peaks.so): best of three sequences of `launches` launches."""
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_1108_5882_gb300", "lib", "libpwa_peaks.so"))
    lib.pwa_peak_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    blocks = 4 * sm_count
    iters = 64 if fp64 else 2048  # ~2 ms per FP32 launch
    best = 0.0
    for _ in range(3):
        ms, fl = ctypes.c_float(0), ctypes.c_double(0)
        rc = lib.pwa_peak_fma(1 if fp64 else 0, blocks, iters, launches, ctypes.byref(ms), ctypes.byref(fl), None)
        if rc != 0:
            raise RuntimeError(f"pwa_peak_fma failed: CUDA error {rc}")
        best = max(best, fl.value / (ms.value * 1e-3) / 1e12)
    return best


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- ranks
def dist_backend():
    """nccl on GPU ranks; gloo for the host-side tests of the rank logic (or PWA_DIST_BACKEND)."""
    import torch
    return os.environ.get("PWA_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")


def dist_init(ngpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = dist_backend()
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput of weak-scaling replicas: each of the `world` ranks processed
    units_per_rank units, and `seconds` is the slowest rank's time (max over ranks)."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------- workload
def setup_workload(name, h, rank):
    """Generate the synthetic workload on the device with the library's own kernels."""
    import torch

    from paper_1108_5882_gb300 import inputs, pwa
    K, N, NMC, P, seed = WORKLOADS[name]
    seed = seed + 1000 * rank
    ws = inputs.wave_set_plain(seed) if name == "plain" else inputs.wave_set_spread(K, seed)
    waves = pwa.waves_from(ws)
    V_true = inputs.production_amplitudes(K, seed)
    C = pwa.pwa_envelope(waves, V_true)
    # data: accept-reject on the device (Philox candidates, candidate-ordered output)
    kin = torch.zeros((3, N), dtype=torch.float32, device="cuda")
    na = torch.zeros(1, dtype=torch.int64, device="cuda")
    Vd = torch.from_numpy(V_true).cuda()
    got, cand0, chunk = 0, 0, 1 << 25
    while got < N:
        tmp = torch.zeros((3, N - got), dtype=torch.float32, device="cuda")
        h.pwa_generate(waves, Vd, seed, 0, cand0, chunk, C, tmp, N - got, na)
        k = min(int(na.item()), N - got)
        kin[:, got:got + k] = tmp[:, :k]
        got += k
        cand0 += chunk
    kin_mc_h = inputs.kinematics(NMC, seed, 5)
    kin_mc = torch.from_numpy(kin_mc_h).cuda()
    A = torch.zeros((K, N), dtype=torch.complex64, device="cuda")
    A_mc = torch.zeros((K, NMC), dtype=torch.complex64, device="cuda")
    h.pwa_amplitudes(waves, kin, N, A)
    h.pwa_amplitudes(waves, kin_mc, NMC, A_mc)
    Psi = torch.zeros((K, K), dtype=torch.complex128, device="cuda")
    h.pwa_normint(A_mc, NMC, Psi)
    torch.cuda.synchronize()
    # parameter sets visited by the steps: perturbations of the truth (a fit's iterates)
    g = np.random.default_rng(seed)
    n_sets = 64
    Vs = []
    for s in range(n_sets):
        if P == 1:
            pert = V_true * (1 + 0.05 * (g.normal(size=K) + 1j * g.normal(size=K)))
            Vs.append(pert.astype(np.complex64)[None, :])
        else:
            Vs.append(inputs.starts(P, K, seed + s))
    Vs = torch.from_numpy(np.stack(Vs)).cuda()
    return dict(K=K, N=N, NMC=NMC, P=P, seed=seed, waves=waves, kin=kin, kin_mc=kin_mc, kin_mc_h=kin_mc_h,
                A=A, A_mc=A_mc, Psi=Psi, Vs=Vs, ws=ws, V_true=V_true)


# ----------------------------------------------------------------------------- our arm
def run_ours(args, world, rank, local):
    import torch

    from paper_1108_5882_gb300 import build, pwa
    if rank == 0 or world > 1:
        build.build()
    torch.cuda.set_device(local)
    h = pwa.Handle(local)
    wl = setup_workload(args.workload, h, rank)
    K, N, P = wl["K"], wl["N"], wl["P"]
    nll = torch.zeros(P, dtype=torch.float64, device="cuda")
    grad = torch.zeros((P, 2 * K), dtype=torch.float64, device="cuda")
    h.pwa_reserve(K, N, P)
    stream = torch.cuda.current_stream()
    # L2 flush: READ a 512 MiB buffer (> 129 MB L2) so that L2 holds clean lines of another buffer;
    # a write-flush would leave ~126 MB of dirty lines whose write-back competes with the step
    flush = torch.ones(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_out = torch.empty((), dtype=torch.float32, device="cuda")

    def l2_flush():
        torch.sum(flush, dim=0, out=flush_out)

    nsets = wl["Vs"].shape[0]

    def step(i):
        h.pwa_nll_grad(wl["A"], N, wl["Vs"][i % nsets], wl["Psi"], float(N), nll, grad)

    for i in range(args.warmup):
        l2_flush()
        step(i)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    with sampler:
        # park the GPU behind a bounded sleep kernel while the host queues every timed launch,
        # so that no step waits for the host (the sleep ends before the first timed event)
        torch.cuda._sleep(int(min(2.0, 2e-4 * args.steps + 0.02) * 2.0e9))
        t0 = time.perf_counter()
        for i in range(args.steps):
            l2_flush()
            ev[i][0].record(stream)
            step(i)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = tot_ms / args.steps
    value = job_rate(N * P * args.steps, world, tot_ms * 1e-3)
    kernel_ms = sum(step_ms) / len(step_ms)  # one launch of the streaming kernel per step
    ok = h.pwa_sync_status()

    # ---- end to end from host buffers through the C ABI
    kin_h = wl["kin"].cpu().pin_memory()
    kin_mc_h = torch.from_numpy(wl["kin_mc_h"]).pin_memory()
    # two device buffers per input: the copies of step t + 1 (on their own stream) overlap the
    # kernels of step t; a buffer is refilled only after the step that read it is done with it
    kin_d = [torch.empty_like(wl["kin"]) for _ in range(2)]
    kin_mc_d = [torch.empty_like(wl["kin_mc"]) for _ in range(2)]
    V_h = wl["Vs"][0].cpu().pin_memory()
    V_d = [torch.empty_like(wl["Vs"][0]) for _ in range(2)]
    nll_h = torch.empty(P, dtype=torch.float64).pin_memory()
    grad_h = torch.empty((P, 2 * K), dtype=torch.float64).pin_memory()
    A, Psi = torch.empty_like(wl["A"]), torch.empty_like(wl["Psi"])
    NMC = wl["NMC"]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]
    for ev in used:
        ev.record(stream)
    step_no = [0]

    def e2e_step():
        b = step_no[0] % 2
        step_no[0] += 1
        copy_stream.wait_event(used[b])
        with torch.cuda.stream(copy_stream):
            kin_d[b].copy_(kin_h, non_blocking=True)
            V_d[b].copy_(V_h, non_blocking=True)
            kin_mc_d[b].copy_(kin_mc_h, non_blocking=True)
            copied[b].record(copy_stream)
        stream.wait_event(copied[b])
        h.pwa_amplitudes(wl["waves"], kin_d[b], N, A)
        h.pwa_normint_from_kinematics(wl["waves"], kin_mc_d[b], NMC, Psi)  # MC amplitudes stay on chip
        h.pwa_nll_grad(A, N, V_d[b], Psi, float(N), nll, grad)
        used[b].record(stream)
        nll_h.copy_(nll, non_blocking=True)
        grad_h.copy_(grad, non_blocking=True)

    n_e2e = max(3, min(20, args.steps))
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    e0.record(stream)
    for ev in used:  # the first timed copies start after e0
        ev.record(stream)
    for _ in range(n_e2e):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / n_e2e, world)
    h2d = kin_h.numel() * 4 + kin_mc_h.numel() * 4 + V_h.numel() * 8
    d2h = nll_h.numel() * 8 + grad_h.numel() * 8
    # the copy part of an e2e step alone (the same three host-to-device copies), for the breakdown
    e0.record(stream)
    for _ in range(n_e2e):
        kin_d[0].copy_(kin_h, non_blocking=True)
        kin_mc_d[0].copy_(kin_mc_h, non_blocking=True)
        V_d[0].copy_(V_h, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    h2d_ms = e0.elapsed_time(e1) / n_e2e

    if P == 1:
        peak, peak_kind = measured_peaks()
        alg_bytes = N * K * 8 + P * K * 8 + K * K * 16
        achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": measured_traffic(f"k_nll_stream_{args.workload}"),
                    "kernel": f"k_nll_stream<{K if K in (4, 8, 16, 32, 48, 64) else 'KMAX'},true,true,true>",
                    "bytes_per_launch": alg_bytes, "kernel_us": kernel_ms * 1e3,
                    "peak_kind": f"{peak_kind} (copy bandwidth)"}
    else:
        # per (event, start): 4K complex multiply-adds for U = A V^T and 4K for G = A^H W (16K
        # flop) + ~12 for |U|^2, 1/I, ln I
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        flops = float(N) * P * (16 * K + 12)
        achieved = flops / (kernel_ms * 1e-3) / 1e12
        ffma = fma_peak_tflops(sms)
        shape = h.pwa_batched_shape(K, N, P)
        if shape == 4:
            # tensor cores: each FP32 product is three TF32 products, so the FP32-emulated peak is
            # the TF32 dense peak / 3; the TF32 peak is the measured bf16 burst x the nominal
            # TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s)
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                bf16 = float(json.load(fh)["bf16_tflops"])
            peak = bf16 * (1.1 / 2.25) / 3.0
            roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": measured_traffic(f"k_nll_tc_{args.workload}"),
                        "kernel": "k_nll_tc (tcgen05 3xTF32) + k_nll_finalize (one step)",
                        "flops_per_launch": flops, "kernel_us": kernel_ms * 1e3,
                        "peak_kind": "of measured: bf16 burst x 1.1/2.25 (TF32 dense) / 3 (FP32 emulation)",
                        "fp32_simt_peak": ffma, "frac_of_fp32_simt": achieved / ffma}
        else:
            roofline = {"bound": "alu", "achieved": achieved, "peak": ffma, "unit": "TFLOP/s", "frac": achieved / ffma,
                        "traffic": None, "kernel": f"k_nll_batched shape {shape} + k_nll_finalize (one step)",
                        "flops_per_launch": flops, "kernel_us": kernel_ms * 1e3,
                        "peak_kind": "measured now: FFMA microbenchmark (libpwa_peaks.so), FP32 SIMT",
                        "peak_derived": sms * 128 * 2 * 2.07e9 / 1e12}
    launches = args.steps * (1 if P == 1 else 2)
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (accept-reject from I on the GPU; flat MC)",
        "config": {"workload": f"{args.workload}: K={K}, N_data={N}, N_MC={wl['NMC']}, P={P}, "
                               "one -lnL+gradient evaluation per step, amplitudes and Psi precomputed",
                   "K": K, "N_data": N, "N_MC": wl["NMC"], "P": P, "l2": "flushed before every step (512 MiB read)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": job_rate(N * P, world, e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "h2d_ms_per_step": h2d_ms,
                "what": "pinned H2D of data+MC kinematics and V (copy stream, double-buffered: step t+1's copies "
                        "overlap step t's kernels), amplitudes(data), Psi from the MC kinematics (MC amplitudes computed on chip), "
                        "-lnL+grad, D2H of nll+grad"},
        "gpu_launches": launches,
        "roofline": roofline,
        "clocks": sampler.summary(),
        "status": pwa.status_string(ok), "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    h.close()
    return res


# ----------------------------------------------------------------------------- uneven channels
def setup_uneven(h, rank):
    """64 channels on the device: data drawn by the library's accept-reject from I under a seeded V
    per channel, flat MC drawn by torch's seeded device generator, floating masses and widths of
    waves 0 and K/2 set slightly off the values the data were drawn with."""
    import torch

    from paper_1108_5882_gb300 import inputs, pwa
    n_ch, seed = UNEVEN
    seed = seed + 1000 * rank
    chans = []
    for c, (K, N, NMC) in enumerate(inputs.uneven_channels(n_ch, seed)):
        ws = inputs.wave_set_spread(K, seed, stream=100 + c)
        waves = pwa.waves_from(ws)
        V = inputs.production_amplitudes(K, seed, stream=200 + c)
        C = pwa.pwa_envelope(waves, V)
        ld, ld_mc = N + (N & 1), NMC + (NMC & 1)
        kin = torch.zeros((3, ld), dtype=torch.float32, device="cuda")
        na = torch.zeros(1, dtype=torch.int64, device="cuda")
        Vd = torch.from_numpy(V).cuda()
        got, cand0, chunk = 0, 0, 1 << 26
        while got < N:
            tmp = torch.zeros((3, N - got), dtype=torch.float32, device="cuda")
            h.pwa_generate(waves, Vd, seed, c, cand0, chunk, C, tmp, N - got, na)
            k = min(int(na.item()), N - got)
            kin[:, got:got + k] = tmp[:, :k]
            got += k
            cand0 += chunk
        g = torch.Generator(device="cuda")
        g.manual_seed(seed * 64 + c)
        kin_mc = torch.zeros((3, ld_mc), dtype=torch.float32, device="cuda")
        u = torch.rand((3, NMC), generator=g, device="cuda")
        kin_mc[0, :NMC] = inputs.M_LO + (inputs.M_HI - inputs.M_LO) * u[0]
        kin_mc[1, :NMC] = 2.0 * u[1] - 1.0
        kin_mc[2, :NMC] = torch.clamp(2.0 * math.pi * u[2], max=math.nextafter(2.0 * math.pi, 0.0))
        del u
        fl = [0, K // 2]
        theta = [ws.M[fl[0]] * 1.002, ws.M[fl[1]] * 0.998, ws.W[fl[0]] * 1.01, ws.W[fl[1]] * 0.99]
        chans.append(dict(waves=waves, K=K, kin=kin, n=N, kin_mc=kin_mc, n_mc=NMC, n_gen=float(NMC), n_factor=float(N),
                          float_wave=[fl[0], fl[1], fl[0], fl[1]], float_kind=[0, 0, 1, 1], V=V, theta=theta, ws=ws))
    torch.cuda.synchronize()
    return chans


def uneven_flops(chans):
    """Algorithmic FP32 work of one evaluation of every channel: per (event, wave) one Breit-Wigner
    (11 flop), the complex multiply-add into u (8) and into the gradient (8); per event and
    floating parameter its derivative term (10); per event |u|^2, ln I and w (12)."""
    return float(sum((c["n"] + c["n_mc"]) * (27 * c["K"] + 10 * len(c["float_wave"]) + 12) for c in chans))


def cpu_baseline_uneven(chans, seconds):
    """The oracle on whole channels (FP64 amplitudes with their mass and width derivatives, then
    f and the gradient in V and theta), smallest channels first for about `seconds`; a full
    evaluation of all channels is extrapolated linearly in (events x waves)."""
    import oracle
    order = sorted(range(len(chans)), key=lambda c: (chans[c]["n"] + chans[c]["n_mc"]) * chans[c]["K"])
    done, work_done, t_tot = 0, 0.0, 0.0
    for c in order:
        ch = chans[c]
        ws = ch["ws"]
        kin = np.ascontiguousarray(ch["kin"][:, :ch["n"]].cpu().numpy())
        kin_mc = np.ascontiguousarray(ch["kin_mc"][:, :ch["n_mc"]].cpu().numpy())
        M, W = ws.M.copy(), ws.W.copy()
        for q, (r, k) in enumerate(zip(ch["float_wave"], ch["float_kind"])):
            (M if k == 0 else W)[r] = ch["theta"][q]
        t0 = time.perf_counter()
        A, dM, dW = oracle.amplitudes(ws.J, ws.lam, M, W, kin, derivs=True)
        Am, dMm, dWm = oracle.amplitudes(ws.J, ws.lam, M, W, kin_mc, derivs=True)
        dA = np.stack([(dM if k == 0 else dW)[r] for r, k in zip(ch["float_wave"], ch["float_kind"])])
        dAm = np.stack([(dMm if k == 0 else dWm)[r] for r, k in zip(ch["float_wave"], ch["float_kind"])])
        oracle.nll_grad_shape(A.astype(np.complex64), dA.astype(np.complex64), Am.astype(np.complex64),
                              dAm.astype(np.complex64), ch["float_wave"], ch["V"], n_factor=ch["n_factor"],
                              n_gen=ch["n_gen"])
        t_tot += time.perf_counter() - t0
        done += 1
        work_done += (ch["n"] + ch["n_mc"]) * ch["K"]
        if t_tot >= seconds:
            break
    work_all = float(sum((c["n"] + c["n_mc"]) * c["K"] for c in chans))
    full_s = t_tot * work_all / work_done
    n_all = sum(c["n"] for c in chans)
    return {"value": n_all / full_s, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
            "nproc": os.cpu_count(), "full_iteration_s": full_s, "full_iteration_extrapolated": done < len(chans),
            "sample": f"FP64 amplitudes (with mass and width derivatives) and -lnL+gradient of the {done} smallest of "
                      f"{len(chans)} channels, {t_tot:.1f} s; one evaluation of all channels extrapolated linearly in "
                      f"events x waves ({work_done / work_all:.4f} of the work): {full_s:.1f} s"}


def run_uneven(args, world, rank, local):
    import torch

    from paper_1108_5882_gb300 import build, pwa
    if rank == 0 or world > 1:
        build.build()
    torch.cuda.set_device(local)
    h = pwa.Handle(local)
    chans = setup_uneven(h, rank)
    descs = [dict(waves=c["waves"], kin=c["kin"], n=c["n"], kin_mc=c["kin_mc"], n_mc=c["n_mc"], n_gen=c["n_gen"],
                  n_factor=c["n_factor"], float_wave=c["float_wave"], float_kind=c["float_kind"]) for c in chans]
    V = torch.from_numpy(np.concatenate([c["V"] for c in chans])).cuda()
    theta = torch.tensor(np.concatenate([c["theta"] for c in chans]), dtype=torch.float64, device="cuda")
    nll = torch.zeros(len(chans), dtype=torch.float64, device="cuda")
    grad = torch.zeros(sum(2 * c["K"] + len(c["float_wave"]) for c in chans), dtype=torch.float64, device="cuda")
    n_data = sum(c["n"] for c in chans)
    n_events = sum(c["n"] + c["n_mc"] for c in chans)
    stream = torch.cuda.current_stream()

    def step():
        h.pwa_nll_grad_uneven(descs, V, theta, nll, grad)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    with sampler:
        torch.cuda._sleep(int(min(2.0, 3e-3 * args.steps + 0.02) * 2.0e9))
        t0 = time.perf_counter()
        for i in range(args.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = tot_ms / args.steps
    value = job_rate(n_data * args.steps, world, tot_ms * 1e-3)
    ok = h.pwa_sync_status()
    # ---- end to end: every step copies all kinematics from pinned host memory, evaluates, reads back
    kin_h = [c["kin"].cpu().pin_memory() for c in chans]
    kin_mc_h = [c["kin_mc"].cpu().pin_memory() for c in chans]
    V_h, theta_h = V.cpu().pin_memory(), theta.cpu().pin_memory()
    nll_h = torch.empty_like(nll, device="cpu").pin_memory()
    grad_h = torch.empty_like(grad, device="cpu").pin_memory()
    n_e2e = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for _ in range(n_e2e):
        for c, a, b in zip(chans, kin_h, kin_mc_h):
            c["kin"].copy_(a, non_blocking=True)
            c["kin_mc"].copy_(b, non_blocking=True)
        V.copy_(V_h, non_blocking=True)
        theta.copy_(theta_h, non_blocking=True)
        step()
        nll_h.copy_(nll, non_blocking=True)
        grad_h.copy_(grad, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / n_e2e, world)
    h2d = sum(t.numel() * 4 for t in kin_h + kin_mc_h) + V_h.numel() * 8 + theta_h.numel() * 8
    d2h = nll_h.numel() * 8 + grad_h.numel() * 8
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    ffma = fma_peak_tflops(sms)
    flops = uneven_flops(chans)
    kernel_ms = sum(step_ms) / len(step_ms)
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    peak_hbm, _ = measured_peaks()
    kin_bytes = 12.0 * n_events
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (accept-reject from I per channel on the GPU; flat MC from a seeded device generator)",
        "config": {"workload": f"uneven: {len(chans)} channels, K ~ U{{4..48}}, N_data log-U[1e4, 4e6] (sum {n_data}), "
                               f"N_MC = 5 N_data (sum {n_events - n_data}), 2 floating masses + 2 floating widths per "
                               "channel; one step = f and the gradient in (V, M, Gamma) of every channel in one "
                               "persistent launch, every amplitude recomputed from the kinematics",
                   "channels": len(chans), "N_data_total": n_data, "N_MC_total": n_events - n_data,
                   "units": "data events (the MC events are streamed in the same step and not counted)",
                   "l2": f"inputs ({kin_bytes / 1e9:.1f} GB of kinematics) larger than L2",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": job_rate(n_data, world, e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "what": "pinned H2D of every channel's data and MC kinematics, V and theta; the persistent "
                        "evaluation; D2H of f and the gradient"},
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": ffma, "unit": "TFLOP/s", "frac": achieved / ffma,
                     "traffic": None, "kernel": "k_uneven (persistent, all channels)", "flops_per_launch": flops,
                     "kernel_us": kernel_ms * 1e3,
                     "peak_kind": "measured now: FFMA microbenchmark (libpwa_peaks.so), FP32 SIMT",
                     "hbm_frac": kin_bytes / (kernel_ms * 1e-3) / 1e9 / peak_hbm,
                     "design": "recompute from kinematics (12 bytes per event); FP32-bound"},
        "clocks": sampler.summary(), "status": pwa.status_string(ok), "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline_uneven(chans, args.cpu_seconds)
    h.close()
    return res


# ----------------------------------------------------------------------------- oracle arm
def oracle_sample(wl_name, n_sample, n_sets=4):
    """The first n_sample events of the workload's wave set for the oracle, with n_sets of its
    parameter sets.  The events are flat phase-space points (the oracle's cost does not depend on
    where they lie; it consumes complex64 amplitudes exactly like the GPU path)."""
    import oracle
    from paper_1108_5882_gb300 import inputs
    K, N, NMC, P, seed = WORKLOADS[wl_name]
    ws = inputs.wave_set_plain(seed) if wl_name == "plain" else inputs.wave_set_spread(K, seed)
    V_true = inputs.production_amplitudes(K, seed)
    kin = inputs.kinematics(n_sample, seed, 4)
    A = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin).astype(np.complex64)
    kin_mc = inputs.kinematics(min(n_sample, 100_000), seed, 5)
    Psi = oracle.normint(oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin_mc).astype(np.complex64))
    if P == 1:
        V = V_true[None, :]
    else:
        V = inputs.starts(min(P, n_sets), K, seed)
    return A, V, Psi, N, P


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform module)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(wl, seconds):
    """The oracle on every data event of the workload and min(P, 4) of its parameter sets, repeated
    for about `seconds`; a full iteration (all P sets) is extrapolated linearly in the sets."""
    import oracle
    name = [k for k, v in WORKLOADS.items() if v[0] == wl["K"] and v[1] == wl["N"]][0]
    K, N, NMC, P, seed = WORKLOADS[name]
    A, V, Psi, _, _ = oracle_sample(name, N, n_sets=min(P, 4))
    evals = 0
    t0 = time.perf_counter()
    while True:
        oracle.nll_grad(A, V, Psi, n_factor=float(N))
        evals += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    ps = V.shape[0]
    full_s = dt / evals * P / ps
    sample = (f"{evals} FP64 -lnL+gradient evaluations of all {A.shape[1]} data events x {ps} of the {P} parameter "
              f"sets (K={K}), {dt:.1f} s")
    if ps < P:
        sample += f"; one full iteration ({P} sets) extrapolated linearly from {ps}/{P} of the sets: {full_s:.1f} s"
    return {"value": A.shape[1] * ps * evals / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
            "cpu_model": cpu_model(), "nproc": os.cpu_count(), "full_iteration_s": full_s,
            "full_iteration_extrapolated": ps < P}


def run_reference_uneven(args, world):
    """The oracle arm of the uneven workload: each step evaluates the smallest channel in full
    (FP64 amplitudes with derivatives, then f and the gradient in V, M and Gamma) on flat events."""
    import oracle
    from paper_1108_5882_gb300 import inputs
    n_ch, seed = UNEVEN
    specs = inputs.uneven_channels(n_ch, seed)
    c = min(range(n_ch), key=lambda i: (specs[i][1] + specs[i][2]) * specs[i][0])
    K, N, NMC = specs[c]
    ws = inputs.wave_set_spread(K, seed, stream=100 + c)
    V = inputs.production_amplitudes(K, seed, stream=200 + c)
    kin, kin_mc = inputs.kinematics(N, seed, 300 + c), inputs.kinematics(NMC, seed, 400 + c)
    fwave, fkind = [0, K // 2, 0, K // 2], [0, 0, 1, 1]

    def one():
        A, dM, dW = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin, derivs=True)
        Am, dMm, dWm = oracle.amplitudes(ws.J, ws.lam, ws.M, ws.W, kin_mc, derivs=True)
        dA = np.stack([(dM if k == 0 else dW)[r] for r, k in zip(fwave, fkind)]).astype(np.complex64)
        dAm = np.stack([(dMm if k == 0 else dWm)[r] for r, k in zip(fwave, fkind)]).astype(np.complex64)
        oracle.nll_grad_shape(A.astype(np.complex64), dA, Am.astype(np.complex64), dAm, fwave, V, n_factor=float(N))

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = N * args.steps / dt
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": f"each step: the smallest of {n_ch} channels (K={K}, N_data={N}, N_MC={NMC}) in full"}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"uneven: {n_ch} channels (oracle on its smallest channel per step)"},
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    if args.workload == "uneven":
        return run_reference_uneven(args, world)
    K, N, NMC, P, seed = WORKLOADS[args.workload]
    n_s = min(N, 100_000 if P == 1 else 250_000)
    A, V, Psi, _, _ = oracle_sample(args.workload, n_s, n_sets=4)
    for _ in range(args.warmup):
        oracle.nll_grad(A, V, Psi, n_factor=float(N))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.nll_grad(A, V, Psi, n_factor=float(N))
    dt = time.perf_counter() - t0
    value = A.shape[1] * V.shape[0] * args.steps / dt
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": f"each step: FP64 -lnL+gradient of the first {A.shape[1]} of {N} events x {V.shape[0]} of "
                     f"{P} set(s)"}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{args.workload}: K={K}, N_data={N}, P={P} (oracle on a "
                                                        f"bounded sample of {A.shape[1]} events)",
                                             "K": K, "N_data": N, "P": P},
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="multistart", choices=sorted(WORKLOADS) + ["uneven"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        res = run_reference(args, world, rank)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    world, rank, local = dist_init(args.gpus)
    res = (run_uneven if args.workload == "uneven" else run_ours)(args, world, rank, local)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
