#!/usr/bin/env python3
"""Throughput benchmark of the fused LCT (XFT) kernel.

Workload (default): 16384 complex64 signals of N = 4096 samples, per-signal
parameters from generator G1 (a, d ~ U[-2, 2], |b| ~ U[0.2, 2] with random
sign, c = (ad - 1)/b; Gaussian-windowed random chirps plus 1e-3 noise), one
batch plan.  One step = one lct_execute over the whole batch (the whole hot
path: chirp, 4096-point DFT, chirp + scale, in one kernel).  Inputs are
resident in HBM; each buffer (512 MiB) is larger than L2.

Reported next to it: the plain FP64 GPU path (chirp kernel, cuFFT Z2Z,
chirp kernel) on the same batch, an end-to-end number with host buffers,
and the CPU oracle (O(N^2) FP64) on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own batch (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "LCT points/s at N=4096 batched vs plain FP64 GPU path at <=1e-5 rel err; %HBM"
N_DEFAULT, COUNT_DEFAULT = 4096, 16384
BYTES_PER_POINT = 16          # complex64: 8 B read + 8 B written
FALLBACK_HBM_GBS = 6800.0
COMMON_SOURCES = ["paper_0912_1379_gb300/csrc/xft_common.cuh", "paper_0912_1379_gb300/csrc/xft_engine.cuh",
                  "paper_0912_1379_gb300/csrc/xft_chirp.cuh", "paper_0912_1379_gb300/csrc/xft_async.cuh"]
KERNEL_SOURCES = ["paper_0912_1379_gb300/csrc/k_fused.cu", "paper_0912_1379_gb300/csrc/k_fused_pair.cu"] + COMMON_SOURCES
SPLIT_SOURCES = ["paper_0912_1379_gb300/csrc/k_split.cu"] + COMMON_SOURCES
SPLIT_UMMA_SOURCES = ["paper_0912_1379_gb300/csrc/k_split_umma.cu", "paper_0912_1379_gb300/csrc/xft_umma.cuh",
                      "paper_0912_1379_gb300/csrc/umma_desc.h"] + COMMON_SOURCES
# ncu DRAM-traffic summaries, one per kernel: (file, sources whose hash it records)
TRAFFIC_FILES = {
    "k_xft_fused<12, float>": ("traffic_xft_fused_f32_n4096.json", KERNEL_SOURCES),
    "k_xft_split<12, bf16, 3 products>": ("traffic_xft_split_bf16_n4096.json", SPLIT_SOURCES),
    "k_xft_split_umma (tcgen05, bf16, 3 products)": ("traffic_xft_split_umma_bf16_n4096.json",
                                                     SPLIT_UMMA_SOURCES),
    "k_xft_split_umma (tcgen05, fp16, 3 products)": ("traffic_xft_split_umma_fp16_n4096.json",
                                                     SPLIT_UMMA_SOURCES),
    "k_xft_split_umma (tcgen05, fp16, 1 product)": ("traffic_xft_split_umma_fp16x1_n4096.json",
                                                    SPLIT_UMMA_SOURCES),
    "k_xft_split<12, fp16, 3 products>": ("traffic_xft_split_fp16_n4096.json", SPLIT_SOURCES),
    "k_xft_split<12, fp16, 1 product>": ("traffic_xft_split_fp16x1_n4096.json", SPLIT_SOURCES),
}


PRECISIONS = {"native": 0, "split_bf16": 1, "split_fp16": 2, "fp16": 3}
DTYPES = {"native": "f32", "split_bf16": "bf16 hi+lo operands, f32 accumulate",
          "split_fp16": "f16 hi+lo operands, f32 accumulate", "fp16": "f16 operands, f32 accumulate"}
VARIANT_KERNELS = {0: "k_xft_fused<12, float>", 1: "k_xft_fused_tma<12, false>",
                   2: "k_xft_fused_tma<12, true>", 3: "k_xft_pair<12, 2>", 4: "k_xft_pair_tma<12>",
                   5: "k_xft_cluster", 6: "k_xft_pair<12, 2, 3>",
                   7: "k_xft_pass_a + k_xft_pass_b (two passes)", 8: "k_xft_fused_tmat<12>",
                   10: "k_xft_fused<12, float, packed, radix 8>",
                   11: "k_xft_fused<12, float, one signal per CTA>"}
SPLIT_KERNELS = {"split_bf16": "k_xft_split<12, bf16, 3 products>",
                 "split_fp16": "k_xft_split<12, fp16, 3 products>",
                 "fp16": "k_xft_split<12, fp16, 1 product>"}


def kernel_name(variant, precision):
    if variant is not None:
        return VARIANT_KERNELS[variant]
    if os.environ.get("LCT_SPLIT_KERNEL", "") != "mma":          # the library's default
        return {"split_bf16": "k_xft_split_umma (tcgen05, bf16, 3 products)",
                "split_fp16": "k_xft_split_umma (tcgen05, fp16, 3 products)",
                "fp16": "k_xft_split_umma (tcgen05, fp16, 1 product)"}[precision]
    return SPLIT_KERNELS[precision]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--count", type=int, default=COUNT_DEFAULT)
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 path")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-clocks", action="store_true", help="skip clock sampling (profiler runs)")
    ap.add_argument("--variant", default="auto", choices=["auto", "0", "1", "2", "3", "4", "5", "6", "7", "8", "9", "10", "11"],
                    help="fused kernel variant (auto: the library's autotuner)")
    ap.add_argument("--nonpow2-n", type=int, default=3000,
                    help="nonpow2 workload: N (7-smooth: mixed radix; else chirp convolution)")
    ap.add_argument("--ragged-scale", type=float, default=1.0,
                    help="ragged workload: scale of every kind's count (1.0: the 20000-instance batch)")
    ap.add_argument("--precision", default="native",
                    choices=["native", "split_bf16", "split_fp16", "fp16"],
                    help="native: FP32 fused kernel (headline); split_*/fp16: the DFT passes "
                         "on the tensor cores")
    ap.add_argument("--workload", default="uniform",
                    choices=["uniform", "ragged", "fields2d", "backward", "config0", "uniform1024",
                             "hermite", "nonpow2", "mehler"],
                    help="uniform: 16384 x N=4096 (headline); ragged: 20000 mixed-N, mixed-kind "
                         "instances in one graph launch; fields2d: separable 2-D LCT forward + "
                         "backward on 8 fields of 2048 x 2048; backward: lct_backward (adjoint "
                         "+ per-signal parameter gradients) on the 16384 x N=4096 batch; config0: "
                         "12 x N=256 complex128 latency; uniform1024: 4096 x N=1024 (L2 flushed); "
                         "hermite: the Hermite-zero FrFT of eq. (tmat), 4096 x N=1024; nonpow2: "
                         "16384 x N=3000; mehler: complex-z FrFT on the real nodes (eq. (primcuad)), 16384 x N=4096")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def kernel_hash(sources=None) -> str:
    h = hashlib.sha256()
    for rel in (KERNEL_SOURCES if sources is None else sources):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_profile(kernel: str):
    """The committed ncu summary of `kernel` if it was taken on the current
    kernel source, else None."""
    if kernel not in TRAFFIC_FILES:
        return None
    fname, sources = TRAFFIC_FILES[kernel]
    try:
        with open(os.path.join(ROOT, "profiles", fname)) as fh:
            j = json.load(fh)
    except Exception:
        return None
    if j.get("kernel_hash") != kernel_hash(sources) or j.get("kernel") != kernel:
        return None
    return j


def traffic_per_launch(n_points: int, kernel: str):
    """DRAM bytes per launch of `kernel` from its committed ncu summary,
    scaled to this launch size (None without a current summary)."""
    j = kernel_profile(kernel)
    if j is None:
        return None
    per_point = float(j["dram_bytes"]) / float(j["points"])
    return per_point * n_points


# ---------------------------------------------------------------------------
# clocks: nvidia-smi sampled in the background
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.t is not None:
                self.t.join(timeout=5)

    def summary(self, t0: float, t1: float):
        sm, smax, reasons = [], [], set()
        for ts, line in self.lines:
            if not (t0 <= ts <= t1):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def timed_loop(torch, step, steps, stream, device_index, barrier, max_over_ranks, no_clocks=False):
    """Time `steps` calls of step() with CUDA events on `stream` (barrier and
    synchronize on both sides, max over ranks), sampling the SM clocks with
    nvidia-smi during the timed region.  If the region lasts under a second,
    the same launch loop continues for 1.5 s so that the clock record has
    samples under load.  Returns (ms per step, clocks summary or None)."""
    sampler = ClockSampler(device_index)
    if not no_clocks:
        sampler.start()
        time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1)) / steps
    note = "timed region"
    if t_wall1 - t_wall0 < 1.0 and not no_clocks:
        t_end = time.time() + 1.5
        while time.time() < t_end:
            for _ in range(max(1, min(200, int(50.0 / max(ms, 1e-3))))):
                step()
            torch.cuda.synchronize()
        t_wall1 = time.time()
        note = "timed region + 1.5 s continuation of the same launch loop"
    clocks = sampler.summary(t_wall0, t_wall1)
    sampler.stop()
    if clocks is not None:
        clocks["window"] = note
    return ms, clocks


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def cpu_oracle_rate(x, params, f, min_seconds: float = 10.0, max_signals: int = 1024):
    import oracle as O
    O.build()
    done, t0 = 0, time.perf_counter()
    chunk = 8
    outs = []
    while done < max_signals:
        s = slice(done, done + chunk)
        outs.append(O.lct(f[s].astype(np.complex128), params[s]))
        done += f[s].shape[0]
        if time.perf_counter() - t0 >= min_seconds or done >= f.shape[0]:
            break
    dt = time.perf_counter() - t0
    N = f.shape[1]
    return done * N / dt, done, dt, O.num_threads(), np.concatenate(outs)


def reference_arm(args, rank, world):
    """The CPU oracle as the reference implementation (rank 0 only)."""
    if rank != 0:
        return
    import oracle as O
    N = args.n
    O.build()
    x = O.nodes(N)
    per_step = 2
    count = per_step * (args.steps + args.warmup)
    params, f = W.uniform_batch(x, count, seed=W.SEED_UNIFORM_4096, dtype=np.complex64)
    f64 = f.astype(np.complex128)
    for s in range(args.warmup):
        sl = slice(s * per_step, (s + 1) * per_step)
        O.lct(f64[sl], params[sl])
    t0 = time.perf_counter()
    for s in range(args.warmup, args.warmup + args.steps):
        sl = slice(s * per_step, (s + 1) * per_step)
        O.lct(f64[sl], params[sl])
    dt = time.perf_counter() - t0
    value = args.steps * per_step * N / dt
    sample = "%d signals of N=%d per step from the G1 workload (seed %d)" % (per_step, N, W.SEED_UNIFORM_4096)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "uniform batch N=4096 complex64, G1 per-signal parameters (bounded sample)",
                   "N": N},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": O.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# shared pieces of the secondary arms
# ---------------------------------------------------------------------------
def rel_l2_rows(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return np.linalg.norm(got - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


def accuracy_block(err, against):
    err = np.atleast_1d(np.asarray(err, dtype=np.float64))
    return {"rel_l2_max": float(err.max()), "rel_l2_median": float(np.median(err)),
            "signals": int(err.size), "against": against}


def flush_l2(torch, scratch):
    """Write a buffer larger than L2 (129 MB), so the next launch reads its
    inputs from HBM."""
    scratch.add_(1)


def per_step_flushed(torch, step, steps, stream, scratch, barrier, max_over_ranks):
    """Mean of `steps` per-launch CUDA-event intervals on `stream`, with L2
    flushed outside the timed intervals (for inputs that fit in L2)."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    barrier()
    torch.cuda.synchronize()
    for e0, e1 in evs:
        flush_l2(torch, scratch)
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    times = [e0.elapsed_time(e1) for e0, e1 in evs]
    return max_over_ranks(sum(times) / steps), max_over_ranks(statistics.median(times))


# ---------------------------------------------------------------------------
# ragged workload: 20000 instances, N = 2^6..2^16, four kinds, one graph launch
# ---------------------------------------------------------------------------
def ragged_arm(args, rank, world, lct, torch, barrier, max_over_ranks, local):
    """The 20000-instance batch.  Under torchrun every rank builds the same
    global batch and transforms its share from lct_partition (cost-balanced,
    largest first): strong scaling, no collective on the data path."""
    r = W.ragged_plan(count_scale=args.ragged_scale, seed=W.SEED_RAGGED)
    M = len(r["kind"])
    Ns = (1 << r["log2n"]).astype(np.int64)
    abcd = r["abcd"].copy()
    for s in np.nonzero(r["kind"] == W.KIND_FRFT)[0]:
        z = complex(r["z"][s])
        abcd[s] = [(z + 1 / z) / 2, (1 / z - z) / 2j, 1j * (1 / z - z) / 2, (z + 1 / z) / 2]
    owner, load = lct.lct_partition(Ns, world, abcd)
    mine = np.nonzero(owner == rank)[0]
    offs = np.concatenate([[0], np.cumsum(Ns[mine])[:-1]]).astype(np.int64)
    local_pts = int(Ns[mine].sum())
    buf = np.empty(local_pts, dtype=np.complex64)
    rng = r["rng"]
    pos = {int(s): k for k, s in enumerate(mine)}
    for s in range(M):                       # the draw order defines the workload
        sig = W.ragged_signal(lct.lct_input_grid(int(Ns[s])), r["s"][s], r["q"][s], rng)
        if s in pos:
            k = pos[s]
            buf[offs[k]:offs[k] + Ns[s]] = sig
    # autotuned schedule: each N of the batch is tuned once on a uniform batch of
    # its own signal count (synthetic G1 signals); the ragged graph's groups then
    # take the tuned kernel variant / schedule from the library's cache
    schedules = {}
    if args.variant == "auto":
        for n in sorted({int(v) for v in Ns[mine]}):
            cnt = int((Ns[mine] == n).sum())
            tp, tf = W.uniform_batch(lct.lct_input_grid(n), cnt, seed=W.SEED_RAGGED + n,
                                     dtype=np.complex64)
            tplan = lct.Plan.batch([n] * cnt, tp, np.arange(cnt, dtype=np.int64) * n,
                                   dtype=lct.LCT_C64)
            t_in = torch.from_numpy(tf).cuda()
            t_out = torch.empty_like(t_in)
            schedules[n] = tplan.autotune(t_in, t_out, cnt, torch.cuda.current_stream())
            tplan.destroy()
            del t_in, t_out
    plan = lct.Plan.batch(Ns[mine], abcd[mine], offs, dtype=lct.LCT_C64)
    persistent = args.variant == "9"
    if persistent:
        plan.set_variant(9)              # one persistent launch over a work queue
    # one kernel per (N, kind) group in the graph (b = 0 signals form their own groups)
    n_groups = 1 if persistent else len({(int(Ns[s]), bool(abcd[s][1] == 0)) for s in mine})
    d_in = torch.from_numpy(buf).cuda()
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream()
    count = len(mine)

    def step():
        plan.execute(d_in, d_out, count, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if lct.lct_device_status(plan.handle) != 0:
        raise RuntimeError("device status after warm-up")
    ms, clocks = timed_loop(torch, step, args.steps, stream, local, barrier, max_over_ranks,
                            args.no_clocks)
    total = int(Ns.sum())
    value = total / (ms * 1e-3)
    peak, peak_kind = measured_peak()
    achieved = total * BYTES_PER_POINT / world / (ms * 1e-3) / 1e9     # per GPU
    accuracy = cpu = None
    if rank == 0 and not args.no_cpu:
        # one signal of every (kind, N) owned here, N up to 32768: the oracle
        # on those (bounded CPU time) and the GPU output against it
        import oracle as O
        O.build()
        G = d_out.cpu().numpy()
        errs, pts, t_cpu = [], 0, 0.0
        kind_names = {W.KIND_GENERIC: "generic", W.KIND_FRFT: "frft", W.KIND_FOURIER: "fourier",
                      W.KIND_B0: "b0"}
        worst = {}
        for kind in range(4):
            for log2n in range(6, 16):
                cand = [k for k, s in enumerate(mine) if r["kind"][s] == kind and r["log2n"][s] == log2n]
                if not cand:
                    continue
                k = cand[0]
                s = mine[k]
                N = int(Ns[s])
                f = buf[offs[k]:offs[k] + N].astype(np.complex128)
                t0 = time.perf_counter()
                ref = O.lct(f, abcd[s])
                t_cpu += time.perf_counter() - t0
                pts += N
                e = float(rel_l2_rows(G[offs[k]:offs[k] + N], ref))
                errs.append(e)
                key = kind_names[kind]
                worst[key] = max(worst.get(key, 0.0), e)
        accuracy = accuracy_block(errs, "FP64 oracle, one signal of every (kind, N <= 32768)")
        accuracy["rel_l2_max_by_kind"] = worst
        cpu = {"value": pts / t_cpu, "unit": "points/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": "one signal of every (kind, N = 64..32768) of the workload: %d signals, "
                         "%d points, %.1f s (O(N^2) per signal)" % (len(errs), pts, t_cpu)}
    plan.destroy()
    if rank == 0:
        by_n = {int(n): int((Ns == n).sum()) for n in np.unique(Ns)}
        print(json.dumps({
            "metric": "LCT points/s, ragged batch (%d instances, N=2^6..2^16, 4 kinds)" % M,
            "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "ragged: %d instances (%s), log2 N ~ U{6..16}, seed %d"
                                   % (M, ", ".join("%d %s" % (int((r["kind"] == k).sum()), nm) for k, nm in
                                                   ((W.KIND_GENERIC, "generic"), (W.KIND_FRFT, "complex-z FrFT"),
                                                    (W.KIND_FOURIER, "Fourier"), (W.KIND_B0, "b=0"))),
                                      W.SEED_RAGGED),
                       "points": total, "signals_by_N": by_n,
                       "autotuned_variant_by_N": schedules or None,
                       "sharding": "lct_partition over %d ranks (cost N log2 N, largest first); "
                                   "load imbalance %.2e" % (world, load.max() / load.mean() - 1),
                       "l2": "inputs larger than L2 (%.2f GB per buffer at one GPU), no flush" % (total * 8 / 1e9),
                       "launch": "one persistent kernel over a largest-first work queue" if persistent
                                 else "CUDA graph: one kernel per N group + one b = 0 launch"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": ("k_xft_ragged (persistent, all items)" if persistent else
                                    "whole graph (one kernel per N group + b = 0 chunks)") + ", 16 B/point"},
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": args.steps * n_groups,
        }), flush=True)


# ---------------------------------------------------------------------------
# 2-D fields: forward + backward (input gradient and (a, b, d) per axis)
# ---------------------------------------------------------------------------
def fields2d_arm(args, rank, world, lct, torch, barrier, max_over_ranks, local):
    """8 complex64 fields of 2048 x 2048 (Gaussian beam x bicubic phase
    screen).  One step = lct2d_execute (rows, then columns) + lct2d_backward
    (columns, then rows, each with the parameter-gradient sums) for a fixed
    upstream gradient dl/dG of the intensity loss sum (|G|^2 - I)^2.
    Forward and backward are timed as two loops of their own (each clocked);
    the step time is their sum."""
    B, n = 8, 2048
    x = lct.lct_input_grid(n)
    fields, ax, ay = W.fields_batch(x, B, seed=W.SEED_FIELDS + rank)
    plan = lct.lct2d_plan_create(n, n, ay, ax, lct.LCT_C64)
    stream = torch.cuda.current_stream()
    xf = torch.from_numpy(fields.astype(np.complex64)).cuda()
    mid, out = torch.empty_like(xf), torch.empty_like(xf)
    gmid, gin = torch.empty_like(xf), torch.empty_like(xf)
    gp = torch.zeros(6, dtype=torch.float64, device="cuda")
    lct.lct2d_execute(plan, xf, mid, out, B, stream)
    target = (out.abs() ** 2).roll(shifts=(7, -5), dims=(1, 2))      # a shifted intensity
    g = (2 * (out.abs() ** 2 - target) * 2 * out).contiguous()       # dl/dG*, fixed
    torch.cuda.synchronize()

    def fwd():
        lct.lct2d_execute(plan, xf, mid, out, B, stream)

    def bwd():
        lct.lct2d_backward(plan, g, xf, mid, out, gmid, gin, gp, B, stream)

    for _ in range(args.warmup):
        fwd()
        bwd()
    torch.cuda.synchronize()
    f_ms, f_clocks = timed_loop(torch, fwd, args.steps, stream, local, barrier, max_over_ranks,
                                args.no_clocks)
    b_ms, b_clocks = timed_loop(torch, bwd, args.steps, stream, local, barrier, max_over_ranks,
                                args.no_clocks)
    fwd()
    torch.cuda.synchronize()
    ms = f_ms + b_ms
    pts = B * n * n
    peak, peak_kind = measured_peak()
    fwd_bytes, bwd_bytes = 32 * pts, 64 * pts
    phases = {
        "forward": {"ms": f_ms, "kernels": "k_xft_fused<11, float> rows + k_xft_cols<11, G=4> columns",
                    "algorithmic_bytes": fwd_bytes, "achieved_gbs": fwd_bytes / (f_ms * 1e-3) / 1e9,
                    "frac": fwd_bytes / (f_ms * 1e-3) / 1e9 / peak, "clocks": f_clocks},
        "backward": {"ms": b_ms, "kernels": "k_xft_cols<11, G=4> adjoint+gradient columns, then k_xft_gen<11> "
                                            "rows; two gradient finalize kernels",
                     "algorithmic_bytes": bwd_bytes, "achieved_gbs": bwd_bytes / (b_ms * 1e-3) / 1e9,
                     "frac": bwd_bytes / (b_ms * 1e-3) / 1e9 / peak, "clocks": b_clocks},
    }
    achieved = bwd_bytes / (b_ms * 1e-3) / 1e9
    accuracy = cpu = None
    if rank == 0 and not args.no_cpu:
        # each pass against the oracle on sampled lines: rows of the row
        # pass (mid) from the input, columns of the column pass (out) from the
        # GPU's own mid; the oracle rate on those 1-D transforms is the CPU
        # baseline (a 2-D point needs two of them)
        import oracle as O
        O.build()
        h_in, h_mid, h_out = xf.cpu().numpy(), mid.cpu().numpy(), out.cpu().numpy()
        errs, pts_cpu, t_cpu = [], 0, 0.0
        rng = np.random.default_rng(5)
        k = 0
        while (t_cpu < 10.0 and k < 256) or k < 16:
            b = int(rng.integers(B))
            line = int(rng.integers(n))
            t0 = time.perf_counter()
            if k % 2 == 0:
                ref = O.lct(h_in[b, line, :].astype(np.complex128), ax)
                got = h_mid[b, line, :]
            else:
                ref = O.lct(h_mid[b, :, line].astype(np.complex128), ay)
                got = h_out[b, :, line]
            t_cpu += time.perf_counter() - t0
            pts_cpu += n
            errs.append(float(rel_l2_rows(got, ref)))
            k += 1
        accuracy = accuracy_block(errs, "FP64 oracle on sampled rows (row pass) and columns "
                                        "(column pass, from the GPU's row-pass output)")
        rate_1d = pts_cpu / t_cpu
        cpu = {"value": rate_1d / 2, "unit": "points/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": "%d random rows/columns of 2048 (O(N^2) each), %.1f s; 2-D forward "
                         "points/s = 1-D rate / 2 (forward only)" % (k, t_cpu)}
    lct.lct2d_plan_destroy(plan)
    if rank == 0:
        print(json.dumps({
            "metric": "2-D LCT forward + backward points/s (8 x 2048 x 2048 complex64)",
            "value": world * pts / (ms * 1e-3), "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "fields2d: 8 fields 2048 x 2048, Gaussian beam x bicubic 64x64 "
                                   "phase screen, G1 (a,b,c,d) per axis, seed %d" % W.SEED_FIELDS,
                       "points": pts,
                       "l2": "inputs larger than L2 (256 MiB per buffer), no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "backward phase (k_xft_cols + k_xft_gen launches: each reads g, "
                                   "G, f and writes h, 32 B/pt)"},
            "phases": phases,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "clocks": b_clocks,
            "gpu_launches": 6 * args.steps,
        }), flush=True)


# ---------------------------------------------------------------------------
# 1-D backward on the headline batch
# ---------------------------------------------------------------------------
def backward_arm(args, rank, world, lct, torch, barrier, max_over_ranks, local):
    """One step = lct_backward of the 16384 x 4096 batch plan: grad_in =
    L^H g and (dl/da, dl/db, dl/dd) per signal (the adjoint kernel with the
    gradient sums reads g, f and G and writes grad_in: 32 B/point)."""
    N, count = args.n, args.count
    x = lct.lct_input_grid(N)
    params, f = W.uniform_batch(x, count, seed=W.SEED_UNIFORM_4096 + rank, dtype=np.complex64)
    plan = lct.Plan.batch([N] * count, params, np.arange(count, dtype=np.int64) * N, dtype=lct.LCT_C64)
    stream = torch.cuda.current_stream()
    d_in = torch.from_numpy(f).cuda()
    d_out = torch.empty_like(d_in)
    plan.execute(d_in, d_out, count, stream)
    g = torch.randn(d_in.shape, dtype=torch.complex64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(7))
    gin = torch.empty_like(d_in)
    gp = torch.zeros(3 * count, dtype=torch.float64, device="cuda")
    res = {}
    clocks = None
    for name, grad_abd, bpp in [("with_param_grads", gp, 32), ("adjoint_only", None, 16)]:
        def step():
            lct.lct_backward(plan.handle, g, d_in, d_out, gin, grad_abd, count, stream)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ms, ck = timed_loop(torch, step, args.steps, stream, local, barrier, max_over_ranks,
                            args.no_clocks)
        if clocks is None:
            clocks = ck
        res[name] = {"ms": ms, "algorithmic_bytes": bpp * count * N,
                     "achieved_gbs": bpp * count * N / (ms * 1e-3) / 1e9, "clocks": ck}
    # leave the with-gradient results in gin and gp for the accuracy check
    lct.lct_backward(plan.handle, g, d_in, d_out, gin, gp, count, stream)
    torch.cuda.synchronize()
    accuracy = cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle as O
        O.build()
        ks = 8
        gg = g[:ks].cpu().numpy().astype(np.complex128)
        ff = f[:ks].astype(np.complex128)
        t0 = time.perf_counter()
        h_ref = O.lct_adjoint(gg, params[:ks])
        p_ref = O.lct_grad_params(ff, gg, params[:ks])
        t_cpu = time.perf_counter() - t0
        err_h = rel_l2_rows(gin[:ks].cpu().numpy(), h_ref)
        p_got = gp[:3 * ks].cpu().numpy().reshape(ks, 3)
        err_p = np.abs(p_got - p_ref).max(axis=1) / np.abs(p_ref).max(axis=1)
        accuracy = accuracy_block(err_h, "FP64 oracle adjoint (grad_in) on the first %d signals" % ks)
        accuracy["param_grad_rel_max"] = float(err_p.max())
        accuracy["param_grad_against"] = "oracle dense-matrix gradient (max |error| / max |grad| per signal)"
        cpu = {"value": ks * N / t_cpu, "unit": "points/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": "first %d signals: O(N^2) adjoint + dense-matrix parameter gradient, %.1f s"
                         % (ks, t_cpu)}
    plan.destroy()
    peak, peak_kind = measured_peak()
    main = res["with_param_grads"]
    if rank == 0:
        print(json.dumps({
            "metric": "LCT backward points/s (adjoint + parameter gradients), 16384 x N=4096",
            "value": world * count * N / (main["ms"] * 1e-3), "unit": "points/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "backward: uniform batch %d x N=%d complex64, G1 per-signal "
                                   "(a,b,c,d), seed %d; g ~ CN(0,1)" % (count, N, W.SEED_UNIFORM_4096),
                       "l2": "inputs larger than L2 (512 MiB per buffer), no flush"},
            "roofline": {"bound": "hbm", "achieved": main["achieved_gbs"], "peak": peak,
                         "unit": "GB/s", "frac": main["achieved_gbs"] / peak, "traffic": None,
                         "peak_kind": peak_kind,
                         "kernel": "k_xft_gen<12, float, adjoint, gradient sums> (+ finalize)"},
            "phases": res,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": 2 * args.steps,
        }), flush=True)


# ---------------------------------------------------------------------------
# small configurations: 12 x 256 complex128 (latency) and 4096 x 1024
# complex64 (fits in L2: flushed between launches)
# ---------------------------------------------------------------------------
def config0_arm(args, rank, world, lct, torch, barrier, max_over_ranks, local):
    """The FP64 case: the polynomial e^{-x^2/2}(1 + 0.3x + 0.1x^3) and the
    Hermite functions psi_0..psi_10 (12 signals of N = 256, complex128),
    rotation angle 0.7.  One step = one lct_execute; microseconds per batch
    (launch and latency bound), L2 flushed between launches."""
    N = 256
    x = lct.lct_input_grid(N)
    f = W.config0_signals(x)
    abcd = W.config0_params()
    B = f.shape[0]
    plan = lct.Plan.create(N, *abcd, dtype=lct.LCT_C128)
    stream = torch.cuda.current_stream()
    d_in = torch.from_numpy(f).cuda()
    d_out = torch.empty_like(d_in)
    scratch = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")    # 256 MiB > L2

    def step():
        plan.execute(d_in, d_out, B, stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    steps = max(args.steps, 50)
    mean_ms, med_ms = per_step_flushed(torch, step, steps, stream, scratch, barrier, max_over_ranks)
    _, clocks = timed_loop(torch, step, steps, stream, local, barrier, max_over_ranks, args.no_clocks)
    G = d_out.cpu().numpy()
    plain_us = None
    if not args.no_plain:
        pp = lct.Plan.create(N, *abcd, dtype=lct.LCT_C128).set_precision(lct.LCT_PREC_PLAIN64)
        o2 = torch.empty_like(d_in)
        for _ in range(3):
            pp.execute(d_in, o2, B, stream)
        pm, _ = per_step_flushed(torch, lambda: pp.execute(d_in, o2, B, stream), steps, stream,
                                 scratch, barrier, max_over_ranks)
        plain_us = pm * 1e3
        pp.destroy()
    accuracy = cpu = None
    if rank == 0:
        import oracle as O
        O.build()
        reps, t0 = 0, time.perf_counter()
        while True:
            ref = O.lct(f, abcd)
            reps += 1
            if time.perf_counter() - t0 > 2.0:
                break
        t_cpu = (time.perf_counter() - t0) / reps
        accuracy = accuracy_block(rel_l2_rows(G, ref), "FP64 oracle, all 12 signals")
        if not args.no_cpu:
            cpu = {"value": t_cpu * 1e6, "unit": "us per batch", "cores": O.num_threads(),
                   "kind": "oracle", "sample": "the whole batch (12 x 256), %d repetitions" % reps}
    plan.destroy()
    if rank == 0:
        print(json.dumps({
            "metric": "LCT latency, 12 x N=256 complex128 (FP64), rotation 0.7",
            "value": mean_ms * 1e3, "unit": "us per batch", "n_gpus": world, "steps": steps,
            "warmup": max(3, args.warmup), "ms_per_step": mean_ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "config0: e^{-x^2/2}(1+0.3x+0.1x^3) + psi_0..psi_10, N=256, "
                                   "complex128, (a,b,c,d) = rotation 0.7",
                       "median_us": med_ms * 1e3,
                       "l2": "L2 flushed (256 MiB write) before every timed launch",
                       "kernel": "k_xft_fused<8, double, one signal per CTA>"},
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "plain64_us": plain_us,
            "clocks": clocks,
            "gpu_launches": steps,
        }), flush=True)


def uniform1024_arm(args, rank, world, lct, torch, barrier, max_over_ranks, local):
    """4096 complex64 signals of N = 1024, G1 per-signal parameters (seed
    1001).  The 32 MiB input fits in L2, so L2 is flushed before every timed
    launch; one step = one lct_execute."""
    N, count = 1024, 4096
    x = lct.lct_input_grid(N)
    params, f = W.uniform_batch(x, count, seed=W.SEED_UNIFORM_1024 + rank, dtype=np.complex64)
    plan = lct.Plan.batch([N] * count, params, np.arange(count, dtype=np.int64) * N, dtype=lct.LCT_C64)
    stream = torch.cuda.current_stream()
    d_in = torch.from_numpy(f).cuda()
    d_out = torch.empty_like(d_in)
    scratch = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")
    variant = plan.autotune(d_in, d_out, count, stream)

    def step():
        plan.execute(d_in, d_out, count, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    steps = max(args.steps, 50)
    mean_ms, med_ms = per_step_flushed(torch, step, steps, stream, scratch, barrier, max_over_ranks)
    _, clocks = timed_loop(torch, step, steps, stream, local, barrier, max_over_ranks, args.no_clocks)
    G = d_out.cpu().numpy()
    plains = {}
    if not args.no_plain:
        for name, prec in [("plain64", lct.LCT_PREC_PLAIN64), ("plain32", lct.LCT_PREC_PLAIN32)]:
            pp = lct.Plan.batch([N] * count, params, np.arange(count, dtype=np.int64) * N,
                                dtype=lct.LCT_C64).set_precision(prec)
            o2 = torch.empty_like(d_in)
            for _ in range(3):
                pp.execute(d_in, o2, count, stream)
            pm, _ = per_step_flushed(torch, lambda: pp.execute(d_in, o2, count, stream), steps,
                                     stream, scratch, barrier, max_over_ranks)
            plains[name] = {"ms_per_step": pm, "value": world * count * N / (pm * 1e-3),
                            "unit": "points/s"}
            pp.destroy()
    accuracy = cpu = None
    if rank == 0 and not args.no_cpu:
        rate, nsig, dt, cores, ref = cpu_oracle_rate(x, params, f)
        cpu = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
               "sample": "first %d signals of the %d x N=%d workload, %.1f s" % (nsig, count, N, dt)}
        accuracy = accuracy_block(rel_l2_rows(G[:nsig], ref), "FP64 oracle on the cpu_baseline sample")
    plan.destroy()
    peak, peak_kind = measured_peak()
    achieved = count * N * BYTES_PER_POINT / (mean_ms * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "LCT points/s at N=1024 batched (4096 signals, complex64); %HBM",
            "value": world * count * N / (mean_ms * 1e-3), "unit": "points/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "uniform batch 4096 x N=1024 complex64, G1 per-signal (a,b,c,d), "
                                   "seed %d" % W.SEED_UNIFORM_1024,
                       "median_ms": med_ms, "kernel_variant": variant,
                       "l2": "L2 flushed (256 MiB write) before every timed launch"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "k_xft_fused<10, float> (variant %s)" % variant},
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "baselines": plains,
            "clocks": clocks,
            "gpu_launches": steps,
        }), flush=True)

# ---------------------------------------------------------------------------
# Hermite-zero discrete fractional transform (Sec. 2, eq. (tmat))
# ---------------------------------------------------------------------------
FP64_NOMINAL_TFLOPS = 1.25            # GB300 FP64 (nominal, CUDA cores)
FP32_DERIVED_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max clock


def tf32_peak_tflops():
    """Dense TF32 tensor peak: the measured BF16 burst rate times the nominal
    TF32/BF16 ratio (1.1 / 2.25 PFLOP/s), else the nominal 1.1 PFLOP/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
        return bf16 * 1.1 / 2.25, "measured bf16 burst x nominal tf32/bf16 (1.1/2.25)"
    except Exception:
        return 1100.0, "nominal dense tf32"


def hermite_arm(args, rank, world, lct, torch, barrier, max_over_ranks, local):
    """F_z = sqrt(2 pi) U^T D(z) U applied to a batch of signals sampled at
    the zeros of H_N: two real-by-complex products of N x N by N x batch
    (8 N^2 flops per signal), FP64 for complex128 (the headline of this arm)
    and FP32 for complex64.  The basis is built once before timing."""
    N, B = 1024, 4096
    z = np.exp(-0.7j)
    x, _ = lct.frft_hermite_basis(N, with_matrix=False)
    rng = W.rng_for(W.SEED_UNIFORM_1024 + 17 + rank)
    env = np.exp(-x * x / 6.0)
    f = (env * (rng.standard_normal((B, N)) + 1j * rng.standard_normal((B, N)))).astype(np.complex128)
    stream = torch.cuda.current_stream()
    res = {}
    clocks = None
    outs = {}
    for name, dt, code in [("c128", np.complex128, lct.LCT_C128), ("c64", np.complex64, lct.LCT_C64)]:
        d_in = torch.from_numpy(f.astype(dt)).cuda()
        d_out = torch.empty_like(d_in)

        def step():
            lct.frft_hermite_execute(N, z, d_in, d_out, B, code, stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        steps = max(3, min(args.steps, 10)) if name == "c128" else args.steps
        ms, ck = timed_loop(torch, step, steps, stream, local, barrier, max_over_ranks, args.no_clocks)
        flops = 8.0 * N * N * B
        if name == "c128":
            res[name] = {"ms": ms, "steps": steps, "tflops": flops / (ms * 1e-3) / 1e12,
                         "peak_tflops": FP64_NOMINAL_TFLOPS,
                         "frac": flops / (ms * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS,
                         "kernel": "k_herm_gemm<double> (CUDA cores)", "clocks": ck}
        else:
            # tensor cores: split TF32, three products per useful one
            tf32_peak = tf32_peak_tflops()
            tensor = 3.0 * flops / (ms * 1e-3) / 1e12
            res[name] = {"ms": ms, "steps": steps, "tflops": flops / (ms * 1e-3) / 1e12,
                         "tensor_tflops": tensor, "peak_tflops": tf32_peak[0],
                         "peak_kind": tf32_peak[1], "frac": tensor / tf32_peak[0],
                         "fp32_simt_peak_tflops": FP32_DERIVED_TFLOPS,
                         "kernel": "k_herm_umma (tcgen05.mma kind::tf32, 3 split products)",
                         "clocks": ck}
        if clocks is None:
            clocks = ck
        outs[name] = d_out[:64].cpu().numpy()
    accuracy = cpu = None
    if rank == 0 and not args.no_cpu:
        from oracle import hermite as H
        t0 = time.perf_counter()
        _, F = H.hermite_zero_frft(N, z)
        ref = f[:64] @ F.T
        t_cpu = time.perf_counter() - t0
        e64 = rel_l2_rows(outs["c128"], ref)
        e32 = rel_l2_rows(outs["c64"], f[:64].astype(np.complex64).astype(np.complex128) @ F.T)
        accuracy = accuracy_block(e64, "oracle B (eigensolver basis, dense F_z), first 64 signals, complex128")
        accuracy["complex64_rel_l2_max"] = float(e32.max())
        cpu = {"value": 64 * N / t_cpu, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "oracle B: tridiagonal eigensolver + dense F_z (N = %d) + 64 signals, %.2f s"
                         % (N, t_cpu)}
    main = res["c128"]
    if rank == 0:
        print(json.dumps({
            "metric": "Hermite-zero discrete FrFT (eq. tmat) points/s, N=1024, complex128 (FP64)",
            "value": world * B * N / (main["ms"] * 1e-3), "unit": "points/s", "n_gpus": world,
            "steps": main["steps"], "warmup": args.warmup, "ms_per_step": main["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "hermite: %d signals x N=%d at the zeros of H_N, Gaussian-windowed "
                                   "complex noise, z = e^{-0.7i}" % (B, N),
                       "l2": "inputs larger than L2 (64 MiB complex128 in + out + 64 MiB workspace; "
                             "U 8 MiB stays in L2), no flush"},
            "roofline": {"bound": "alu", "achieved": main["tflops"], "peak": FP64_NOMINAL_TFLOPS,
                         "unit": "TFLOP/s", "frac": main["frac"], "traffic": None,
                         "peak_kind": "nominal GB300 FP64 rate (1.25 TFLOP/s)",
                         "kernel": "k_herm_gemm<double> x 2 (8 N^2 flops per signal)"},
            "phases": res,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": 2 * main["steps"],
        }), flush=True)


# ---------------------------------------------------------------------------
# N that is not a power of two (chirp convolution of length M >= 2N - 1)
# ---------------------------------------------------------------------------
def nonpow2_arm(args, rank, world, lct, torch, barrier, max_over_ranks, local):
    """16384 complex64 signals of N = 3000 (default; --nonpow2-n), G1
    per-signal parameters; one step = one lct_execute.  7-smooth N (3000 =
    2^3 3 5^3) runs the mixed-radix kernel (chirp, DFT_N in passes of radix
    8, 5, 5, 5, 3, chirp); other N the chirp convolution (pre-chirp, FFT_M,
    spectrum, inverse FFT_M, post-chirp, M >= 2N - 1)."""
    N, count = args.nonpow2_n, 16384
    smooth = N
    for q in (2, 3, 5, 7):
        while smooth % q == 0:
            smooth //= q
    M = 1
    while M < 2 * N - 1:
        M *= 2
    kernel = ("k_xft_mixed<float> (16 B/point; one mixed-radix DFT of N per signal)" if smooth == 1 else
              "k_xft_blue<%d, float> (16 B/point; two FFTs of M = %d per signal)" % (M.bit_length() - 1, M))
    x = lct.lct_input_grid(N)
    params, f = W.uniform_batch(x, count, seed=W.SEED_UNIFORM_4096 + 31 + rank, dtype=np.complex64)
    plan = lct.Plan.batch([N] * count, params, np.arange(count, dtype=np.int64) * N, dtype=lct.LCT_C64)
    stream = torch.cuda.current_stream()
    d_in = torch.from_numpy(f).cuda()
    d_out = torch.empty_like(d_in)

    def step():
        plan.execute(d_in, d_out, count, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if lct.lct_device_status(plan.handle) != 0:
        raise RuntimeError("device status after warm-up")
    ms, clocks = timed_loop(torch, step, args.steps, stream, local, barrier, max_over_ranks,
                            args.no_clocks)
    accuracy = cpu = None
    if rank == 0 and not args.no_cpu:
        rate, nsig, dt, cores, ref = cpu_oracle_rate(x, params, f, min_seconds=10.0)
        cpu = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
               "sample": "first %d signals of the %d x N=%d workload, %.1f s" % (nsig, count, N, dt)}
        accuracy = accuracy_block(rel_l2_rows(d_out[:nsig].cpu().numpy(), ref),
                                  "FP64 oracle on the cpu_baseline sample")
    plan.destroy()
    pts = count * N
    peak, peak_kind = measured_peak()
    achieved = pts * BYTES_PER_POINT / (ms * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "LCT points/s at N=%d (not a power of two), 16384 signals complex64; %%HBM" % N,
            "value": world * pts / (ms * 1e-3), "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "nonpow2: 16384 x N=%d complex64, G1 per-signal (a,b,c,d)" % N,
                       "path": "mixed radix" if smooth == 1 else "chirp convolution, M = %d" % M,
                       "l2": "inputs larger than L2 (%d MB per buffer), no flush" % (count * N * 8 // 10**6)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": kernel},
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": args.steps,
        }), flush=True)


# ---------------------------------------------------------------------------
# complex-z fractional transform on the real nodes (eqs. (fasy), (primcuad))
# ---------------------------------------------------------------------------
MEHLER_Z = 0.6 * complex(np.cos(2.2), np.sin(2.2))


def mehler_arm(args, rank, world, lct, torch, barrier, max_over_ranks, local):
    """16384 complex64 signals of N = 4096 at z = 0.6 e^{2.2i} (Re z < 0: the
    reversed form); one step = one frft_mehler_execute (the lag kernel's
    spectrum, one CTA, then the weighted convolution of length M = 8192)."""
    import oracle as O
    N, count = 4096, 16384
    z = MEHLER_Z
    x = lct.lct_input_grid(N)
    _, f = W.uniform_batch(x, count, seed=W.SEED_UNIFORM_4096 + 47 + rank, dtype=np.complex64)
    stream = torch.cuda.current_stream()
    d_in = torch.from_numpy(f).cuda()
    d_out = torch.empty_like(d_in)

    def step():
        lct.frft_mehler_execute(N, z, d_in, d_out, count, lct.LCT_C64, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms, clocks = timed_loop(torch, step, args.steps, stream, local, barrier, max_over_ranks,
                            args.no_clocks)
    accuracy = cpu = None
    if rank == 0 and not args.no_cpu:
        O.build()
        # bounded sample: calls of 4 signals (each forms its N^2 kernel entries)
        # until 10 s of CPU work
        nsig, refs, t0 = 0, [], time.perf_counter()
        while nsig < 64 and (nsig == 0 or time.perf_counter() - t0 < 10.0):
            refs.append(O.frft_mehler(f[nsig:nsig + 4].astype(np.complex128), z))
            nsig += 4
        dt = time.perf_counter() - t0
        ref = np.concatenate(refs)
        cpu = {"value": nsig * N / dt, "unit": "points/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": "first %d signals of the %d x N=%d workload (dense eq. (fasy) rows, "
                         "N^2 kernel entries per call), %.1f s" % (nsig, count, N, dt)}
        accuracy = accuracy_block(rel_l2_rows(d_out[:nsig].cpu().numpy(), ref),
                                  "FP64 oracle (dense Riemann sum) on the cpu_baseline sample")
    pts = count * N
    peak, peak_kind = measured_peak()
    achieved = pts * BYTES_PER_POINT / (ms * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "complex-z FrFT points/s on the real nodes at N=4096, 16384 signals complex64; %HBM",
            "value": world * pts / (ms * 1e-3), "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "mehler: 16384 x N=4096 complex64 G1 signals, z = 0.6 e^{2.2i}",
                       "M": 8192, "l2": "inputs larger than L2 (512 MiB per buffer), no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "k_xft_blue<13, float, Mehler> (16 B/point; two FFTs of M = 8192 "
                                   "per signal) + k_mehler_spectrum (one CTA)"},
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": 2 * args.steps,
        }), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    import paper_0912_1379_gb300 as lct

    lct.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    arms = {"ragged": ragged_arm, "fields2d": fields2d_arm, "backward": backward_arm,
            "config0": config0_arm, "uniform1024": uniform1024_arm, "hermite": hermite_arm,
            "nonpow2": nonpow2_arm, "mehler": mehler_arm}
    if args.workload in arms:
        arms[args.workload](args, rank, world, lct, torch, barrier, max_over_ranks, local)
        if dist is not None:
            dist.destroy_process_group()
        return
    N, count = args.n, args.count
    x = lct.lct_input_grid(N)
    params, f = W.uniform_batch(x, count, seed=W.SEED_UNIFORM_4096 + rank, dtype=np.complex64)
    plan = lct.Plan.batch([N] * count, params, np.arange(count, dtype=np.int64) * N, dtype=lct.LCT_C64)
    prec_code = PRECISIONS[args.precision]
    h_in = torch.from_numpy(f).pin_memory()
    d_in = h_in.cuda()
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream()
    n_points = count * N

    def step():
        plan.execute(d_in, d_out, count, stream)

    if prec_code != lct.LCT_PREC_NATIVE:
        variant = None
        plan.set_precision(prec_code)
    elif args.variant == "auto":
        variant = plan.autotune(d_in, d_out, count, stream)
    else:
        variant = int(args.variant)
        plan.set_variant(variant)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    status = lct.lct_device_status(plan.handle)
    if status != 0:
        raise RuntimeError("device status %d after warm-up" % status)

    ms_per_step, clocks = timed_loop(torch, step, args.steps, stream, local, barrier,
                                     max_over_ranks, args.no_clocks)

    value = world * n_points / (ms_per_step * 1e-3)
    peak, peak_kind = measured_peak()
    achieved = n_points * BYTES_PER_POINT / (ms_per_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": traffic_per_launch(n_points, kernel_name(variant, args.precision)),
                "kernel": kernel_name(variant, args.precision) + " (N=4096, complex64)",
                "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                "algorithmic_bytes_per_launch": n_points * BYTES_PER_POINT}
    if args.precision != "native":
        # tensor-pipe activity of the same kernel source (ncu, one launch)
        prof = kernel_profile(kernel_name(variant, args.precision))
        if prof is not None and "tensor_pipe_active_pct" in prof:
            roofline["tensor_pipe_active_pct"] = prof["tensor_pipe_active_pct"]

    # the unfused paths on the same batch: FP64 (the named comparison) and FP32
    plain = plain32 = None
    if not args.no_plain:
        for prec in (lct.LCT_PREC_PLAIN64, lct.LCT_PREC_PLAIN32):
            plan.set_precision(prec)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            pms = max_over_ranks(e0.elapsed_time(e1)) / args.steps
            if prec == lct.LCT_PREC_PLAIN64:
                plain = {"value": world * n_points / (pms * 1e-3), "unit": "points/s",
                         "ms_per_step": pms,
                         "path": "chirp kernel + cuFFT Z2Z + chirp kernel, FP64 workspace"}
            else:
                plain32 = {"value": world * n_points / (pms * 1e-3), "unit": "points/s",
                           "ms_per_step": pms,
                           "path": "FP32 chirp kernel + cuFFT C2C + FP32 chirp kernel (unfused, "
                                   "same arithmetic as the fused kernel)"}
        torch.cuda.synchronize()
        # release the plain paths' workspace
        plan.destroy()
        plan = lct.Plan.batch([N] * count, params, np.arange(count, dtype=np.int64) * N, dtype=lct.LCT_C64)
        if variant is None:
            plan.set_precision(prec_code)
        else:
            plan.set_variant(variant)
        step()
        torch.cuda.synchronize()

    # end to end with host buffers: H2D copy, transform, D2H copy per step
    e2e = None
    if not args.no_e2e:
        h_out = torch.empty_like(h_in).pin_memory()

        def e2e_step():
            plan.execute_host(h_in, h_out, count, stream)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1)) / args.steps
        nbytes = count * N * 8
        e2e = {"value": world * n_points / (ems * 1e-3), "unit": "points/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": ems,
               "api": "lct_execute_host on pinned host buffers (mapped page-locked memory: the "
                      "kernels read the input and write the output over the host link in place; "
                      "the bytes above cross it every step)"}

    cpu = None
    accuracy = None
    if rank == 0 and not args.no_cpu:
        torch.cuda.synchronize()
        rate, nsig, dt, cores, ref = cpu_oracle_rate(x, params, f)
        cpu = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
               "sample": "first %d signals of the %d x N=%d workload, %.1f s" % (nsig, count, N, dt)}
        got = d_out[:nsig].cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        accuracy = {"rel_l2_max": float(err.max()), "rel_l2_median": float(np.median(err)),
                    "signals": int(nsig), "against": "FP64 oracle on the cpu_baseline sample"}

    plan.destroy()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic",
            "config": {"workload": "uniform batch %d x N=%d complex64, G1 per-signal (a,b,c,d), seed %d"
                                   % (count, N, W.SEED_UNIFORM_4096),
                       "signals_per_gpu": count, "N": N, "transforms_per_s": value / N,
                       "precision": args.precision, "kernel_variant": variant,
                       "l2": "inputs larger than L2 (512 MiB per buffer), no flush",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clocks,
            "plain64": plain,
            "speedup_vs_plain64": (plain["ms_per_step"] / ms_per_step) if plain else None,
            "plain32": plain32,
            "speedup_vs_plain32": (plain32["ms_per_step"] / ms_per_step) if plain32 else None,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
