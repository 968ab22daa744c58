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
# ncu DRAM-traffic summaries, one per kernel: (file, sources whose hash it records)
TRAFFIC_FILES = {
    "k_xft_fused<12, float>": ("traffic_xft_fused_f32_n4096.json", KERNEL_SOURCES),
    "k_xft_split<12, bf16, 3 products>": ("traffic_xft_split_bf16_n4096.json", SPLIT_SOURCES),
    "k_xft_split<12, fp16, 3 products>": ("traffic_xft_split_fp16_n4096.json", SPLIT_SOURCES),
    "k_xft_split<12, fp16, 1 product>": ("traffic_xft_split_fp16x1_n4096.json", SPLIT_SOURCES),
}


PRECISIONS = {"native": 0, "split_bf16": 1, "split_fp16": 2, "fp16": 3}
DTYPES = {"native": "f32", "split_bf16": "bf16 hi+lo operands, f32 accumulate",
          "split_fp16": "f16 hi+lo operands, f32 accumulate", "fp16": "f16 operands, f32 accumulate"}
VARIANT_KERNELS = {0: "k_xft_fused<12, float>", 1: "k_xft_fused_tma<12, false>",
                   2: "k_xft_fused_tma<12, true>", 3: "k_xft_pair<12, 2>", 4: "k_xft_pair_tma<12>",
                   5: "k_xft_cluster", 6: "k_xft_pair<12, 2, 3>",
                   7: "k_xft_pass_a + k_xft_pass_b (two passes)"}
SPLIT_KERNELS = {"split_bf16": "k_xft_split<12, bf16, 3 products>",
                 "split_fp16": "k_xft_split<12, fp16, 3 products>",
                 "fp16": "k_xft_split<12, fp16, 1 product>"}


def kernel_name(variant, precision):
    return VARIANT_KERNELS[variant] if variant is not None else SPLIT_KERNELS[precision]


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
    ap.add_argument("--variant", default="auto", choices=["auto", "0", "1", "2", "3", "4", "5", "6", "7"],
                    help="fused kernel variant (auto: the library's autotuner)")
    ap.add_argument("--precision", default="native",
                    choices=["native", "split_bf16", "split_fp16", "fp16"],
                    help="native: FP32 fused kernel (headline); split_*/fp16: the DFT passes "
                         "on the tensor cores")
    ap.add_argument("--workload", default="uniform", choices=["uniform", "ragged", "fields2d", "backward"],
                    help="uniform: 16384 x N=4096 (headline); ragged: 20000 mixed-N, mixed-kind "
                         "instances in one graph launch; fields2d: separable 2-D LCT forward + "
                         "backward on 8 fields of 2048 x 2048; backward: lct_backward (adjoint "
                         "+ per-signal parameter gradients) on the 16384 x N=4096 batch")
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


def traffic_per_launch(n_points: int, kernel: str):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, if
    it was taken on the current kernel source (else None), scaled to this
    launch size."""
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
# ragged workload: 20000 instances, N = 2^6..2^16, four kinds, one graph launch
# ---------------------------------------------------------------------------
def ragged_arm(args, rank, world, lct, torch, barrier, max_over_ranks):
    """The 20000-instance batch.  Under torchrun every rank builds the same
    global batch and transforms its share from lct_partition (cost-balanced,
    largest first): strong scaling, no collective on the data path."""
    r = W.ragged_plan(seed=W.SEED_RAGGED)
    M = len(r["kind"])
    Ns = (1 << r["log2n"]).astype(np.int64)
    abcd = r["abcd"].copy()
    for s in np.nonzero(r["kind"] == W.KIND_FRFT)[0]:
        z = complex(r["z"][s])
        abcd[s] = [(z + 1 / z) / 2, (1 / z - z) / 2j, 1j * (1 / z - z) / 2, (z + 1 / z) / 2]
    owner, load = lct.lct_partition(Ns, world, abcd)
    mine = np.nonzero(owner == rank)[0]
    offs = np.concatenate([[0], np.cumsum(Ns[mine])[:-1]]).astype(np.int64)
    local = int(Ns[mine].sum())
    buf = np.empty(local, dtype=np.complex64)
    rng = r["rng"]
    pos = {int(s): k for k, s in enumerate(mine)}
    for s in range(M):                       # the draw order defines the workload
        sig = W.ragged_signal(lct.lct_input_grid(int(Ns[s])), r["s"][s], r["q"][s], rng)
        if s in pos:
            k = pos[s]
            buf[offs[k]:offs[k] + Ns[s]] = sig
    plan = lct.Plan.batch(Ns[mine], abcd[mine], offs, dtype=lct.LCT_C64)
    # one kernel per (N, kind) group in the graph (b = 0 signals form their own groups)
    n_groups = len({(int(Ns[s]), bool(abcd[s][1] == 0)) for s in mine})
    d_in = torch.from_numpy(buf).cuda()
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream()
    count = len(mine)
    for _ in range(args.warmup):
        plan.execute(d_in, d_out, count, stream)
    torch.cuda.synchronize()
    if lct.lct_device_status(plan.handle) != 0:
        raise RuntimeError("device status after warm-up")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        plan.execute(d_in, d_out, count, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1)) / args.steps
    plan.destroy()
    total = int(Ns.sum())
    value = total / (ms * 1e-3)
    peak, peak_kind = measured_peak()
    achieved = total * BYTES_PER_POINT / world / (ms * 1e-3) / 1e9     # per GPU
    if rank == 0:
        by_n = {int(n): int((Ns == n).sum()) for n in np.unique(Ns)}
        print(json.dumps({
            "metric": "LCT points/s, ragged batch (20000 instances, N=2^6..2^16, 4 kinds)",
            "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "ragged: 20000 instances (9000 generic, 5000 complex-z FrFT, "
                                   "4000 Fourier, 2000 b=0), log2 N ~ U{6..16}, seed %d" % W.SEED_RAGGED,
                       "points": total, "signals_by_N": by_n,
                       "sharding": "lct_partition over %d ranks (cost N log2 N, largest first); "
                                   "load imbalance %.2e" % (world, load.max() / load.mean() - 1),
                       "l2": "inputs larger than L2 (1.9 GB per buffer at one GPU)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind},
            "gpu_launches": args.steps * n_groups,
        }), flush=True)


# ---------------------------------------------------------------------------
# 2-D fields: forward + backward (input gradient and (a, b, d) per axis)
# ---------------------------------------------------------------------------
def fields2d_arm(args, rank, world, lct, torch, barrier, max_over_ranks):
    """8 complex64 fields of 2048 x 2048 (Gaussian beam x bicubic phase
    screen).  One step = lct2d_execute (rows, then columns) + lct2d_backward
    (columns, then rows, each with the parameter-gradient sums) for a fixed
    upstream gradient dl/dG of the intensity loss sum (|G|^2 - I)^2."""
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
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(args.steps):
        fwd()
        ev[2 * k + 1].record(stream)
        bwd()
        ev[2 * k + 2].record(stream)
    torch.cuda.synchronize()
    barrier()
    f_ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)) / args.steps
    b_ms = sum(ev[2 * k + 1].elapsed_time(ev[2 * k + 2]) for k in range(args.steps)) / args.steps
    f_ms, b_ms = max_over_ranks(f_ms), max_over_ranks(b_ms)
    ms = f_ms + b_ms
    lct.lct2d_plan_destroy(plan)
    pts = B * n * n
    peak, peak_kind = measured_peak()
    fwd_bytes, bwd_bytes = 32 * pts, 64 * pts     # see the docstring of the phases below
    phases = {
        "forward": {"ms": f_ms, "kernels": "k_xft_fused<11, float> rows + k_xft_cols<11, G=4> columns",
                    "algorithmic_bytes": fwd_bytes, "achieved_gbs": fwd_bytes / (f_ms * 1e-3) / 1e9},
        "backward": {"ms": b_ms, "kernels": "k_xft_cols<11, G=4> adjoint+gradient columns, then k_xft_gen<11> "
                                            "rows; two gradient finalize kernels",
                     "algorithmic_bytes": bwd_bytes, "achieved_gbs": bwd_bytes / (b_ms * 1e-3) / 1e9},
    }
    achieved = bwd_bytes / (b_ms * 1e-3) / 1e9
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
            "gpu_launches": 6 * args.steps,
        }), flush=True)


# ---------------------------------------------------------------------------
# 1-D backward on the headline batch
# ---------------------------------------------------------------------------
def backward_arm(args, rank, world, lct, torch, barrier, max_over_ranks):
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
    for name, grad_abd, bpp in [("with_param_grads", gp, 32), ("adjoint_only", None, 16)]:
        def step():
            lct.lct_backward(plan.handle, g, d_in, d_out, gin, grad_abd, count, stream)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1)) / args.steps
        res[name] = {"ms": ms, "algorithmic_bytes": bpp * count * N,
                     "achieved_gbs": bpp * count * N / (ms * 1e-3) / 1e9}
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

    if args.workload == "ragged":
        return ragged_arm(args, rank, world, lct, torch, barrier, max_over_ranks)
    if args.workload == "fields2d":
        return fields2d_arm(args, rank, world, lct, torch, barrier, max_over_ranks)
    if args.workload == "backward":
        return backward_arm(args, rank, world, lct, torch, barrier, max_over_ranks)
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

    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
        time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1))
    ms_per_step = ms_total / args.steps
    # Clock samples need ~1 s under load; if the K steps were shorter, the same
    # launch loop continues for 1.5 s and the samples come from both.
    clock_note = "timed region"
    if t_wall1 - t_wall0 < 1.0 and not args.no_clocks:
        t_end = time.time() + 1.5
        while time.time() < t_end:
            for _ in range(50):
                step()
            torch.cuda.synchronize()
        t_wall1 = time.time()
        clock_note = "timed region + 1.5 s continuation of the same launch loop"
    clocks = sampler.summary(t_wall0, t_wall1)
    sampler.stop()
    if clocks is not None:
        clocks["window"] = clock_note

    value = world * n_points / (ms_per_step * 1e-3)
    peak, peak_kind = measured_peak()
    achieved = n_points * BYTES_PER_POINT / (ms_per_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": traffic_per_launch(n_points, kernel_name(variant, args.precision)),
                "kernel": kernel_name(variant, args.precision) + " (N=4096, complex64)",
                "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                "algorithmic_bytes_per_launch": n_points * BYTES_PER_POINT}

    # plain FP64 path on the same batch
    plain = None
    if not args.no_plain:
        plan.set_precision(lct.LCT_PREC_PLAIN64)
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
        plain = {"value": world * n_points / (pms * 1e-3), "unit": "points/s", "ms_per_step": pms,
                 "path": "chirp kernel + cuFFT Z2Z + chirp kernel, FP64 workspace"}
        torch.cuda.synchronize()
        # release the plain path's workspace
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
               "api": "lct_execute_host on pinned host buffers (32 MiB chunks: copy-in, transform, "
                      "copy-out pipelined on three streams)"}

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
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
