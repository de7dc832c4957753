"""Benchmark of the GB300 pair-collision path (one JSON line on stdout).

Default workload (the headline): one step = the three single-set counts of the large
integer configuration, through the C ABI:
  N = 262144 and N = 262145 int32 points uniform in [0,1024)^3, r2 = 9, and the
  same-cell predicate (r2 = 0) on N = 262144 points in [0,256)^3.
metric: G pair-tests/s = sum of N(N-1)/2 over the step / device time of the step.

Also measured in the same run (secondary keys of the JSON line):
  e2e          the same step through the C ABI with host inputs: pinned host->device
               copies and the device->host read of the counts inside the timed region
               (the copies of the next set overlap the count of the current one);
  roofline     dominant kernel (the pair kernel), timed with CUDA events on its stream;
  cpu_baseline the CPU oracle (plain pairwise loop) on the host cores, full step once;
  f32_spheres  N = 131072 FP32 spheres: count and interaction sum;
  batched      ~100k pruned sets in one graph-captured launch vs one plain launch per set;
  serving      Poisson queries through the continuous-batching server vs serial launches.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 run under torchrun (one process per GPU); every rank counts its own
independently seeded sets (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "G pair-tests/s"
WORKLOAD = ("single set N=262144 and N=262145 int32 uniform [0,1024)^3 r2=9, plus same-cell "
            "r2=0 on N=262144 in [0,256)^3 (three counts per step)")
L2_FLUSH_BYTES = 256 << 20


def pairs(n: int) -> int:
    return n * (n - 1) // 2


def step_inputs(rank: int = 0):
    """The three sets of one step; rank > 0 draws independent sets (weak scaling)."""
    sets = []
    for n, same in ((262144, False), (262145, False), (262144, True)):
        c = synth.cfg2(n, same_cell=same) if rank == 0 else _rank_set(n, same, rank)
        sets.append((c["x"], c["y"], c["z"], c["r2"]))
    return sets


def max_over_ranks(vals, dist, device):
    """Element-wise maximum of a list of floats over all ranks (timing only)."""
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def aggregate_value(tests_per_step_per_rank, world, steps, max_ms):
    """Whole-job throughput: the pair tests all ranks processed over the slowest rank's
    time (weak scaling: every rank has the same per-step work)."""
    return tests_per_step_per_rank * world * steps / (max_ms * 1e-3) / 1e9


def _rank_set(n, same, rank):
    bits = 8 if same else 10
    x, y, z = synth.int_points(n, bits, synth.SEED_BASE + 1000 * rank + (100 if same else 0))
    return dict(x=x, y=y, z=z, r2=0 if same else 9)


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons), samples=len(sm))


# ---------------------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    oracle.set_threads(0)
    cores = oracle.get_threads()
    sets = step_inputs(0)
    sample_n = args.ref_sample
    work = [(x[:sample_n], y[:sample_n], z[:sample_n], r2) for (x, y, z, r2) in sets]
    tests = sum(pairs(len(w[0])) for w in work)

    def step():
        return [oracle.count_i32(*w) for w in work]

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = tests * args.steps / dt / 1e9
    sample = (f"first {sample_n} points of each of the three sets of the step "
              f"({tests:.3e} pair tests per step)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": METRIC,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

# Sources of each pair kernel; a committed ncu traffic record is used only while the
# hash of these files matches the one recorded with it.
KERNEL_SOURCES = {
    "fp32": ("paper_1901_11204_gb300/csrc/cc_single.cu", "paper_1901_11204_gb300/csrc/cc_pairs.cuh",
             "paper_1901_11204_gb300/csrc/cc_internal.cuh"),
    "tensor": ("paper_1901_11204_gb300/csrc/cc_tc.cu", "paper_1901_11204_gb300/csrc/cc_tcgen05.cuh",
               "paper_1901_11204_gb300/csrc/cc_internal.cuh"),
}
TRAFFIC_FILES = {"fp32": "k_pairs_traffic.json", "tensor": "k_pairs_tc_traffic.json"}


def kernel_source_hash(kind: str = "fp32") -> str:
    """Hash of the kernel sources with comments and blank space removed: the DRAM counters
    of a capture stay valid while the code they measured is unchanged."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, rel)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", " ", src).encode())
    return h.hexdigest()


def measured_traffic(kind: str = "fp32"):
    """DRAM bytes per launch of the pair kernel from the committed ncu capture, or None
    when the kernel sources changed since that capture."""
    p = os.path.join(ROOT, "profiles", TRAFFIC_FILES[kind])
    if not os.path.exists(p):
        return None, "no capture"
    with open(p) as f:
        d = json.load(f)
    if d.get("source_sha256") != kernel_source_hash(kind):
        return None, "kernel changed since the capture"
    return float(d["dram_bytes_per_launch"]), d.get("workload", "")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


def roofline_peak_int(sms: int, mhz: float) -> float:
    """Pair tests/s bound of the exact-integer kernel: the FP32 pipe does 128 lane-ops per
    clock per SM and the expanded form needs 4 FP32-pipe operations per pair (three
    products as fused multiply-adds and one add of the per-object constant)."""
    return sms * 128.0 * mhz * 1e6 / 4.0


# Tensor-core form: one TF32 contraction of K = 8 terms per pair test (16 flops).
TC_FLOPS_PER_PAIR = 16
# Hardware rates of the tensor-core kernel's own instruction shapes, measured on GB300 with
# python -m paper_1901_11204_gb300.microbench (summary in profiles/): TMEM->register reads
# with eight warps of tcgen05.ld.red.32x32b.x128.min per SM, and back-to-back
# tcgen05.mma kind::tf32 M=128 N=256 K=8 (32768 pair tests each).
TMEM_READ_BYTES_PER_CLK = 870
MMA_CLK_PER_UNIT = 128.2
# The kernel's accumulator hand-over loop with nothing else in it (one issuing thread, two
# 256-column accumulators, eight epilogue warps loading and voting): SM clocks per unit,
# measured by the same tool. Within the kernel's design this is the bound: a shared-memory
# read that the next MMA issue waits for costs the issuing thread about 170-200 clocks.
HANDOVER_CLK_PER_UNIT = 458.0
PAIRS_PER_UNIT = 128 * 256
# TF32 / BF16 dense tensor throughput ratio of the part's nominal figures (1.1 / 2.25 PF).
TF32_PER_BF16 = 1.1 / 2.25


def issue_roofline(sms: int, mhz: float, instr_per_pair: int) -> float:
    """Pair tests/s (in G) at one warp-instruction per clock per SMSP and the stated
    thread-instructions per pair test."""
    return sms * 4 * 32 * mhz * 1e6 / instr_per_pair / 1e9


def roofline_peak_f32(sms: int, mhz: float) -> float:
    """FP32 sphere predicate: 10 FP32-pipe operations per pair (3 sub, 3 mul, 2 add,
    radius add, radius square)."""
    return sms * 128.0 * mhz * 1e6 / 10.0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ref-sample", type=int, default=65536)
    ap.add_argument("--no-extras", action="store_true", help="skip f32/batched/serving/cpu legs")
    ap.add_argument("--serving-queries", type=int, default=50000)
    ap.add_argument("--leg", choices=["config1", "batched", "batched_plan", "f32_spheres", "i32_sums"],
                    help="run only this secondary leg and print its JSON (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1901_11204_gb300 as cc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    cc.build()
    cc.lib()
    stream = torch.cuda.current_stream()
    if args.leg:
        props = torch.cuda.get_device_properties(dev)
        peaks, peak_src = load_peaks()
        fmax = float(peaks.get("sm_max_mhz", 2070.0))
        sms = props.multi_processor_count
        legs = {"config1": lambda: bench_config1(cc, torch, dev, sms, fmax),
                "batched": lambda: bench_batched(cc, torch, dev),
                "batched_plan": lambda: bench_batched(cc, torch, dev, with_plain=False),
                "f32_spheres": lambda: bench_f32(cc, torch, dev, sms, fmax, peak_src, peaks),
                "i32_sums": lambda: bench_i32_sums(cc, torch, dev)}
        print(json.dumps({"leg": args.leg, **legs[args.leg]()}), flush=True)
        return 0

    sets = step_inputs(rank)
    tests_per_step = sum(pairs(len(s[0])) for s in sets)
    dsets = [tuple(torch.from_numpy(a).to(dev) for a in s[:3]) + (s[3],) for s in sets]
    outs = [torch.empty(1, dtype=torch.int64, device=dev) for _ in sets]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    for s in dsets:
        cc.reserve(len(s[0]))

    def step():
        for (x, y, z, r2), o in zip(dsets, outs):
            cc.count_pairs(x, y, z, r2=r2, out=o)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    want = [cc.as_u64(o) for o in outs]
    modes = []
    for (x, y, z, r2), o in zip(dsets, outs):     # which pair kernel the device picks per set
        cc.count_pairs(x, y, z, r2=r2, out=o)
        modes.append(cc.stream_mode())
    tensor = all(m == cc.MODE_TENSOR for m in modes)

    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    cc.profile_enable(True)
    cc.profile_read()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k)          # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    kern_ms, kern_launches = cc.profile_read()
    cc.profile_enable(False)
    clocks = sampler.stop()
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    got = [cc.as_u64(o) for o in outs]
    assert got == want, (got, want)
    assert cc.stream_status() == cc.CC_OK

    if world > 1:
        dev_ms, kern_ms = max_over_ranks([dev_ms, kern_ms], dist, dev)

    ms_per_step = dev_ms / args.steps
    value = aggregate_value(tests_per_step, world, args.steps, dev_ms)

    # ---- roofline of the dominant kernel (pair kernel) ---------------------------------
    peaks, peak_src = load_peaks()
    fmax = float(peaks.get("sm_max_mhz", 2070.0))
    pair_rate = tests_per_step * args.steps / (kern_ms * 1e-3) / 1e9 if kern_ms > 0 else None
    if tensor:
        traffic, traffic_note = measured_traffic("tensor")
        peak = float(peaks.get("bf16_tflops", 1900.0)) * TF32_PER_BF16
        achieved = pair_rate * TC_FLOPS_PER_PAIR / 1e3 if pair_rate else None
        roofline = {
            "bound": "tensor", "kernel": "k_pairs_tc (tcgen05 kind::tf32 pair kernel)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_note": f"ncu dram__bytes_read.sum + dram__bytes_write.sum per launch: {traffic_note}",
            "peak_basis": (f"{peak_src} bf16_tflops {peaks.get('bf16_tflops')} x {TF32_PER_BF16:.3f} "
                           "(nominal TF32/BF16 dense ratio); 16 TF32 flops per pair test"),
            "pair_tests_per_s": pair_rate,
            "kernel_share_of_step": (kern_ms / dev_ms) if dev_ms > 0 else None,
            "kernel_launches": kern_launches,
            "timing_note": "events bracket the tensor-core launch and the FP32-pipe launch that "
                           "returns at once in tensor mode",
        }
        # The kernel's own hardware bounds: every pair test's accumulator is read back from
        # TMEM (4 B per pair), and one MMA evaluates 32768 pair tests. Both measured on this
        # GPU with the kernel's instruction shapes; the kernel runs well below either. Its
        # period is set by the accumulator hand-over loop, measured alone as a third bound.
        tmem_peak = sms * TMEM_READ_BYTES_PER_CLK * fmax * 1e6 / 4.0 / 1e9   # G pair tests/s
        roofline["tmem_read_bound"] = {
            "peak_pair_tests_per_s": tmem_peak,
            "frac": (pair_rate / tmem_peak) if pair_rate else None,
            "basis": (f"{TMEM_READ_BYTES_PER_CLK} B/clk/SM TMEM-to-register reads (eight warps of "
                      f"tcgen05.ld.red.32x32b.x128.min, measured) x {sms} SMs x {fmax:.0f} MHz, "
                      "4 B of accumulator per pair test"),
        }
        mma_peak = sms * PAIRS_PER_UNIT / MMA_CLK_PER_UNIT * fmax * 1e6 / 1e9
        roofline["mma_issue_bound"] = {
            "peak_pair_tests_per_s": mma_peak,
            "frac": (pair_rate / mma_peak) if pair_rate else None,
            "basis": (f"one tcgen05.mma kind::tf32 128x256x8 (32768 pair tests) every {MMA_CLK_PER_UNIT} SM "
                      f"clocks (measured back to back) x {sms} SMs x {fmax:.0f} MHz"),
        }
        hand_peak = sms * PAIRS_PER_UNIT / HANDOVER_CLK_PER_UNIT * fmax * 1e6 / 1e9
        roofline["handover_bound"] = {
            "peak_pair_tests_per_s": hand_peak,
            "frac": (pair_rate / hand_peak) if pair_rate else None,
            "basis": (f"the kernel's accumulator hand-over loop alone (one MMA-issuing thread, two 256-column "
                      f"accumulators, eight epilogue warps loading and voting): {HANDOVER_CLK_PER_UNIT} SM clocks "
                      f"per 32768 pair tests (measured) x {sms} SMs x {fmax:.0f} MHz"),
        }
    else:
        traffic, traffic_note = measured_traffic("fp32")
        peak = roofline_peak_int(sms, fmax) / 1e9
        achieved = pair_rate
        roofline = {
            "bound": "alu", "kernel": "k_pairs_w (FP32-pipe pair kernel)",
            "achieved": achieved, "peak": peak, "unit": METRIC,
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_note": f"ncu dram__bytes_read.sum + dram__bytes_write.sum per launch: {traffic_note}",
            "peak_basis": (f"{sms} SMs x 128 FP32 lanes x {fmax:.0f} MHz ({peak_src} sm_max_mhz) / "
                           "4 FP32-pipe ops per pair"),
            "kernel_share_of_step": (kern_ms / dev_ms) if dev_ms > 0 else None,
            "kernel_launches": kern_launches,
        }
    if achieved and clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / (peak * clocks["sm_mhz"] / fmax)
    # The pair-test roofline in which the work is stated: SMs x 4 SMSPs x 32 lanes x f_SM
    # / 8 thread-instructions per integer pair test (3 sub, 3 mul/mad, compare,
    # accumulate) at one warp-instruction per clock per SMSP.
    issue_peak = issue_roofline(sms, fmax, 8)
    issue_roofline_line = {
        "bound": "issue", "peak": issue_peak, "unit": METRIC, "achieved": pair_rate,
        "frac": (pair_rate / issue_peak) if pair_rate else None,
        "peak_basis": f"{sms} SMs x 4 SMSPs x 32 lanes x {fmax:.0f} MHz / 8 thread-instructions per int pair test",
    }

    # ---- end to end through the C ABI from host buffers -------------------------------
    hsets = [tuple(torch.from_numpy(a).pin_memory() for a in s[:3]) for s in sets]
    hout = torch.empty(len(sets), dtype=torch.int64).pin_memory()
    h2d = sum(sum(t.numel() * t.element_size() for t in hs) for hs in hsets)
    d2h = hout.numel() * hout.element_size()

    # The copies of set k + 1 run on a copy stream while set k is counted: the copy stream
    # starts each step after the step's start event (every copy is inside the timed
    # region) and refills a set's buffers only after the previous count of that set.
    copy_stream = torch.cuda.Stream(device=dev)
    landed = [torch.cuda.Event() for _ in sets]
    counted = [torch.cuda.Event() for _ in sets]

    def e2e_step(start):
        copy_stream.wait_event(start)
        for k, ((hx, hy, hz), (x, y, z, r2)) in enumerate(zip(hsets, dsets)):
            copy_stream.wait_event(counted[k])
            with torch.cuda.stream(copy_stream):
                x.copy_(hx, non_blocking=True)
                y.copy_(hy, non_blocking=True)
                z.copy_(hz, non_blocking=True)
            landed[k].record(copy_stream)
        for k, (x, y, z, r2) in enumerate(dsets):
            stream.wait_event(landed[k])
            cc.count_pairs(x, y, z, r2=r2, out=outs[k])
            counted[k].record(stream)
        for k in range(len(outs)):
            hout[k:k + 1].copy_(outs[k], non_blocking=True)

    for _ in range(2):
        w = torch.cuda.Event()
        w.record(stream)
        e2e_step(w)
    torch.cuda.synchronize()
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k)
        ee[k][0].record(stream)
        e2e_step(ee[k][0])
        ee[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in ee)
    assert [int(v) for v in hout.tolist()] == want
    if world > 1:
        e2e_ms = max_over_ranks([e2e_ms], dist, dev)[0]
    e2e = {"value": aggregate_value(tests_per_step, world, args.steps, e2e_ms), "unit": METRIC,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": e2e_ms / args.steps}

    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "tf32" if tensor else "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "input_dtype": ("int32 (exact: TF32 products of integers with <= 11 significant bits, "
                                   "FP32 sums below 2^24)" if tensor else
                                   "int32 (exact: FP32 arithmetic on integers < 2^24)"),
                   "pair_tests_per_step": tests_per_step, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world} (independent sets per GPU)"},
        "roofline": roofline,
        "issue_roofline": issue_roofline_line,
        "e2e": e2e,
        # per count: reset, min/max + mode, record fill, operand fill, the two tensor-core
        # count forms, the FP32-pipe kernel (the kernels and fill not chosen return at
        # once) and the finalisation kernel
        "gpu_launches": (8 if tensor else 5) * len(sets) * args.steps,
        "pair_kernel_modes": modes,
        "clocks": clocks,
        "wall_s_timed_region": wall,
        "counts": got,
    }

    if rank == 0 and not args.no_extras:
        line["fp32_pipe_step"] = bench_fp32_pipe_step(cc, torch, step, outs, want, tests_per_step,
                                                      roofline_peak_int(sms, fmax) / 1e9, flush)
        line["config1"] = bench_config1(cc, torch, dev, sms, fmax)
        line["f32_spheres"] = bench_f32(cc, torch, dev, sms, fmax, peak_src, peaks)
        line["i32_sums"] = bench_i32_sums(cc, torch, dev)
        line["batched"] = bench_batched(cc, torch, dev)
        line["serving"] = bench_serving(cc, torch, dev, args.serving_queries)
        line["schedule_comparison"] = bench_schedules(cc, torch, dev)
        line["linear_same_site"] = bench_linear(cc, torch, dev, peaks)
        line["cpu_baseline"] = cpu_baseline(sets)

    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def bench_fp32_pipe_step(cc, torch, step, outs, want, tests_per_step, peak, flush, reps=5):
    """The same step with the tensor-core kernel switched off (every count on the FP32
    pipe): what the tensor-core formulation gains on this workload."""
    cc.set_tensor_cores(False)
    try:
        step()
        torch.cuda.synchronize()
        mode = cc.stream_mode()
        stream = torch.cuda.current_stream()
        cc.profile_enable(True)
        cc.profile_read()
        tot = 0.0
        for k in range(reps):
            flush.fill_(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        kern_ms, _ = cc.profile_read()
        cc.profile_enable(False)
        assert [cc.as_u64(o) for o in outs] == want
    finally:
        cc.set_tensor_cores(True)
    value = tests_per_step * reps / (tot * 1e-3) / 1e9
    kern = tests_per_step * reps / (kern_ms * 1e-3) / 1e9 if kern_ms > 0 else None
    return {"value": value, "unit": METRIC, "ms_per_step": tot / reps, "mode": mode,
            "kernel": "k_pairs_w", "kernel_rate": kern, "kernel_frac_of_fp32_pipe_bound": (kern / peak) if kern else None,
            "counts_equal": True}


def _time(fn, reps, torch, stream=None):
    stream = stream or torch.cuda.current_stream()
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _golden_counts():
    out = {}
    path = os.path.join(ROOT, "tests", "golden", "full_size_counts.txt")
    if os.path.exists(path):
        for line in open(path):
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = int(v)
    return out


def bench_config1(cc, torch, dev, sms, fmax, calls=2000):
    """Config 1 (N = 4096 int32 points in [0,64)^3, r2 = 16: one small, latency-bound
    set): the one-launch small-set kernel. Device time per call over back-to-back calls
    (CUDA events), host-observed latency of one call with its synchronisation, the kernel's
    own event-timed duration, and the CPU oracle on the same set; the count must equal the
    oracle's golden value."""
    import oracle
    c = synth.cfg1()
    n = len(c["x"])
    t = [torch.from_numpy(c[k]).to(dev) for k in ("x", "y", "z")]
    out = torch.empty(1, dtype=torch.int64, device=dev)
    cc.count_pairs(*t, r2=c["r2"], out=out)
    torch.cuda.synchronize()
    got = cc.as_u64(out)
    want = _golden_counts().get("cfg1_n4096_r2_16")
    if want is None:
        want = oracle.count_i32(c["x"], c["y"], c["z"], c["r2"])
    assert got == want, (got, want)
    mode = cc.stream_mode()
    ms = _time(lambda: cc.count_pairs(*t, r2=c["r2"], out=out), calls, torch)
    cc.profile_enable(True)
    cc.profile_read()
    for _ in range(200):
        cc.count_pairs(*t, r2=c["r2"], out=out)
    torch.cuda.synchronize()
    kern_ms, kern_n = cc.profile_read()
    cc.profile_enable(False)
    lat = []
    for _ in range(500):
        a = time.perf_counter()
        cc.count_pairs(*t, r2=c["r2"], out=out)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - a)
    oracle.set_threads(1)
    t0 = time.perf_counter()
    reps = 0
    while time.perf_counter() - t0 < 0.5:
        oracle.count_i32(c["x"], c["y"], c["z"], c["r2"])
        reps += 1
    cpu_s = (time.perf_counter() - t0) / reps
    oracle.set_threads(0)
    tests = pairs(n)
    return {"workload": c["name"], "count": got, "count_equals_golden": True, "mode": mode,
            "kernel": "k_small (one launch per call)", "launches_per_call": 1,
            "us_per_call": ms * 1e3, "gpairs_s": tests / (ms * 1e-3) / 1e9,
            "kernel_us": kern_ms / max(kern_n, 1) * 1e3,
            "kernel_gpairs_s": tests / (kern_ms / max(kern_n, 1) * 1e-3) / 1e9 if kern_ms > 0 else None,
            "host_latency_p50_us": float(np.percentile(lat, 50) * 1e6),
            "host_latency_p99_us": float(np.percentile(lat, 99) * 1e6),
            "cpu_oracle_one_core_us": cpu_s * 1e6, "cpu_oracle_gpairs_s": tests / cpu_s / 1e9,
            "issue_roofline_peak": issue_roofline(sms, fmax, 8),
            "note": "latency-bound: 8.4e6 pair tests per call; the roofline fraction is not meaningful"}


def bench_f32(cc, torch, dev, sms, fmax, peak_src, peaks):
    """Config 3 (FP32 spheres): count and sum on the kernel the device chooses (the
    tensor-core screen for this set) and on the FP32-pipe kernel; counts must agree."""
    c = synth.cfg3()
    n = len(c["x"])
    t = [torch.from_numpy(c[k]).to(dev) for k in ("x", "y", "z", "r")]
    legs = {}
    for tc in (True, False):
        cc.set_tensor_cores(tc)
        try:
            ms_c = _time(lambda: cc.count_pairs(t[0], t[1], t[2], r=t[3]), 10, torch)
            cnt_c = cc.as_u64(cc.count_pairs(t[0], t[1], t[2], r=t[3]))
            torch.cuda.synchronize()
            mode = cc.stream_mode()
            ms_s = _time(lambda: cc.interaction_sum(t[0], t[1], t[2], r=t[3]), 10, torch)
            s, cnt = cc.interaction_sum(t[0], t[1], t[2], r=t[3])
            torch.cuda.synchronize()
        finally:
            cc.set_tensor_cores(True)
        g = pairs(n) / (ms_c * 1e-3) / 1e9
        legs["tensor" if tc else "fp32_pipe"] = {
            "mode": mode, "count_ms": ms_c, "count_gpairs_s": g, "sum_ms": ms_s,
            "sum_gpairs_s": pairs(n) / (ms_s * 1e-3) / 1e9, "count": cnt_c, "sum_count": cc.as_u64(cnt),
            "sum": float(s.item())}
    tl, fl = legs["tensor"], legs["fp32_pipe"]
    peak_fp32 = roofline_peak_f32(sms, fmax) / 1e9
    peak_tc = float(peaks.get("bf16_tflops", 1900.0)) * TF32_PER_BF16 * 1e3 / TC_FLOPS_PER_PAIR   # G pair tests/s
    chosen = tl if tl["mode"] == cc.MODE_TENSOR_SPHERES else fl
    g_count = chosen["count_gpairs_s"]
    out = {"workload": f"N={n} FP32 spheres [0,1)^3 r in [0.001,0.004]",
           "kernel": "k_pairs_tc (integer screen + FP32 predicate)" if chosen is tl else "k_pairs_w (FP32 pipe)",
           "count_ms": chosen["count_ms"], "count_gpairs_s": g_count,
           "sum_ms": chosen["sum_ms"], "sum_gpairs_s": chosen["sum_gpairs_s"],
           "count": chosen["count"], "sum": chosen["sum"],
           "counts_equal": tl["count"] == fl["count"] == tl["sum_count"] == fl["sum_count"],
           "sum_rel_diff": abs(tl["sum"] - fl["sum"]) / max(abs(fl["sum"]), 1e-30),
           "tensor": tl, "fp32_pipe": fl,
           "fp32_pipe_roofline_peak": peak_fp32, "fp32_pipe_count_frac": fl["count_gpairs_s"] / peak_fp32,
           "issue_roofline_peak": issue_roofline(sms, fmax, 12),
           "count_frac_of_issue_roofline": g_count / issue_roofline(sms, fmax, 12),
           "peak_basis": (f"FP32 pipe: {sms} SMs x 128 FP32 lanes x {fmax:.0f} MHz ({peak_src}) / 10 FP32 ops per "
                          f"pair; tensor: {peak_tc:.0f} G pair tests/s = measured bf16 x {TF32_PER_BF16:.3f} / "
                          f"{TC_FLOPS_PER_PAIR} TF32 flops per screened pair")}
    if chosen is tl:
        out["tensor_roofline_peak"] = peak_tc
        out["tensor_count_frac"] = g_count / peak_tc
    return out


def bench_i32_sums(cc, torch, dev, n=262144):
    """Interaction sums of integer points on both kernels (tensor-core and FP32 pipe),
    on the headline workload's first set at two hit densities, and the count at the dense
    one (the tensor-core kernel's in-register count form)."""
    c = synth.cfg2(n)
    t = [torch.from_numpy(c[k]).to(dev) for k in ("x", "y", "z")]
    out = {"workload": f"N={n} int32 points uniform in [0,1024)^3"}
    for r2 in (9, 400):
        row = {}
        for tc in (True, False):
            cc.set_tensor_cores(tc)
            try:
                ms = _time(lambda: cc.interaction_sum(t[0], t[1], t[2], r2=r2), 10, torch)
                s, cnt = cc.interaction_sum(t[0], t[1], t[2], r2=r2)
                torch.cuda.synchronize()
                mode = cc.stream_mode()
            finally:
                cc.set_tensor_cores(True)
            row["tensor" if tc else "fp32_pipe"] = {
                "sum_ms": ms, "sum_gpairs_s": pairs(n) / (ms * 1e-3) / 1e9, "mode": mode,
                "count": cc.as_u64(cnt), "sum": float(s.item())}
        a, b = row["tensor"], row["fp32_pipe"]
        row["counts_equal"] = a["count"] == b["count"]
        row["sum_rel_diff"] = abs(a["sum"] - b["sum"]) / max(abs(b["sum"]), 1e-30)
        out[f"r2={r2}"] = row
    # the count at the dense radius: the tensor-core kernel's in-register count form
    row = {}
    for tc in (True, False):
        cc.set_tensor_cores(tc)
        try:
            ms = _time(lambda: cc.count_pairs(t[0], t[1], t[2], r2=400), 10, torch)
            cnt = cc.count_pairs(t[0], t[1], t[2], r2=400)
            torch.cuda.synchronize()
            mode = cc.stream_mode()
        finally:
            cc.set_tensor_cores(True)
        row["tensor" if tc else "fp32_pipe"] = {"count_ms": ms, "count_gpairs_s": pairs(n) / (ms * 1e-3) / 1e9,
                                                "mode": mode, "count": cc.as_u64(cnt)}
    row["counts_equal"] = row["tensor"]["count"] == row["fp32_pipe"]["count"]
    out["count_r2=400"] = row
    return out


def bench_linear(cc, torch, dev, peaks):
    """Algorithm 1 of Section 3 (linear-time same-site collisions) on the GPU, against the
    pairwise kernel with r2 = 0 on the same input (both exact, same count)."""
    out = {}
    for n, bits in ((262144, 8), (16_777_216, 8)):
        x, y, z = synth.int_points(n, bits, synth.SEED_BASE + 102)
        t = [torch.from_numpy(a).to(dev) for a in (x, y, z)]
        ms_lin = _time(lambda: cc.count_same_site(t[0], t[1], t[2]), 20, torch)
        cnt = cc.as_u64(cc.count_same_site(t[0], t[1], t[2]))
        rec = {"n": n, "box": f"[0,{1 << bits})^3", "linear_ms": ms_lin, "count": cnt,
               "beads_per_s": n / (ms_lin * 1e-3),
               # algorithmic bytes per bead: read 3 int32 coordinates (12 B), zero its site
               # (4 B), atomic read-modify-write of the site (4 B read + 4 B write)
               "algorithmic_gbs": 24.0 * n / (ms_lin * 1e-3) / 1e9,
               "hbm_peak_gbs": peaks.get("hbm_gbs")}
        if n <= 262144:
            ms_pair = _time(lambda: cc.count_pairs(t[0], t[1], t[2], r2=0), 5, torch)
            rec["pairwise_ms"] = ms_pair
            rec["speedup_linear_vs_pairwise"] = ms_pair / ms_lin
            rec["pairwise_count_equal"] = cc.as_u64(cc.count_pairs(t[0], t[1], t[2], r2=0)) == cnt
        out[f"n{n}"] = rec
    return out


def bench_schedules(cc, torch, dev, n=600_000):
    """The paper's GPU comparison (Section 5) restated on this GPU: balanced cyclic
    schedule vs the straightforward one (each group of 1024 objects against all later
    objects), same records and inner loop on the FP32 pipe, FP32 spheres of diameter 1,
    N > 525,000. The tensor-core screen's time on the same set is reported beside it."""
    x, y, z, r = synth.unit_spheres(n)
    t = [torch.from_numpy(a).to(dev) for a in (x, y, z, r)]
    cc.set_tensor_cores(False)   # the schedule comparison runs one kernel family
    try:
        ms_cyc = _time(lambda: cc.count_pairs(t[0], t[1], t[2], r=t[3]), 3, torch)
        a = cc.count_pairs(t[0], t[1], t[2], r=t[3])
        torch.cuda.synchronize()
        mode_cyc = cc.stream_mode()
    finally:
        cc.set_tensor_cores(True)
    ms_str = _time(lambda: cc.count_pairs_straightforward(t[0], t[1], t[2], r=t[3]), 3, torch)
    b = cc.count_pairs_straightforward(t[0], t[1], t[2], r=t[3])
    ms_tc = _time(lambda: cc.count_pairs(t[0], t[1], t[2], r=t[3]), 3, torch)
    c = cc.count_pairs(t[0], t[1], t[2], r=t[3])
    torch.cuda.synchronize()
    mode_tc = cc.stream_mode()
    return {"workload": f"N={n} FP32 spheres of diameter 1, centres uniform in [0,200)^3",
            "cyclic_ms": ms_cyc, "straightforward_ms": ms_str, "speedup_cyclic": ms_str / ms_cyc,
            "cyclic_mode": mode_cyc,
            "counts_equal": cc.as_u64(a) == cc.as_u64(b) == cc.as_u64(c), "count": cc.as_u64(a),
            "tensor_screen_ms": ms_tc, "tensor_screen_mode": mode_tc,
            "paper": "1.12x on a Tesla P100 (Section 5), context only"}


def bench_batched(cc, torch, dev, with_plain=True):
    c = synth.cfg4()
    off = c["offsets"]
    S = len(off) - 1
    t = [torch.from_numpy(a).to(dev) for a in (c["x"], c["y"], c["z"], off)]
    tune_path = os.path.join(ROOT, "paper_1901_11204_gb300", "tune_gb300.json")
    tune = open(tune_path).read() if os.path.exists(tune_path) else None
    plan = cc.Plan(S, len(c["x"]), tune)
    holder = {}

    def run():
        holder["c"], _ = plan.count_pairs_batched(t[0], t[1], t[2], t[3], r2=c["r2"])

    ms = _time(run, 20, torch)
    items = plan.last_items()
    n = np.diff(off)
    tests = int((n * (n - 1) // 2).sum())
    if not with_plain:
        plan.close()
        return {"workload": f"{S} pruned sets, {int(off[-1])} int32 points, r2={c['r2']}", "ms": ms,
                "sets_per_s": S / (ms * 1e-3), "gpairs_s": tests / (ms * 1e-3) / 1e9, "work_items": items}
    # plain per-set launches on the same GPU, every set: cc_count_pairs per set, which for
    # sets below 8192 objects is one launch of the small-set kernel (the same stage loop,
    # no preparation pass), and the tensor-core path for the one set of 8192
    outs = torch.empty(S, dtype=torch.int64, device=dev)
    xs = [(int(off[k]), int(off[k + 1])) for k in range(S)]
    views = [(t[0][a:b], t[1][a:b], t[2][a:b]) for (a, b) in xs]
    out_views = [outs[k:k + 1] for k in range(S)]
    r2 = c["r2"]

    def plain():
        for v, o in zip(views, out_views):
            cc.count_pairs(*v, r2=r2, out=o)

    plain()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    e0.record()
    plain()
    e1.record()
    torch.cuda.synchronize()
    wall_plain = time.perf_counter() - w0
    ms_plain = e0.elapsed_time(e1)
    ok = bool((outs == holder["c"]).all().item())
    # the same per-set launches recorded once into a CUDA graph and replayed: no host work
    # per launch, the most favourable form of plain launches
    cap = torch.cuda.Stream()
    cc.reserve(8192, stream=cap)
    outs.fill_(-1)
    with torch.cuda.stream(cap):
        for v, o in zip(views, out_views):
            cc.count_pairs(*v, r2=r2, out=o, stream=cap)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        for v, o in zip(views, out_views):
            cc.count_pairs(*v, r2=r2, out=o, stream=cap)
    outs.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    ok_graph = bool((outs == holder["c"]).all().item())
    ms_graph = _time(graph.replay, 3, torch)
    del graph
    plan.close()
    return {"workload": f"{S} pruned sets, {int(off[-1])} int32 points, r2={c['r2']}",
            "tile_table": "autotuned (paper_1901_11204_gb300/tune_gb300.json)" if tune else "built-in defaults",
            "ms": ms, "sets_per_s": S / (ms * 1e-3), "gpairs_s": tests / (ms * 1e-3) / 1e9,
            "work_items": items, "pair_tests": tests,
            "plain_ms": ms_plain, "plain_wall_s": wall_plain, "plain_us_per_set": ms_plain / S * 1e3,
            "plain_graph_ms": ms_graph, "plain_graph_us_per_set": ms_graph / S * 1e3,
            "plain_launches_per_set": 1,
            "speedup_vs_plain": ms_plain / ms, "speedup_vs_plain_graph": ms_graph / ms,
            "plain_sets": S, "plain_matches_batched": ok and ok_graph,
            "plain_note": "one cc_count_pairs call per set over all sets (one small-set kernel launch each; the "
                          "tensor-core path for the set of 8192): plain_ms is the Python loop between events "
                          "(host enqueue rate included), plain_graph_ms the same launches replayed from one "
                          "captured CUDA graph"}


def bench_serving(cc, torch, dev, nq):
    pool = synth.cfg5_pool(2048)
    srv = cc.Server(8 << 30, 4096)
    ids = [srv.register_set(p["x"], p["y"], p["z"], r=p.get("r")) for p in pool]
    # serial plain launches (one request at a time, synchronised): baseline capacity
    dsets = [[torch.from_numpy(p[k]).to(dev) for k in (("x", "y", "z") if p["kind"] == "i32" else ("x", "y", "z", "r"))]
             for p in pool]
    qs = synth.cfg5_queries(nq, len(pool), 1.0)
    ops = qs["op"]
    sid = qs["set_id"]
    probe = min(nq, 2000)

    def serial(k):
        s = dsets[int(sid[k])]
        if len(s) == 3:
            cc.count_pairs(*s, r2=9)
        elif ops[k] == 2:
            cc.interaction_sum(s[0], s[1], s[2], r=s[3])
        else:
            cc.count_pairs(s[0], s[1], s[2], r=s[3])
        torch.cuda.synchronize()

    for k in range(50):
        serial(k)
    lat = []
    t0 = time.perf_counter()
    for k in range(probe):
        a = time.perf_counter()
        serial(k)
        lat.append(time.perf_counter() - a)
    serial_rate = probe / (time.perf_counter() - t0)

    def serial_stream(rate, count):
        """Serial plain launches under the same Poisson arrivals: each request waits for
        its arrival time and for the previous request, then runs synchronously; latency is
        completion minus arrival (the queueing a one-at-a-time service sees)."""
        q = synth.cfg5_queries(count, len(pool), rate)
        lat_s = []
        start = time.perf_counter()
        for k in range(count):
            target = start + q["t"][k]
            while time.perf_counter() < target:
                pass
            s = dsets[int(q["set_id"][k])]
            if len(s) == 3:
                cc.count_pairs(*s, r2=9)
            elif q["op"][k] == 2:
                cc.interaction_sum(s[0], s[1], s[2], r=s[3])
            else:
                cc.count_pairs(s[0], s[1], s[2], r=s[3])
            torch.cuda.synchronize()
            lat_s.append(time.perf_counter() - target)
        end = time.perf_counter()
        lat_s = np.array(lat_s)
        return {"offered_qps": rate, "queries": count, "achieved_qps": count / (end - start),
                "p50_ms": float(np.percentile(lat_s, 50) * 1e3), "p99_ms": float(np.percentile(lat_s, 99) * 1e3)}

    def run_stream(rate, count=None):
        count = nq if count is None else count
        q = synth.cfg5_queries(count, len(pool), rate)
        start = time.perf_counter()
        t = q["t"]
        for k in range(count):
            target = start + t[k]
            while True:
                d = target - time.perf_counter()
                if d <= 0:
                    break
                if d > 2e-4:
                    time.sleep(d - 1e-4)
            op = cc.CC_OP_SUM if q["op"][k] == 2 else cc.CC_OP_COUNT
            srv.submit(ids[int(q["set_id"][k])], op, 9, k)
        srv.drain(300)
        end = time.perf_counter()
        res = []
        while True:
            g = srv.poll(65536)
            if not g:
                break
            res += g
        lat = np.array([r["t_done"] - r["t_arrive"] for r in res])
        return {"offered_qps": rate, "queries": len(res), "achieved_qps": len(res) / (end - start),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "errors": int(sum(1 for r in res if r["status"] != 0))}

    # saturation throughput: all queries offered at once
    sat = run_stream(1e9)
    runs = [sat]
    for frac in (0.5, 0.8):
        runs.append(run_stream(frac * sat["achieved_qps"]))
    # served against serial plain launches at equal offered rates: half the serial
    # capacity (both keep up), the serial capacity, and a tenth of the served saturation
    low = min(nq, 10000)
    equal_rate = []
    for label, rate in (("0.5x serial capacity", 0.5 * serial_rate), ("serial capacity", serial_rate),
                        ("0.1x served saturation", 0.1 * sat["achieved_qps"])):
        served = run_stream(rate, low)
        plain = serial_stream(rate, min(low, 4000))
        equal_rate.append({"label": label, "offered_qps": rate, "served": served, "serial_plain": plain})
    st = srv.stats()
    resident = st["peak_bytes"]
    srv.close()
    # a tight budget (resident bytes + 2 MiB of per-request scratch): admission binds, the
    # stream still completes with the same results
    tight = int(resident) + (2 << 20)
    srv2 = cc.Server(tight, 4096)
    ids2 = [srv2.register_set(p["x"], p["y"], p["z"], r=p.get("r")) for p in pool]
    q2 = synth.cfg5_queries(min(nq, 5000), len(pool), 0.8 * sat["achieved_qps"])
    t0 = time.perf_counter()
    for k in range(len(q2["t"])):
        target = t0 + q2["t"][k]
        while time.perf_counter() < target:
            pass
        srv2.submit(ids2[int(q2["set_id"][k])], cc.CC_OP_SUM if q2["op"][k] == 2 else cc.CC_OP_COUNT, 9, k)
    srv2.drain(300)
    res2 = []
    while True:
        g = srv2.poll(65536)
        if not g:
            break
        res2 += g
    lat2 = np.array([r["t_done"] - r["t_arrive"] for r in res2])
    st2 = srv2.stats()
    srv2.close()
    tight_run = {"budget_bytes": tight, "queries": len(res2), "p50_ms": float(np.percentile(lat2, 50) * 1e3),
                 "p99_ms": float(np.percentile(lat2, 99) * 1e3), "peak_inflight": st2["peak_inflight"],
                 "batches": st2["batches"], "errors": int(sum(1 for r in res2 if r["status"] != 0))}
    return {"workload": f"{nq} Poisson queries over {len(pool)} resident sets (lognormal n in [16,65536])",
            "budget_note": "the 8 GiB budget never binds for this pool (peak bytes in server_stats); "
                           "tight_budget repeats 0.8 load with resident + 2 MiB",
            "tight_budget": tight_run,
            "serial_plain_qps": serial_rate,
            "serial_plain_p50_ms": float(np.percentile(lat, 50) * 1e3),
            "serial_plain_p99_ms": float(np.percentile(lat, 99) * 1e3),
            "runs": runs, "equal_rate": equal_rate, "server_stats": st,
            "speedup_vs_serial": sat["achieved_qps"] / serial_rate}


def cpu_baseline(sets):
    import oracle
    oracle.build()
    oracle.set_threads(0)
    cores = oracle.get_threads()
    t0 = time.perf_counter()
    for x, y, z, r2 in sets:
        oracle.count_i32(x, y, z, r2)
    dt = time.perf_counter() - t0
    tests = sum(pairs(len(s[0])) for s in sets)
    # the literal loop on one core, on a bounded sample (the first 32768 points of the
    # first set: 5.4e8 pair tests)
    x, y, z, r2 = sets[0]
    m = min(len(x), 32768)
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.count_i32(x[:m], y[:m], z[:m], r2)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(0)
    return {"value": tests / dt / 1e9, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": "the full step (all three sets) once", "seconds": dt,
            "one_core": {"value": pairs(m) / dt1 / 1e9, "unit": METRIC, "cores": 1,
                         "sample": f"first {m} points of the first set, r2 = {r2}", "seconds": dt1}}


if __name__ == "__main__":
    sys.exit(main())
