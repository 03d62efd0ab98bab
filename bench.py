#!/usr/bin/env python
"""Throughput benchmark of the Squares generator (arXiv:2004.06278) on GB300.

One step = one pass of the hot path over the single-stream throughput
workload: squares64 into uint64[2^30] (8 GiB) and squares32 into
uint32[2^32] (16 GiB), one key (first key of seed 2), counter base drawn
uniformly from [0, 2^64) (seed 3). With N ranks each rank generates the same
amount from its own disjoint counter range (weak scaling; no collective on
the data path -- the only collectives are the timing barrier and the max of
the elapsed times).

Printed: one JSON line with value = whole-job Gsamples/s (device-resident
outputs), the roofline of the dominant kernel (squares32), the oracle timed
on the host cores, the end-to-end rate with outputs copied into pinned host
memory, the SM clocks sampled during the timed region, and a breakdown of
the other kernels (ragged batch vs plain, transforms, fused statistics,
cuRAND Philox4x32-10 as context), each measured outside the timed region.

--impl reference times the oracle (plain C on the host cores) on a bounded
sample of the same workload and prints the same metric with
"impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gsamples/s squares32/64, batched vs plain, % of IMAD/HBM-store roofline"
N64 = 1 << 30
N32 = 1 << 32
WORKLOAD = ("squares64 -> uint64[2^30] + squares32 -> uint32[2^32], one key (sq_make_keys seed 2), "
            "counter base uniform in [0,2^64) (seed 3)")
# Integer work per sample on the FMA-heavy pipe (the one that executes the
# 32-bit multiply-adds), in cycles per warp of 32 samples: each round after
# the first is one wide multiply-add (4 cycles) and one multiply-add (2);
# round 1 is carried by additions (second-order Weyl recurrence). squares32
# has 3 such rounds, squares64 4. Four sub-partitions per SM, 32 lanes each.
HEAVY_CYCLES_SQ32 = 18
HEAVY_CYCLES_SQ64 = 24
LANES_PER_SM = 128


def parse_args():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-extras", action="store_true", help="skip the breakdown section")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="use the default launch table")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--tune-file", help="load the launch table from this file if it exists "
                                       "(no tuning); otherwise tune and save it there")
    p.add_argument("--profile", choices=["u32", "u64", "batch", "uniform_f32", "uniform_bf16",
                                         "normal_f32", "uniform2_f32", "uniform_f64", "fused",
                                         "u32_stride3", "u64_stride3", "keys_u32", "keys_u64",
                                         "batch_short", "batch_tiny", "batch_mid"],
                   help="run one kernel on a small case (for ncu) instead of the benchmark")
    p.add_argument("--profile-n", type=int, default=1 << 28)
    p.add_argument("--profile-variant", help="batch variant name for the batch_* profile cases "
                                             "(default: the one named in the case)")
    p.add_argument("--profile-block", type=int, default=0,
                   help="block size for the batch_* profile cases (default: the tuner's pick)")
    p.add_argument("--reference-budget-s", type=float, default=60.0,
                   help="wall time the reference arm aims to spend on its K steps")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def shard_base(base: int, n_per_rank: int, rank: int) -> int:
    """First counter of rank's shard: the ranks split one contiguous counter
    range [base, base + world * n_per_rank) mod 2^64 into equal parts, as
    the paper divides the 2^64 counter space among cores (Section 3)."""
    return (base + rank * n_per_rank) % (1 << 64)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over all ranks (the job's elapsed time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="sq_clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


# --------------------------------------------------------------------------
# reference arm: the oracle on the host cores

def oracle_sample_rate(n64: int, n32: int, chunk: int = 1 << 26, threads: int | None = None):
    """Time the oracle (as it stands) on n64 squares64 and n32 squares32
    samples, in chunks, on `threads` threads (default: all host cores);
    returns (samples/s, seconds, threads)."""
    import oracle

    key = int(oracle.make_keys(2, 1)[0])
    from paper_2004_06278_gb300 import workloads

    base = workloads.throughput_base(3)
    threads = threads or oracle.default_threads()
    oracle.fill32(key, base, 1 << 16)  # load the library outside the timing
    t0 = time.perf_counter()
    for a in range(0, n64, chunk):
        oracle.fill64(key, (base + a) % (1 << 64), min(chunk, n64 - a), threads=threads)
    for a in range(0, n32, chunk):
        oracle.fill32(key, (base + a) % (1 << 64), min(chunk, n32 - a), threads=threads)
    dt = time.perf_counter() - t0
    return (n64 + n32) / dt, dt, threads


CPU_SAMPLE = (1 << 28, 1 << 30)  # squares64, squares32 samples: 1/4 of a step


def cpu_model() -> str:
    """Host CPU model name (lscpu), for the record beside the oracle timing."""
    import platform
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def cpu_baseline_block():
    rate, dt, threads = oracle_sample_rate(*CPU_SAMPLE)
    rate1, dt1, _ = oracle_sample_rate(CPU_SAMPLE[0] >> 4, CPU_SAMPLE[1] >> 4, threads=1)
    return {"value": rate / 1e9, "unit": "Gsamples/s", "cores": threads, "kind": "oracle",
            "sample": f"2^28 squares64 + 2^30 squares32 samples of the step's workload "
                      f"(1/4 of a step), oracle in 2^26-sample calls on {threads} threads, "
                      f"{dt:.2f} s wall",
            "cpu_model": cpu_model(),
            "single_thread": {"value": rate1 / 1e9, "unit": "Gsamples/s",
                              "sample": f"2^24 squares64 + 2^26 squares32 samples, {dt1:.2f} s wall"}}


def reference_arm(args, rank, world):
    """The oracle timed as it stands on the host cores. Each step is a
    bounded sample of the workload (same 1:4 mix of squares64 and squares32
    samples), sized from a calibration run so that all K steps take about a
    minute."""
    if rank != 0:
        return 0
    rate, _, threads = oracle_sample_rate(1 << 20, 1 << 22)  # calibration / warm-up
    budget_s = args.reference_budget_s
    per_step = rate * budget_s / max(1, args.steps)
    unit = 5 << 20  # 2^20 squares64 + 2^22 squares32
    units = int(max(1, min((N64 + N32) // unit, per_step // unit)))
    n64, n32 = units << 20, units << 22
    for _ in range(args.warmup):  # untimed, same size as a timed step
        oracle_sample_rate(n64, n32)
    times = []
    for _ in range(args.steps):
        _, dt, threads = oracle_sample_rate(n64, n32)
        times.append(dt)
    total = sum(times)
    value = args.steps * (n64 + n32) / total / 1e9
    sample = f"{n64} squares64 + {n32} squares32 samples per step of the GPU step's workload"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gsamples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": sample,
                   "parallelism": f"{threads} host threads"},
        "cpu_baseline": {"value": value, "unit": "Gsamples/s", "cores": threads, "kind": "oracle",
                         "sample": sample + "; plain-C oracle in 2^26-sample calls"},
        "e2e": {"value": value, "unit": "Gsamples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm

def source_hash(*rel):
    """Hash of the kernel sources' code (comments and whitespace removed)."""
    from paper_2004_06278_gb300 import build as libbuild

    return libbuild.code_hash([os.path.join(ROOT, r) for r in rel])


KERNEL_SOURCES = ("paper_2004_06278_gb300/csrc/kernels_plain.cu",
                  "paper_2004_06278_gb300/csrc/stores.cuh", "include/squares_device.cuh")


def profiled_traffic(name: str):
    """DRAM bytes per launch recorded by ncu for `name`, if the profile was
    taken on the current kernel source (same hash), else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    cur = source_hash(*KERNEL_SOURCES)
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and parts[0] == name and parts[2] == cur:
                return int(parts[1])
    return None


class Timer:
    def __init__(self, torch, stream):
        self.torch = torch
        self.stream = stream
        self.pairs = []

    def span(self):
        a = self.torch.cuda.Event(enable_timing=True)
        b = self.torch.cuda.Event(enable_timing=True)
        self.pairs.append((a, b))
        return a, b

    def mean_ms(self):
        return sum(a.elapsed_time(b) for a, b in self.pairs) / max(1, len(self.pairs))


def run_ours(args, rank, world, local):
    import torch

    import paper_2004_06278_gb300 as sq
    from paper_2004_06278_gb300 import _lib as C
    from paper_2004_06278_gb300 import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sq.load()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)
    key = int(sq.make_keys(2, 1)[0])
    base0 = workloads.throughput_base(3)
    base64 = shard_base(base0, N64, rank)
    base32 = shard_base(base0, N32, rank)
    out64 = torch.empty(N64, dtype=torch.int64, device=dev)
    out32 = torch.empty(N32, dtype=torch.int32, device=dev)
    tuned_from_file = bool(args.tune_file and os.path.exists(args.tune_file))
    if tuned_from_file:
        try:
            C.sq_autotune_load(args.tune_file)
        except C.SquaresError as e:  # tuned on other kernel code: tune again
            print(f"bench: {e}; tuning again", file=sys.stderr)
            tuned_from_file = False
    if not tuned_from_file and not args.no_tune:
        C.sq_autotune(C.SQ_KERNEL_U64, N64)
        C.sq_autotune(C.SQ_KERNEL_U32, N32)
    cfg32 = C.sq_get_config(C.SQ_KERNEL_U32, N32)
    cfg64 = C.sq_get_config(C.SQ_KERNEL_U64, N64)

    t64 = Timer(torch, stream)
    t32 = Timer(torch, stream)

    def step(timed: bool):
        if timed:
            a, b = t64.span()
            a.record(stream)
        C.sq_u64(key, base64, N64, out64.data_ptr(), sh)
        if timed:
            b.record(stream)
            a, b = t32.span()
            a.record(stream)
        C.sq_u32(key, base32, N32, out32.data_ptr(), sh)
        if timed:
            b.record(stream)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
        time.sleep(0.3)  # let nvidia-smi start sampling
    barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        step(True)
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clock_info = clocks.stop() if rank == 0 else None
    elapsed = max_over_ranks(start.elapsed_time(end) / 1000.0, world, dev)
    samples = world * args.steps * (N64 + N32)
    value = samples / elapsed / 1e9
    ms32 = t32.mean_ms()
    ms64 = t64.mean_ms()

    result = None
    if rank == 0:
        peaks, peak_src = measured_peaks()
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count
        sm_max = float(clock_info.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
        lane_cycles = sms * LANES_PER_SM * sm_max * 1e6  # sample-lanes x cycles per second
        r32 = N32 / (ms32 / 1e3)
        r64 = N64 / (ms64 / 1e3)
        hbm = float(peaks["hbm_gbs"])
        r_hbm32 = hbm * 1e9 / 4
        r_int32 = lane_cycles / HEAVY_CYCLES_SQ32
        r_int64 = lane_cycles / HEAVY_CYCLES_SQ64
        store = store_ceiling(torch, C, out32, N32, stream)
        # The ceiling of DRAM writes: the best of the write-only sweep and of
        # what the squares64 launches of the timed region themselves wrote.
        store_gbs = max(store["GBps"], r64 * 8 / 1e9)
        store_src = ("sq_fill_u32 sweep" if store["GBps"] >= r64 * 8 / 1e9
                     else "squares64 launches of the timed region (above the sq_fill_u32 sweep)")
        # Bound from the counters: the squares32 kernel runs as fast without
        # its stores as with them and its FMA-heavy pipe is the busiest unit
        # (profiles/sq_u32_plain_2p28.md), so it is bound by integer issue,
        # not by HBM; the peak is the integer model of the algorithm (three
        # multiplying rounds, 18 FMA-heavy cycles per warp of samples).
        roof = {"bound": "alu", "achieved": r32 / 1e9, "peak": r_int32 / 1e9,
                "unit": "Gsamples/s", "frac": r32 / r_int32}
        roof.update({
            "kernel": "sq_u32 (plain squares32, 2^32 outputs per launch)",
            "traffic": profiled_traffic("sq_u32_plain"),
            "traffic_unit": "bytes per launch (dram read + write)",
            "algorithmic_bytes": 4 * N32,
            "avg_launch_ms": ms32,
            "peak_source": f"integer model: {sms} SMs x {LANES_PER_SM} lanes x {sm_max} MHz / "
                           f"{HEAVY_CYCLES_SQ32} FMA-heavy cycles per warp-sample = "
                           f"{r_int32 / 1e9:.0f} Gsamples/s; hbm copy {hbm} GB/s ("
                           + ("measured, MEASURED_PEAKS.json" if peak_src == "measured"
                              else "fallback figure: MEASURED_PEAKS.json absent")
                           + f"); store-only ceiling: the best DRAM write rate measured here, "
                           f"of {store['configs']} sq_fill_u32 shapes and the squares64 launches",
            "limiter": "FMA-heavy pipe (ncu: busiest unit; the kernel without stores takes the "
                       "same time as with them)",
            "achieved_GBps": r32 * 4 / 1e9,
            "frac_hbm": (r32 * 4 / 1e9) / hbm,
            "peak_store_only": store_gbs,
            "frac_store_only": (r32 * 4 / 1e9) / store_gbs,
            "store_only_source": store_src,
            "store_only_sweep": {"GBps": store["GBps"], "best": store["best"],
                                 "configs": store["configs"]},
            "frac_int": r32 / r_int32,
            "squares64": {"avg_launch_ms": ms64, "Gsamples_per_s": r64 / 1e9,
                          "GBps": r64 * 8 / 1e9, "bound": "hbm" if store_gbs * 1e9 / 8 < r_int64 else "alu",
                          "frac_hbm": (r64 * 8 / 1e9) / hbm, "frac_store_only": (r64 * 8 / 1e9) / store_gbs,
                          "frac_int": r64 / r_int64},
        })
        result = {
            "metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed * 1000 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "samples_per_step_per_gpu": N64 + N32,
                       "bytes_written_per_step_per_gpu": 8 * N64 + 4 * N32,
                       "l2": "outputs (24 GiB per step) exceed the 129 MB L2; no flush",
                       "parallelism": f"{world} rank(s), disjoint counter ranges, no collective",
                       "launch": {"sq_u32": [C.sq_variant_name(0, cfg32.variant), cfg32.block,
                                             cfg32.ctas_per_sm],
                                  "sq_u64": [C.sq_variant_name(1, cfg64.variant), cfg64.block,
                                             cfg64.ctas_per_sm],
                                  "tuned": "file" if tuned_from_file else not args.no_tune}},
            "roofline": roof,
            "clocks": clock_info,
            "gpu_launches": 2 * args.steps,
        }
    del out64, out32
    torch.cuda.empty_cache()

    if rank == 0 and not args.no_e2e:
        result["e2e"] = e2e_block(torch, C, key, base64, base32, dev, args.e2e_steps)
    if rank == 0 and not args.no_extras:
        result["breakdown"] = breakdown(torch, sq, C, workloads, dev, ms32, tuned_from_file,
                                        with_oracle=world == 1 and not args.no_cpu_baseline)
    if rank == 0 and args.tune_file and not tuned_from_file:
        C.sq_autotune_save(args.tune_file)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_block()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    return 0


def store_ceiling(torch, C, buf, n, stream, reps=3):
    """Write-only ceiling of HBM for the generators' store path: sq_fill_u32
    (their chunking, grid and store variants, no arithmetic) over n uint32
    elements of `buf`, in every store variant, block size and CTA count the
    plain kernels use, and paced (each thread pausing after each chunk) in
    the few-thread shapes where a flood of stores is slower than a paced
    stream; CUDA events on `stream`. Returns the best rate (GB/s written),
    its configuration and pause, and how many were timed."""
    sh = int(stream.cuda_stream)
    shapes = [((v, block, ctas), 0) for v in range(C.sq_num_variants(C.SQ_KERNEL_U32))
              for block in (128, 256, 512) for ctas in (1, 2, 4, 0)]
    shapes += [((v, block, ctas), pause) for v in (0, 1, 4, 5) for block in (128, 256)
               for ctas in (1, 2) for pause in (64, 128, 256, 512)]
    best, best_cfg = 0.0, None
    for cfg, pause in shapes:
        C.sq_fill_u32(0x5A5A5A5A, n, buf.data_ptr(), cfg, pause, sh)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            C.sq_fill_u32(0x5A5A5A5A, n, buf.data_ptr(), cfg, pause, sh)
        b.record(stream)
        torch.cuda.synchronize()
        gbs = n * 4 * reps / (a.elapsed_time(b) / 1e3) / 1e9
        if gbs > best:
            best = gbs
            best_cfg = [C.sq_variant_name(C.SQ_KERNEL_U32, cfg[0]), cfg[1], cfg[2], f"pause {pause} ns"]
    return {"GBps": best, "best": best_cfg, "configs": len(shapes)}


def e2e_block(torch, C, key, base64, base32, dev, steps):
    """The same step through the C ABI with the outputs landing in pinned
    host memory. Two paths are timed and the faster is reported:
      copy:   per 2 GiB chunk the kernel writes a device staging buffer and
              a cudaMemcpyAsync moves it to the host; two streams alternate
              so copies overlap generation;
      direct: the kernels store straight into the pinned host buffers (the
              buffers are mapped into the device's address space; on GB300
              the stores cross NVLink-C2C). For host-resident outputs the
              library uses the contiguous 32-byte-per-lane stores whatever
              variant is tuned for device memory.
    The step's inputs are two 64-bit scalars passed by value in the launch
    (no host-to-device copy). `copy_engine_GBps` is a plain device-to-host
    copy of one staging buffer: the ceiling of the copy path, and of the
    direct path while the copy engine runs at its usual rate."""
    chunk = 1 << 28  # elements
    host64 = torch.empty(N64, dtype=torch.int64, pin_memory=True)
    host32 = torch.empty(N32, dtype=torch.int32, pin_memory=True)
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    stage = [torch.empty(chunk * 8, dtype=torch.uint8, device=dev) for _ in streams]

    def run_copy():
        k = 0
        for fn, host, n, es, base in ((C.sq_u64, host64, N64, 8, base64),
                                      (C.sq_u32, host32, N32, 4, base32)):
            for a in range(0, n, chunk):
                m = min(chunk, n - a)
                s = streams[k % 2]
                buf = stage[k % 2]
                with torch.cuda.stream(s):
                    fn(key, (base + a) % (1 << 64), m, buf.data_ptr(), int(s.cuda_stream))
                    dst = host.view(torch.uint8)[a * es:(a + m) * es]
                    dst.copy_(buf[:m * es], non_blocking=True)
                k += 1
        for s in streams:
            s.synchronize()

    def run_direct():
        s = streams[0]
        C.sq_u64(key, base64, N64, host64.data_ptr(), int(s.cuda_stream))
        C.sq_u32(key, base32, N32, host32.data_ptr(), int(s.cuda_stream))
        s.synchronize()

    def timed(fn):
        fn()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        return (time.perf_counter() - t0) / steps

    def run_link():
        with torch.cuda.stream(streams[0]):
            host64.view(torch.uint8)[:chunk * 8].copy_(stage[0], non_blocking=True)
        streams[0].synchronize()

    # Host-link probes into the same pinned memory: several copies at once
    # (one per stream, separate staging buffers and host ranges), and the SMs
    # storing straight across the link (sq_fill_u32, no arithmetic).
    link_streams = [torch.cuda.Stream(dev) for _ in range(4)]
    link_stage = stage + [torch.empty(chunk * 8, dtype=torch.uint8, device=dev) for _ in range(2)]
    host_bytes = host32.view(torch.uint8)

    def run_copies(k):
        def run():
            for i in range(k):
                with torch.cuda.stream(link_streams[i]):
                    host_bytes[i * chunk * 8:(i + 1) * chunk * 8].copy_(link_stage[i], non_blocking=True)
            for st in link_streams[:k]:
                st.synchronize()
        return run

    def run_fill():
        C.sq_fill_u32(0x5A5A5A5A, N32, host32.data_ptr(), None, 0, int(streams[0].cuda_stream))
        streams[0].synchronize()

    dt_copy = timed(run_copy)
    dt_direct = timed(run_direct)
    dt_link = timed(run_link)
    probes = {"copy_x1_GBps": chunk * 8 / dt_link / 1e9}
    for k in (2, 4):
        probes[f"copies_x{k}_GBps"] = k * chunk * 8 / timed(run_copies(k)) / 1e9
    probes["sm_stores_GBps"] = 4 * N32 / timed(run_fill) / 1e9
    link = max(probes.values())
    d2h = 8 * N64 + 4 * N32
    best = min(dt_copy, dt_direct)
    res = {"value": (N64 + N32) / best / 1e9, "unit": "Gsamples/s", "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": d2h, "ms_per_step": best * 1000, "steps": steps,
           "d2h_GBps": d2h / best / 1e9, "copy_engine_GBps": probes["copy_x1_GBps"],
           "frac_of_copy_engine": (d2h / best / 1e9) / probes["copy_x1_GBps"],
           "link_ceiling_GBps": link, "frac_of_link": (d2h / best / 1e9) / link,
           "link_probes": probes,
           "note": "link_ceiling_GBps: the best of one 2 GiB cudaMemcpyAsync, 2 and 4 such copies "
                   "at once on separate streams, and the SMs storing constants straight into the "
                   "pinned buffer (sq_fill_u32), all into the same pinned memory",
           "path": "direct: kernels store into pinned host memory" if dt_direct <= dt_copy else
                   "copy: 2 GiB device chunks, cudaMemcpyAsync to pinned host, 2 streams",
           "copy_ms_per_step": dt_copy * 1000, "direct_ms_per_step": dt_direct * 1000}
    del link_stage
    del host64, host32, stage
    return res


def _time_graph(torch, fn, reps, stream):
    """Capture fn() into a CUDA graph on `stream`; mean ms per replay."""
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        fn()
        stream.synchronize()
        with torch.cuda.graph(g, stream=stream):
            fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):  # replays go to the stream the events are on
        g.replay()
        a.record(stream)
        for _ in range(reps):
            g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _time_launches(torch, fn, reps, stream):
    with torch.cuda.stream(stream):
        fn()
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def breakdown(torch, sq, C, workloads, dev, ms32_plain, tuned_from_file=False, with_oracle=True):
    """Every other configuration of the benchmark suite, measured outside the
    timed region; with_oracle adds the oracle's rate on the host cores to each
    configuration's row and the transforms' error against FP64."""
    import numpy as np

    out = {}
    stream = torch.cuda.Stream(dev)
    sh = lambda: int(stream.cuda_stream)  # noqa: E731
    plain_rate = N32 / (ms32_plain / 1e3)
    out["squares32_plain"] = {"Gsamples_per_s": plain_rate / 1e9, "GBps": plain_rate * 4 / 1e9}

    # squares32 from counter 0, first key of seed 1, 2^24 outputs (the parity
    # configuration; its 64 MiB of output fits in L2)
    key1 = int(sq.make_keys(1, 1)[0])
    n1 = 1 << 24
    buf1 = torch.empty(n1, dtype=torch.int32, device=dev)
    ms = _time_launches(torch, lambda: C.sq_u32(key1, 0, n1, buf1.data_ptr(), sh()), 20, stream)
    out["single_2p24"] = {"Gsamples_per_s": n1 / (ms / 1e3) / 1e9, "ms": ms,
                          "note": "64 MiB of output: L2-resident writes"}
    if with_oracle:
        out["single_2p24"]["cpu_baseline"] = oracle_rate_pair(
            lambda th: __import__("oracle").fill32(key1, 0, n1, threads=th), n1,
            lambda th: __import__("oracle").fill32(key1, 0, n1 >> 2, threads=th), n1 >> 2,
            "all 2^24 outputs of the configuration", "the first 2^22 outputs")
    del buf1

    # ragged batch, 4096 streams, one persistent launch replayed from a CUDA graph
    b = workloads.ragged_batch(4096, seed=7)
    keys = torch.from_numpy(sq.make_keys(b.key_seed, b.nstreams).view(np.int64)).to(dev)
    bases = torch.from_numpy(b.bases.view(np.int64)).to(dev)
    lengths = torch.from_numpy(b.lengths).to(dev)
    offsets = torch.from_numpy(b.offsets).to(dev)
    outb = torch.empty(b.total, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()  # inputs were copied on the default stream
    if not tuned_from_file:
        C.sq_autotune_batch(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(),
                            offsets.data_ptr(), b.nstreams, outb.data_ptr())
    cfgb = C.sq_get_config(C.SQ_KERNEL_BATCH, b.nstreams)

    def run_batch():
        C.sq_batch(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(), offsets.data_ptr(),
                   b.nstreams, outb.data_ptr(), sh())

    ms_b = _time_graph(torch, run_batch, 10, stream)
    rate_b = b.total / (ms_b / 1e3)
    out["batched_ragged"] = {
        "streams": b.nstreams, "samples": b.total, "ms": ms_b, "Gsamples_per_s": rate_b / 1e9,
        "GBps": rate_b * 4 / 1e9, "per_sample_vs_plain": rate_b / plain_rate,
        "launch": [C.sq_variant_name(2, cfgb.variant), cfgb.block, cfgb.ctas_per_sm],
        "timing": "CUDA graph of one persistent launch, 10 replays"}
    if with_oracle:
        out["batched_ragged"]["cpu_baseline"] = oracle_batch_rate(np, b)
    del outb, keys, bases, lengths, offsets
    torch.cuda.empty_cache()

    # mid-length and many short streams, each with the configuration the
    # batch tuner picks for it (then the long-stream choice is restored)
    for name, S_, lo_, hi_ in (("batched_mid_streams", 1 << 14, 3e3, 3e4),
                               ("batched_short_streams", 1 << 20, 30, 300),
                               ("batched_tiny_streams", 1 << 22, 3, 30)):
        out[name] = _batch_regime(torch, sq, C, workloads, np, dev, stream, sh, S_, lo_, hi_,
                                  plain_rate)
    torch.cuda.empty_cache()

    # transforms, 2^30 outputs each (two floats or one normal pair per
    # squares64 output for uniform2_f32 / normal_f32)
    key = int(sq.make_keys(11, 1)[0])
    n = 1 << 30
    buf = torch.empty(n * 8, dtype=torch.uint8, device=dev)
    for name, kid, fn, es in (("uniform_f32", C.SQ_KERNEL_UNIFORM_F32, C.sq_uniform_f32, 4),
                              ("uniform_bf16", C.SQ_KERNEL_UNIFORM_BF16, C.sq_uniform_bf16, 2),
                              ("normal_f32", C.SQ_KERNEL_NORMAL_F32, C.sq_normal_f32, 4),
                              ("uniform2_f32", C.SQ_KERNEL_UNIFORM2_F32, C.sq_uniform2_f32, 4),
                              ("uniform_f64", C.SQ_KERNEL_UNIFORM_F64, C.sq_uniform_f64, 8)):
        if not tuned_from_file:
            C.sq_autotune(kid, n)
        ms = _time_launches(torch, lambda: fn(key, 0, n, buf.data_ptr(), sh()), 10, stream)
        out[name] = {"Gsamples_per_s": n / (ms / 1e3) / 1e9, "GBps": n * es / (ms / 1e3) / 1e9,
                     "ms": ms}
        if with_oracle and name in ("uniform_f32", "uniform_bf16", "normal_f32"):
            torch.cuda.synchronize()
            out[name]["precision"] = transform_precision(torch, np, name, buf, key, n)
            out[name]["cpu_baseline"] = oracle_transform_rate(name, key)

    # strided counters (Section 4's increments other than one), 2^30 outputs
    for name, fn, es in (("u32_stride3", C.sq_u32_strided, 4), ("u64_stride3", C.sq_u64_strided, 8)):
        ms = _time_launches(torch, lambda: fn(key, 5, 3, n, buf.data_ptr(), sh()), 10, stream)
        out[name] = {"Gsamples_per_s": n / (ms / 1e3) / 1e9, "GBps": n * es / (ms / 1e3) / 1e9,
                     "ms": ms}
    del buf
    torch.cuda.empty_cache()

    # key-counter mode (Section 4): one output per key at a fixed counter,
    # 2^27 keys (2^22 distinct keys tiled 32 times: the host key utility
    # takes ~0.4 us per key); bytes = 8 read + 4 or 8 written per key
    nk = 1 << 27
    kk = torch.from_numpy(sq.make_keys(17, 1 << 22).view(np.int64)).to(dev).repeat(nk >> 22)
    kbuf = torch.empty(nk * 8, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    for name, fn, es in (("keys_u32", C.sq_keys_u32, 4), ("keys_u64", C.sq_keys_u64, 8)):
        ms = _time_launches(torch, lambda: fn(kk.data_ptr(), nk, 0, kbuf.data_ptr(), sh()), 10, stream)
        out[name] = {"Gsamples_per_s": nk / (ms / 1e3) / 1e9, "GBps": nk * (8 + es) / (ms / 1e3) / 1e9,
                     "ms": ms, "keys": nk, "distinct_keys": 1 << 22}
    del kk, kbuf
    torch.cuda.empty_cache()

    # generation-only statistics, 2^20 streams x 2^18 counters
    S, cps = 1 << 20, 1 << 18
    fk = torch.from_numpy(sq.make_keys(13, S).view(np.int64)).to(dev)
    fb = torch.zeros(S, dtype=torch.int64, device=dev)
    fx = torch.empty(S, dtype=torch.int32, device=dev)
    fs = torch.empty(S, dtype=torch.int64, device=dev)
    fh = torch.empty(256, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    # default launch configuration (block 256, as many CTAs as fit): tuning on a
    # 2^32-counter subset picked 128-thread blocks, 1 % slower at full size
    cfgf = C.sq_get_config(C.SQ_KERNEL_FUSED, S * cps)
    ms = _time_launches(torch, lambda: C.sq_fused_stats(fk.data_ptr(), fb.data_ptr(), S, cps,
                                                        fx.data_ptr(), fs.data_ptr(),
                                                        fh.data_ptr(), sh()), 3, stream)
    props = torch.cuda.get_device_properties(dev)
    peaks, _ = measured_peaks()
    lane_cycles = props.multi_processor_count * LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6
    rate = S * cps / (ms / 1e3)
    out["fused_stats"] = {"Gsamples_per_s": rate / 1e9, "ms": ms,
                          "frac_int": rate / (lane_cycles / HEAVY_CYCLES_SQ32),
                          "launch": [C.sq_variant_name(C.SQ_KERNEL_FUSED, cfgf.variant), cfgf.block,
                                     cfgf.ctas_per_sm]}
    if with_oracle:
        fkeys = sq.make_keys(13, 1 << 14)
        fbases = np.zeros(1 << 14, dtype=np.uint64)
        out["fused_stats"]["cpu_baseline"] = oracle_rate_pair(
            lambda th: __import__("oracle").fused_stats(fkeys, fbases, cps, threads=th), (1 << 14) * cps,
            lambda th: __import__("oracle").fused_stats(fkeys[:1 << 8], fbases[:1 << 8], cps, threads=th),
            (1 << 8) * cps, "the first 2^14 of the 2^20 streams, all 2^18 counters each",
            "the first 2^8 streams")

    # context: cuRAND Philox4x32-10 (library call) on the same GPU
    out["curand_philox4x32_10"] = curand_context(torch, dev, stream)
    return out


def _repeat_timed(fn, threads, min_s=0.3, max_reps=64):
    """Seconds per call of fn(threads), repeating short calls until at least
    min_s have passed; returns (seconds per call, calls)."""
    reps, total = 0, 0.0
    while reps < max_reps and (reps == 0 or total < min_s):
        t0 = time.perf_counter()
        fn(threads)
        total += time.perf_counter() - t0
        reps += 1
    return total / reps, reps


def oracle_rate_pair(run_all, n_all, run_one, n_one, sample_all, sample_one):
    """The oracle as it stands, timed on all host cores and on one: run_all /
    run_one take a thread count and compute n_all / n_one samples."""
    import oracle

    threads = oracle.default_threads()
    run_one(1)  # load the library outside the timing
    dt, r = _repeat_timed(run_all, threads)
    dt1, r1 = _repeat_timed(run_one, 1)
    return {"value": n_all / dt / 1e9, "unit": "Gsamples/s", "cores": threads, "kind": "oracle",
            "sample": f"{sample_all}; {dt:.3f} s per call, {r} calls",
            "single_thread": {"value": n_one / dt1 / 1e9, "unit": "Gsamples/s",
                              "sample": f"{sample_one}; {dt1:.3f} s per call, {r1} calls"}}


def oracle_batch_rate(np, b, prefix=1 << 29):
    """oracle.batch32 on the first streams of the batch holding at most
    `prefix` samples, the streams split over the host cores (each thread
    writes its streams' disjoint ranges of one array)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    keys = oracle.make_keys(b.key_seed, b.nstreams)
    ends = b.offsets + b.lengths
    k = max(1, int(np.searchsorted(ends, prefix, side="right")))
    total = int(ends[k - 1])
    res = np.empty(total, dtype=np.uint32)

    def run(threads, kk):
        parts = np.array_split(np.arange(kk), threads)
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda idx: oracle.batch32(keys[idx], b.bases[idx], b.lengths[idx],
                                                   b.offsets[idx], res) if idx.size else None,
                        parts))

    k1 = max(1, int(np.searchsorted(ends, prefix >> 4, side="right")))
    return oracle_rate_pair(lambda th: run(th, k), total, lambda th: run(1, k1), int(ends[k1 - 1]),
                            f"the first {k} of {b.nstreams} streams ({total} samples)",
                            f"the first {k1} streams ({int(ends[k1 - 1])} samples)")


def oracle_transform_rate(name, key):
    """The oracle's transform (FP32/BF16 uniforms, FP64 normals) on 2^27
    outputs on all host cores and 2^23 on one."""
    import oracle

    fn = {"uniform_f32": oracle.uniform_f32, "uniform_bf16": oracle.uniform_bf16,
          "normal_f32": oracle.normal_f64}[name]
    return oracle_rate_pair(lambda th: fn(key, 0, 1 << 27, threads=th), 1 << 27,
                            lambda th: fn(key, 0, 1 << 23, threads=th), 1 << 23,
                            "the first 2^27 outputs of the configuration", "the first 2^23 outputs")


def transform_precision(torch, np, name, buf, key, n, chunk=1 << 26):
    """Error of the GPU transform over all n outputs in `buf` (counter base
    0) against the oracle, chunk by chunk: uniforms as mismatching bit
    patterns (0 is exact), normals as max absolute error where |z| < 5, max
    relative error where |z| >= 5, the number of such tail values and the
    largest |z|."""
    import oracle

    if name == "normal_f32":
        max_abs = max_rel = max_z = 0.0
        tail = 0
        for a in range(0, n, chunk):
            m = min(chunk, n - a)
            z = buf[4 * a:4 * (a + m)].view(torch.float32).cpu().numpy().astype(np.float64)
            ref = oracle.normal_f64(key, a // 2, m)
            err = np.abs(z - ref)
            core = np.abs(ref) < 5
            if core.any():
                max_abs = max(max_abs, float(err[core].max()))
            if (~core).any():
                max_rel = max(max_rel, float((err[~core] / np.abs(ref[~core])).max()))
                tail += int((~core).sum())
            max_z = max(max_z, float(np.abs(ref).max()))
        return {"outputs": n, "reference": "oracle Box-Muller in FP64 on the same integers",
                "max_abs_core": max_abs, "max_rel_tail": max_rel, "tail_count": tail,
                "max_abs_z": max_z, "bound_abs_core": 2e-6, "bound_rel_tail": 1e-5}
    es, ref_fn, dt = ((4, oracle.uniform_f32, np.uint32) if name == "uniform_f32"
                      else (2, oracle.uniform_bf16, np.uint16))
    bad = 0
    for a in range(0, n, chunk):
        m = min(chunk, n - a)
        got = buf[es * a:es * (a + m)].cpu().numpy().view(dt)
        bad += int(np.count_nonzero(got != ref_fn(key, a, m).view(dt)))
    return {"outputs": n, "mismatching_bit_patterns": bad,
            "reference": "oracle: floor(squares32 / 2^8) 2^-24" +
                         (", rounded toward zero to bfloat16" if name == "uniform_bf16" else "")}


def _batch_regime(torch, sq, C, workloads, np, dev, stream, sh, S, lo, hi, plain_rate):
    """One ragged batch of S streams of log-uniform length in [lo, hi), timed
    in the configuration sq_autotune_batch picks for it (kept in the batch
    table's entry for S streams)."""
    bs = workloads.ragged_batch(S, seed=7, lo=lo, hi=hi)
    keys = torch.from_numpy(sq.make_keys(bs.key_seed, bs.nstreams).view(np.int64)).to(dev)
    bases = torch.from_numpy(bs.bases.view(np.int64)).to(dev)
    lengths = torch.from_numpy(bs.lengths).to(dev)
    offsets = torch.from_numpy(bs.offsets).to(dev)
    outb = torch.empty(bs.total, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    C.sq_autotune_batch(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(),
                        offsets.data_ptr(), bs.nstreams, outb.data_ptr())
    cfg = C.sq_get_config(C.SQ_KERNEL_BATCH, bs.nstreams)

    def run():
        C.sq_batch(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(), offsets.data_ptr(),
                   bs.nstreams, outb.data_ptr(), sh())

    ms = _time_graph(torch, run, 10, stream)
    rate = bs.total / (ms / 1e3)
    return {"streams": bs.nstreams, "mean_length": bs.total / bs.nstreams, "samples": bs.total,
            "ms": ms, "Gsamples_per_s": rate / 1e9, "per_sample_vs_plain": rate / plain_rate,
            "launch": [C.sq_variant_name(2, cfg.variant), cfg.block, cfg.ctas_per_sm],
            "timing": "CUDA graph of one launch, 10 replays; configuration tuned on this batch"}


def curand_context(torch, dev, stream):
    import ctypes

    n = 1 << 32
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            lib = ctypes.CDLL(name)
            break
        except OSError:
            lib = None
    if lib is None:
        return {"unavailable": "libcurand not found"}
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    if lib.curandCreateGenerator(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        return {"unavailable": "curandCreateGenerator failed"}
    try:
        lib.curandSetStream(gen, ctypes.c_void_p(int(stream.cuda_stream)))
        buf = torch.empty(n, dtype=torch.int32, device=dev)
        fn = lambda: lib.curandGenerate(gen, ctypes.c_void_p(buf.data_ptr()), ctypes.c_size_t(n))  # noqa: E731
        ms = _time_launches(torch, fn, 5, stream)
        del buf
        return {"Gsamples_per_s": n / (ms / 1e3) / 1e9, "ms": ms, "n": n,
                "call": "curandGenerate (uint32), CURAND_RNG_PSEUDO_PHILOX4_32_10, 2^32 outputs"}
    finally:
        lib.curandDestroyGenerator(gen)
        torch.cuda.empty_cache()


def profile_case(args):
    """A small case of one kernel for ncu: 2 warm-up launches and 3 measured
    ones on --profile-n outputs (default 2^28: 1 GiB of uint32, larger than
    L2), default launch table unless --no-tune is absent."""
    import numpy as np
    import torch

    import paper_2004_06278_gb300 as sq
    from paper_2004_06278_gb300 import _lib as C
    from paper_2004_06278_gb300 import workloads

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sh = int(torch.cuda.current_stream().cuda_stream)
    n = args.profile_n
    key = int(sq.make_keys(2, 1)[0])
    base = workloads.throughput_base(3)
    kids = {"u32": C.SQ_KERNEL_U32, "u64": C.SQ_KERNEL_U64, "batch": C.SQ_KERNEL_BATCH,
            "uniform2_f32": C.SQ_KERNEL_UNIFORM2_F32, "uniform_f64": C.SQ_KERNEL_UNIFORM_F64,
            "uniform_f32": C.SQ_KERNEL_UNIFORM_F32, "uniform_bf16": C.SQ_KERNEL_UNIFORM_BF16,
            "normal_f32": C.SQ_KERNEL_NORMAL_F32, "fused": C.SQ_KERNEL_FUSED}
    if args.profile in ("u32_stride3", "u64_stride3", "keys_u32", "keys_u64"):
        return profile_next_rows(args, torch, sq, C, dev, sh, n, key)
    # ragged batches of many streams, each in a fixed launch configuration (set
    # directly, so that no tuning launch precedes the profiled ones), with
    # log-uniform lengths in [lo, hi):
    #   batch_mid:   2^14 streams, [3e3, 3e4) (mean ~1.2e4): tile kernel st32.cs,
    #                block 128, as many CTAs per SM as fit;
    #   batch_short: 2^20 streams, [30, 300) (mean ~117): flattened warps,
    #                block 512, as many CTAs per SM as fit;
    #   batch_tiny:  2^22 streams, [3, 30) (mean ~11): the same.
    regimes = {"batch_mid": (1 << 14, 3e3, 3e4, "st32.cs", 128),
               "batch_short": (1 << 20, 30, 300, "flat-seg8", 64),
               "batch_tiny": (1 << 22, 3, 30, "flat-warp", 128)}
    if args.profile in regimes:
        S, lo, hi, vname, block = regimes[args.profile]
        vname = args.profile_variant or vname
        block = args.profile_block or block
        bt = workloads.ragged_batch(S, seed=7, lo=lo, hi=hi)
        k = torch.from_numpy(sq.make_keys(7, bt.nstreams).view(np.int64)).to(dev)
        bb = torch.from_numpy(bt.bases.view(np.int64)).to(dev)
        ll = torch.from_numpy(bt.lengths).to(dev)
        oo = torch.from_numpy(bt.offsets).to(dev)
        out = torch.empty(bt.total, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        v = [i for i in range(C.sq_num_variants(C.SQ_KERNEL_BATCH))
             if C.sq_variant_name(C.SQ_KERNEL_BATCH, i) == vname][0]
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, v, block, 0)
        c = C.sq_get_config(C.SQ_KERNEL_BATCH, 0)
        print(f"profile config: {C.sq_variant_name(C.SQ_KERNEL_BATCH, c.variant)} block {c.block} "
              f"ctas/SM {c.ctas_per_sm}", flush=True)
        for _ in range(5):
            C.sq_batch(k.data_ptr(), bb.data_ptr(), ll.data_ptr(), oo.data_ptr(), bt.nstreams,
                       out.data_ptr(), sh)
        torch.cuda.synchronize()
        print(f"profile case {args.profile} streams={bt.nstreams} samples={bt.total} done",
              flush=True)
        return 0
    set_n = 64 if args.profile == "batch" else n  # the batch case holds 64 streams
    if args.tune_file and os.path.exists(args.tune_file):
        # use the configuration tuned for the benchmark's size of this kernel
        C.sq_autotune_load(args.tune_file)
        # the benchmark's entry: by output count, for the batch by stream count
        # (the 4096-stream workload's bucket, applied to this case's 64 streams)
        full = {"u32": N32, "u64": N64, "batch": 4096}.get(args.profile, 1 << 30)
        c = C.sq_get_config(kids[args.profile], full)
        C.sq_set_config(kids[args.profile], set_n, c.variant, c.block, c.ctas_per_sm)
    elif not args.no_tune:
        C.sq_autotune(kids[args.profile], n)
    c = C.sq_get_config(kids[args.profile], set_n)
    print(f"profile config: {C.sq_variant_name(kids[args.profile], c.variant)} block {c.block} "
          f"ctas/SM {c.ctas_per_sm}", flush=True)
    if args.profile == "fused":
        S, cps = max(1, n >> 18), 1 << 18  # --profile-n 2^30: 2^12 streams, ~1,600 counters per lane per item
        k = torch.from_numpy(sq.make_keys(13, S).view(np.int64)).to(dev)
        b = torch.zeros(S, dtype=torch.int64, device=dev)
        x = torch.empty(S, dtype=torch.int32, device=dev)
        s_ = torch.empty(S, dtype=torch.int64, device=dev)
        h = torch.empty(256, dtype=torch.int64, device=dev)
        run = lambda: C.sq_fused_stats(k.data_ptr(), b.data_ptr(), S, cps, x.data_ptr(),  # noqa: E731
                                       s_.data_ptr(), h.data_ptr(), sh)
    elif args.profile == "batch":
        bt = workloads.ragged_batch(64, seed=7, lo=n / 128, hi=n / 48)
        k = torch.from_numpy(sq.make_keys(7, bt.nstreams).view(np.int64)).to(dev)
        bb = torch.from_numpy(bt.bases.view(np.int64)).to(dev)
        ll = torch.from_numpy(bt.lengths).to(dev)
        oo = torch.from_numpy(bt.offsets).to(dev)
        out = torch.empty(bt.total, dtype=torch.int32, device=dev)
        run = lambda: C.sq_batch(k.data_ptr(), bb.data_ptr(), ll.data_ptr(), oo.data_ptr(),  # noqa: E731
                                 bt.nstreams, out.data_ptr(), sh)
    else:
        fn = {"u32": C.sq_u32, "u64": C.sq_u64, "uniform_f32": C.sq_uniform_f32,
              "uniform_bf16": C.sq_uniform_bf16, "normal_f32": C.sq_normal_f32,
              "uniform2_f32": C.sq_uniform2_f32, "uniform_f64": C.sq_uniform_f64}[args.profile]
        es = {"u64": 8, "uniform_bf16": 2, "uniform_f64": 8}.get(args.profile, 4)
        out = torch.empty(n * es, dtype=torch.uint8, device=dev)
        run = lambda: fn(key, base, n, out.data_ptr(), sh)  # noqa: E731
    for _ in range(5):
        run()
    torch.cuda.synchronize()
    print(f"profile case {args.profile} n={n} done", flush=True)
    return 0


def profile_next_rows(args, torch, sq, C, dev, sh, n, key):
    """Strided counters (stride 3) and key-counter mode: fixed launch shapes,
    no tuning table. Key-counter mode uses n / 4 keys (2^22 distinct, tiled)."""
    import numpy as np

    if args.profile.startswith("keys"):
        nk = max(1 << 22, n >> 2)
        k = torch.from_numpy(sq.make_keys(17, 1 << 22).view(np.int64)).to(dev).repeat(nk >> 22)
        nk = k.numel()
        out = torch.empty(nk * 8, dtype=torch.uint8, device=dev)
        fn = C.sq_keys_u32 if args.profile == "keys_u32" else C.sq_keys_u64
        run = lambda: fn(k.data_ptr(), nk, 0, out.data_ptr(), sh)  # noqa: E731
    else:
        fn = C.sq_u32_strided if args.profile == "u32_stride3" else C.sq_u64_strided
        out = torch.empty(n * 8, dtype=torch.uint8, device=dev)
        run = lambda: fn(key, 5, 3, n, out.data_ptr(), sh)  # noqa: E731
    for _ in range(5):
        run()
    torch.cuda.synchronize()
    print(f"profile case {args.profile} n={n} done", flush=True)
    return 0


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.profile:
        return profile_case(args)
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
