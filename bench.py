#!/usr/bin/env python
"""Benchmark of the runtime-specialized update chain (FP64 size sweep).

One step = for each N in {3, 4, 5, 7, 8, 12, 16, 24, 32}: cj_specialize
(a cache hit: the lookup is part of the path) and cj_launch of the JIT
instantiation over batch = floor(2^27 / N^2) instances with T = 64.
Prints one JSON line (see the repository's bench contract); `value` is the
whole-job FP64 GFLOP/s of the specialized kernels, `generic` the same for the
generic runtime-N kernel, `aot` for the ahead-of-time set {4, 8, 16, 32}.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cj|reference]

--impl reference times the CPU oracle (the plain FP64 C loops) on this
host's cores on a bounded sample of the same workload.
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

METRIC = "specialized vs generic GFLOP/s and % roofline at stated error; JIT compile ms p50"
SWEEP_N = (3, 4, 5, 7, 8, 12, 16, 24, 32)
AOT_N = (4, 8, 16, 32)
T_STEPS = 64
WORKLOAD = ("update chain X_{k+1} = X_k + X_k A/(N T), FP64 size sweep N in {3,4,5,7,8,12,16,24,32}, "
            "T = 64, batch = floor(2^27/N^2) per N, row-major, entries U[-1,1) (SplitMix64 seed 0xC1A2)")


def chain_flops(batch: int, n: int, steps: int) -> float:
    return float(batch) * steps * (2.0 * n ** 3 + 2.0 * n ** 2)


def chain_bytes(batch: int, n: int, esize: int) -> float:
    return float(batch) * 2 * n * n * esize


# Roofline denominators.  FP64: the nominal B300 FP64 rate (1.25 TFLOP/s;
# about 2 FP64 FMA lanes per SM per clock).  FP32: 148 SMs x 128 FMA lanes
# x 2 flops x 2032 MHz.  HBM: the measured copy bandwidth.
PEAK_TFLOPS = {"f64": 1.25, "f32": 148 * 128 * 2 * 2.032e9 / 1e12}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per instance of
# the sweep's roofline kernel, from the ncu capture summarised in
# profiles/update_chain_f64_n32_dram_traffic.md (65,536 instances, 1.07 GB of
# A and X: the writes leave L2 except its last ~40 MB; scaled by the instance
# count, the kernel's traffic grows in proportion).  None for any other
# kernel: the counters then do not describe it.
TRAFFIC_PER_INSTANCE = {"update_chain<double, 32, 0, 1, 8>": (550.644736e6 + 494.461952e6) / 65536}


def measured_peak(key: str, default: float) -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return default


def hbm_peak_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6400.0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks only; no data-path collective)
# ---------------------------------------------------------------------------
def dist_setup(n_gpus: int):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    from paper_1904_08555_b300 import shard
    shard.barrier(world)


def max_over_ranks(world, v: float) -> float:
    from paper_1904_08555_b300 import shard
    return shard.max_over_ranks(world, v, device="cuda")


# ---------------------------------------------------------------------------
# CPU oracle leg (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample_sizes(budget_flops: float) -> dict:
    per_n = budget_flops / len(SWEEP_N)
    return {n: max(8, int(per_n / chain_flops(1, n, T_STEPS))) for n in SWEEP_N}


def calibrated_sizes(seconds: float) -> dict:
    """Sample sizes for about `seconds` of oracle time on this host's cores."""
    sizes = oracle_sample_sizes(2e8 * (os.cpu_count() or 1))
    f, s, _, _ = run_oracle_sweep(sizes)
    return oracle_sample_sizes(f / s * seconds)


def run_oracle_sweep(sizes: dict, rank_offset: int = 0):
    """Oracle on the first sizes[n] instances of each size; returns (flops, seconds, outputs)."""
    import oracle
    cores = os.cpu_count() or 1
    flops, secs, outs = 0.0, 0.0, {}
    for n in SWEEP_N:
        A = synth.uniform_np(synth.SEED_CHAIN_SWEEP, synth.STREAM_A + rank_offset * synth.chain_batch(n) * n * n,
                             sizes[n] * n * n).reshape(sizes[n], n, n)
        t0 = time.perf_counter()
        X = oracle.update_chain(A, T_STEPS, nthreads=cores)
        secs += time.perf_counter() - t0
        flops += chain_flops(sizes[n], n, T_STEPS)
        outs[n] = X
    return flops, secs, outs, cores


def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # every step is one oracle sweep over the same sample as the cpu_baseline
    # leg of the GPU arm (about --cpu-seconds of work), so both legs time
    # the oracle the same way
    sizes = calibrated_sizes(args.cpu_seconds)
    for _ in range(args.warmup):
        run_oracle_sweep(sizes)
    tot_f, tot_s = 0.0, 0.0
    for _ in range(args.steps):
        f, s, _, cores = run_oracle_sweep(sizes)
        tot_f += f
        tot_s += s
    value = tot_f / tot_s / 1e9
    sample = (f"per step: the first {sizes[3]} (N=3) .. {sizes[32]} (N=32) instances of each of the "
              f"{len(SWEEP_N)} sizes, {tot_f / args.steps / 1e9:.1f} GFLOP")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def cj_arm(args):
    import torch
    from paper_1904_08555_b300 import cj, shard

    world, rank, local = dist_setup(args.gpus)
    dev = torch.cuda.current_device()
    # asynchronous specializer: instantiations compile on background threads
    # in parallel; every timed launch below waits for its handle first
    compile_threads = min(16, os.cpu_count() or 4)
    cj.init(sync=False, compile_threads=compile_threads, device=dev)
    stream = torch.cuda.Stream()

    # inputs: rank r holds instances [r*batch, (r+1)*batch) of each size
    A, X, batch = {}, {}, {}
    with torch.cuda.stream(stream):
        for n in SWEEP_N:
            b = synth.chain_batch(n)
            batch[n] = b
            A[n] = synth.uniform_torch(synth.SEED_CHAIN_SWEEP, synth.STREAM_A + shard.element_offset(rank, b, n),
                                       b * n * n, "cuda").view(b, n, n)
            X[n] = torch.empty_like(A[n])
    stream.synchronize()

    t0 = time.perf_counter()
    spec = {n: cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_NO_AOT) for n in SWEEP_N}
    for h in spec.values():
        assert h.wait() == cj.CJ_OK
    compile_wall = time.perf_counter() - t0
    st = cj.stats()
    sweep_compile = {"p50": st["compile_ms_p50"], "p95": st["compile_ms_p95"], "keys": len(SWEEP_N)}
    gen = {n: cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_GENERIC) for n in SWEEP_N}
    aot = {n: cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n) for n in AOT_N}
    assert all(h.variant == "jit" for h in spec.values())
    assert all(h.variant == "aot" for h in aot.values())

    step_flops = sum(chain_flops(batch[n], n, T_STEPS) for n in SWEEP_N)

    def run(kind, sizes, events=None):
        for n in sizes:
            if kind == "spec":
                h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_NO_AOT)
            elif kind == "aot":
                h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n)
            else:
                h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_GENERIC)
            if events is not None:
                events[n][0].record(stream)
            cj.launch_update_chain(h, A[n], X[n], T_STEPS, stream=stream)
            if events is not None:
                events[n][1].record(stream)

    def timed(kind, sizes, steps, warmup, clocks=None):
        for _ in range(warmup):
            run(kind, sizes)
        stream.synchronize()
        per = {n: [] for n in sizes}
        barrier(world)
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        evs = []
        e0.record(stream)
        for _ in range(steps):
            ev = {n: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for n in sizes}
            run(kind, sizes, ev)
            evs.append(ev)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        barrier(world)
        ms = e0.elapsed_time(e1)
        for ev in evs:
            for n in sizes:
                per[n].append(ev[n][0].elapsed_time(ev[n][1]))
        ms = max_over_ranks(world, ms)
        return ms, {n: statistics.mean(v) for n, v in per.items()}, clk

    sampler = ClockSampler(dev)
    ms_spec, per_spec, clocks = timed("spec", SWEEP_N, args.steps, args.warmup, sampler)
    ms_gen, per_gen, _ = timed("generic", SWEEP_N, args.steps, 1)
    ms_aot, per_aot, _ = timed("aot", AOT_N, args.steps, 1)

    value = world * step_flops * args.steps / (ms_spec * 1e-3) / 1e9
    gen_value = world * step_flops * args.steps / (ms_gen * 1e-3) / 1e9
    micro64 = cj.measure_fma_peak(cj.F64, stream.cuda_stream)
    tensor64 = cj.measure_fma_peak(cj.F64, stream.cuda_stream, tensor=True)
    peak64 = PEAK_TFLOPS["f64"]
    per_n = []
    for n in SWEEP_N:
        f = chain_flops(batch[n], n, T_STEPS)
        row = {"N": n, "batch": batch[n], "spec_ms": per_spec[n], "generic_ms": per_gen[n],
               "spec_gflops": f / per_spec[n] / 1e6, "generic_gflops": f / per_gen[n] / 1e6,
               "speedup_vs_generic": per_gen[n] / per_spec[n],
               "spec_frac_of_fp64_peak": f / per_spec[n] / 1e9 / peak64,
               "mapping": {1: "row per thread", 2: "instance per thread",
                           4: "FP64 tensor cores"}.get(int.from_bytes(bytes.fromhex(spec[n].key_hex)[12:16], "little")),
               "spec_regs": spec[n].regs()[0], "generic_regs": gen[n].regs()[0]}
        if n in AOT_N:
            row["aot_ms"] = per_aot[n]
            row["aot_gflops"] = f / per_aot[n] / 1e6
        per_n.append(row)
    dom = max(SWEEP_N, key=lambda n: per_spec[n])
    achieved = chain_flops(batch[dom], dom, T_STEPS) / (per_spec[dom] * 1e-3) / 1e12
    dom_key = bytes.fromhex(spec[dom].key_hex)
    dom_tile = [int.from_bytes(dom_key[12 + 4 * i:16 + 4 * i], "little") for i in range(2)]
    dom_name = f"update_chain<double, {dom}, 0, {dom_tile[0]}, {dom_tile[1]}>"
    traffic = TRAFFIC_PER_INSTANCE.get(dom_name)
    traffic = traffic * batch[dom] if traffic is not None else None

    # end to end through the C ABI with host buffers: every step copies each
    # size's A in from pinned host memory, launches, and copies its X out.
    # The copies run on two copy streams, so that size n's copy-in and size
    # n-1's copy-out overlap size n-1's and n's compute, as a pipelined
    # caller runs them; events order each buffer's reuse across steps (A[n]
    # is rewritten once the previous launch read it, X[n] once the previous
    # copy-out read it).  Every copy of every step is inside the timed region.
    h2d = sum(chain_bytes(batch[n], n, 8) / 2 for n in SWEEP_N)
    host_A = {n: A[n].cpu().pin_memory() for n in SWEEP_N}
    host_X = {n: torch.empty(A[n].shape, dtype=torch.float64).pin_memory() for n in SWEEP_N}
    copy_in, copy_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_in = {n: torch.cuda.Event() for n in SWEEP_N}     # A[n] copied in
    ev_run = {n: torch.cuda.Event() for n in SWEEP_N}    # X[n] computed; A[n] read
    ev_out = {n: torch.cuda.Event() for n in SWEEP_N}    # X[n] copied out

    def e2e_step(first):
        for n in SWEEP_N:
            if not first:
                copy_in.wait_event(ev_run[n])
            with torch.cuda.stream(copy_in):
                A[n].copy_(host_A[n], non_blocking=True)
            ev_in[n].record(copy_in)
            stream.wait_event(ev_in[n])
            if not first:
                stream.wait_event(ev_out[n])
            h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_NO_AOT)
            cj.launch_update_chain(h, A[n], X[n], T_STEPS, stream=stream)
            ev_run[n].record(stream)
            copy_out.wait_event(ev_run[n])
            with torch.cuda.stream(copy_out):
                host_X[n].copy_(X[n], non_blocking=True)
            ev_out[n].record(copy_out)

    with torch.cuda.stream(stream):
        e2e_step(True)
        torch.cuda.synchronize(dev)
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        copy_in.wait_event(e0)      # no copy starts before the timed region
        copy_out.wait_event(e0)
        for _ in range(args.steps):
            e2e_step(False)
        stream.wait_event(ev_out[SWEEP_N[-1]])   # the last copy-out ends the region
        e1.record(stream)
        e1.synchronize()
    ms_e2e = max_over_ranks(world, e0.elapsed_time(e1))
    e2e_value = world * step_flops * args.steps / (ms_e2e * 1e-3) / 1e9

    st = cj.stats()
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_spec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2 (1.07 GB of A per size)",
                       "instances_per_step_per_gpu": sum(batch.values())},
            "generic": {"value": gen_value, "unit": "GFLOP/s", "ms_per_step": ms_gen / args.steps},
            "speedup_vs_generic": value / gen_value,
            "jit_compile_ms_p50": st["compile_ms_p50"], "jit_compile_ms_p95": st["compile_ms_p95"],
            "jit_compile_ms_sweep_keys": sweep_compile, "jit_compile_threads": compile_threads,
            "lookup_ns_p50": st["lookup_ns_p50"], "compile_wall_s_9_sizes": compile_wall,

            "fp64_fma_pipe_tflops_measured": micro64, "fp64_tensor_tflops_measured": tensor64,
            "fp64_nominal_tflops": PEAK_TFLOPS["f64"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                         "frac": achieved / peak64, "traffic": traffic,
                         "traffic_unit": "bytes per launch (ncu dram read + write at 65,536 instances, scaled "
                                         "to the launch's instances)",
                         "algorithmic_bytes": chain_bytes(batch[dom], dom, 8),
                         "kernel": dom_name,
                         "peak_source": "nominal B300 FP64 rate, 1.25 TFLOP/s (profiling recipe); the measured "
                                        "FMA-chain and mma.sync f64 microbenchmarks are reported beside it"},
            "per_n": per_n,
            "e2e": {"value": e2e_value, "unit": "GFLOP/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(h2d)},
            "gpu_launches": args.steps * len(SWEEP_N),
            "clocks": clocks}

    if rank == 0 and not args.no_cpu_baseline:
        sizes = calibrated_sizes(args.cpu_seconds)   # the reference arm's per-step sample
        f, s, outs, cores = run_oracle_sweep(sizes, rank_offset=0)
        worst = 0.0
        for n in SWEEP_N:
            got = X[n][: sizes[n]].cpu().numpy()
            ref = outs[n]
            err = np.linalg.norm((got - ref).reshape(len(ref), -1), axis=1) / np.linalg.norm(ref.reshape(len(ref), -1), axis=1)
            worst = max(worst, float(err.max()))
        line["cpu_baseline"] = {"value": f / s / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                                "sample": f"first {sizes[3]} (N=3) .. {sizes[32]} (N=32) instances of each size, "
                                          f"{f / 1e9:.1f} GFLOP, {s:.1f} s"}
        line["max_rel_frobenius_error_vs_oracle"] = worst
    # the other workloads, in the same run: config 1 (64 x N = 8), config 3
    # (LTimes, 36 orders, FP64 and FP32) and config 4 (10,000-instance uneven
    # batch, FP64 / FP32 / BF16), each with its error against the oracle
    workloads = {}
    if rank == 0 and not args.sweep_only:
        del A, X, host_A, host_X
        torch.cuda.empty_cache()
        lt_reps = max(3, min(args.steps, 5))
        with torch.cuda.stream(stream):
            workloads["config1_small"] = run_config1(torch, cj, stream, args.warmup)
            for d in ("f64", "f32"):
                _request_ltimes(cj, d)
                workloads["config3_ltimes_" + d] = run_config3(torch, cj, stream, d, 1 << 18, lt_reps)
            st13 = cj.stats()
            ref = uneven_reference(("f64", "f32", "bf16"))
            for d in ("f64", "f32", "bf16"):
                workloads["config4_uneven_" + d] = run_config4(torch, cj, stream, d, 10, args.warmup, ref)
        workloads["jit_compile_ms_configs_1_to_3"] = {"p50": st13["compile_ms_p50"], "p95": st13["compile_ms_p95"],
                                                      "compiles": st13["compiles_ok"],
                                                      "compile_threads": compile_threads}
    line["workloads"] = workloads
    line["wait_timeouts"] = cj.stats()["wait_timeouts"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    cj.shutdown()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("cj", "reference"), default="cj")
    p.add_argument("--workload", choices=("sweep", "small", "sweep32", "ltimes", "uneven", "kernel", "costmodel", "eigen",
                                          "pch", "mass"),
                   default="sweep",
                   help="sweep (default): the FP64 size sweep; the others are secondary measurements")
    p.add_argument("--dtype", choices=("f64", "f32", "bf16"), default="f64", help="ltimes / uneven precision")
    p.add_argument("--ltimes-z", type=int, default=1 << 18)
    p.add_argument("--kernel", choices=("chain", "chain-generic", "ltimes", "ltimes-generic", "eigen", "eigen-generic"),
                   default="chain")
    p.add_argument("--n", type=int, default=32)
    p.add_argument("--batch", type=int, default=16384)
    p.add_argument("--layout-in", type=int, default=0)
    p.add_argument("--layout-out", type=int, default=0)
    p.add_argument("--tile", type=int, nargs=4, default=None, help="explicit tile for --workload kernel")
    p.add_argument("--heldout", type=int, default=2000)
    p.add_argument("--train-steps", type=int, default=4000)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--sweep-only", action="store_true", help="default line without the config 1/3/4 sub-objects")
    p.add_argument("--cpu-seconds", type=float, default=4.0,
                   help="oracle seconds per sweep sample: one reference-arm step, and the cpu_baseline leg")
    args = p.parse_args()
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    def lt_alt_tiles(lin, lout):
        # extra LTimes tiles timed beside the default, per (in, out) pair
        if args.dtype != "f32":
            return []
        gi, go = lin in (1, 4), lout in (1, 4)
        tg = 1 if not (gi or go) else (8 if (gi and lout in (0, 2)) or (go and lin in (0, 2)) else 32)
        def tmem(boxes, stages, nconv, g=tg):   # tcgen05 with the A operand in tensor memory (mode 6)
            return (g, 128 // g, 32 * (6 + nconv), (boxes << 20) | (6 << 16) | (stages << 8) | nconv)
        alts = [("tma_b4s2", (tg, 128 // tg, 32 * 14, (4 << 20) | (5 << 16) | (2 << 8) | 8)),
                ("tc_s2p8", (tg, 128 // tg, 32 * 13, (4 << 16) | (2 << 8) | 8)),
                ("tmem_b4s2", tmem(4, 2, 8)), ("tmem_b6s4", tmem(6, 4, 8)), ("tmem_b8s6", tmem(8, 6, 8)),
                ("tmem_b6s4c4", tmem(6, 4, 4))]
        if tg == 8:   # in and out have different fastest column axes: a 16 x 8 box beside the rule's 8 x 16
            alts.append(("tmem_b6s4_tg16", tmem(6, 4, 8, 16)))
        return alts
    args.lt_alt_tiles = lt_alt_tiles
    if args.impl == "reference":
        reference_arm(args)
    else:
        # 32 hardware work queues instead of 8, so that up to 32 of a grouped
        # plan's kernels overlap when it is launched on its streams; read when
        # the CUDA context is created, hence before torch touches the device
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
        if args.workload != "sweep":
            secondary(args)
        else:
            cj_arm(args)



# ---------------------------------------------------------------------------
# Secondary workloads (not the default line): --workload small|sweep32|ltimes|uneven
# ---------------------------------------------------------------------------
def _events(torch, stream, fn, reps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _key_tile(h):
    key = bytes.fromhex(h.key_hex)
    return [int.from_bytes(key[12 + 4 * i:16 + 4 * i], "little") for i in range(4)]


def _relF_rows(got, ref):
    got = got.reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


def run_config1(torch, cj, stream, W):
    """64 FP64 8x8 chains, T = 100: the library's default tile, the tile the
    autotuner picks for this batch, the AoT specialization and the generic
    kernel, each checked against the oracle on every instance."""
    import oracle
    n, b, steps, reps = 8, 64, 100, 200
    A_np = synth.chain_inputs_np(synth.SEED_CHAIN_SMALL, b, n)
    ref = oracle.update_chain(A_np, steps)
    A = torch.from_numpy(A_np).cuda()
    X = torch.empty_like(A)
    f = chain_flops(b, n, steps)
    row, worst = {"N": n, "batch": b, "T": steps}, 0.0

    def timed(name, h):
        nonlocal worst
        assert h.wait() == cj.CJ_OK
        fn = lambda: cj.launch_update_chain(h, A, X, steps, stream=stream)
        _events(torch, stream, fn, W)
        ms = _events(torch, stream, fn, reps)
        stream.synchronize()
        worst = max(worst, float(_relF_rows(X.cpu().numpy(), ref).max()))
        row.update({name + "_us": ms * 1e3, name + "_gflops": f / ms / 1e6, name + "_regs": h.regs()[0],
                    name + "_tile": _key_tile(h)})

    timed("default", cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_NO_AOT))
    timed("aot", cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n))
    timed("generic", cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_GENERIC))
    # the autotuner's choice for this exact batch (tile spaces include one
    # instance per block, which a 64-instance batch needs)
    best, times = cj.autotune(cj.K_UPDATE_CHAIN, cj.F64, cj.chain_launch_vals(A, X, steps), b, stream, reps=20, n=n)
    timed("autotuned", cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, tile=best))
    row["candidates_us"] = {str(list(t)): v * 1e3 for t, v in times}
    return {"value": f / row["autotuned_us"] / 1e3, "dtype": "f64", "us": row["autotuned_us"],
            "generic": {"value": f / row["generic_us"] / 1e3, "unit": "GFLOP/s", "us": row["generic_us"]},
            "speedup_vs_generic": row["generic_us"] / row["autotuned_us"],
            "default_tile_speedup_vs_generic": row["generic_us"] / row["default_us"],
            "max_rel_frobenius_error_vs_oracle": worst, "per_n": [row],
            "roofline": {"bound": "alu", "peak": PEAK_TFLOPS["f64"], "unit": "TFLOP/s",
                         "frac": f / row["autotuned_us"] / 1e6 / PEAK_TFLOPS["f64"],
                         "note": "latency-bound by size: 64 instances on 148 SMs"},
            "config": {"workload": "update chain, 64 FP64 8x8 matrices, T = 100 (seed 0xC1A1); value = the "
                                   "autotuned JIT instantiation, the default tile beside it"}}


def _request_ltimes(cj, dtype):
    """Request the 36 default-tile LTimes instantiations at once (they compile
    in parallel in asynchronous mode) and wait for all of them."""
    dt = cj.F64 if dtype == "f64" else cj.F32
    hs = [cj.specialize(cj.K_LTIMES, dt, layout_a=lin, layout_b=lout, m=36, d=96)
          for lin in range(6) for lout in range(6)]
    for h in hs:
        assert h.wait() == cj.CJ_OK


def run_config3(torch, cj, stream, dtype, Z, reps, alt_tiles=None, samples=384):
    """LTimes over all 36 (in, out) storage orders at M 36, D 96, G 32: the
    default (specialized) tile and the generic kernel, mean ms per order pair;
    each timed output checked against the oracle on `samples` seeded columns;
    expired bounded waits of the tensor-core kernels read afterwards."""
    import oracle
    dt = cj.F64 if dtype == "f64" else cj.F32
    tdt = torch.float64 if dt == cj.F64 else torch.float32
    es = 8 if dt == cj.F64 else 4
    M, D, G = 36, 96, 32
    L, _ = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, 1, 1)
    Lt = torch.from_numpy(L).to("cuda", tdt)
    x = synth.uniform_torch(synth.SEED_LTIMES, synth.STREAM_A, D * G * Z, "cuda").view(D, G, Z).to(tdt)
    rng = np.random.default_rng(0xC1A3)
    gs = torch.from_numpy(rng.integers(0, G, samples)).cuda()
    zs = torch.from_numpy(rng.integers(0, Z, samples)).cuda()
    cols = x[:, gs, zs].double().cpu().numpy()
    ref = oracle.ltimes(L, cols.ravel(), 1, samples, 0, 0).reshape(M, samples)   # [m][sample]
    xin = {lin: x.permute(*synth.LAYOUT_PERMS[lin]).contiguous().view(-1) for lin in range(6)}
    del x
    o = torch.empty(M * G * Z, device="cuda", dtype=tdt)
    f = 2.0 * M * D * G * Z
    byt = es * ((D + M) * G * Z + M * D)

    def err_of(lout):
        pout = o.view(*[(M, G, Z)[p] for p in synth.LAYOUT_PERMS[lout]])
        canon = pout.permute(*np.argsort(synth.LAYOUT_PERMS[lout]).tolist())
        got = canon[:, gs, zs].double().cpu().numpy()
        return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    wt0 = cj.stats()["wait_timeouts"]
    rows, tot_s, tot_g, worst = [], 0.0, 0.0, 0.0
    # every alternative tile is requested first, so that they compile side by side
    alts = {(lin, lout): [(name, cj.specialize(cj.K_LTIMES, dt, layout_a=lin, layout_b=lout, m=M, d=D, tile=alt))
                          for name, alt in (alt_tiles(lin, lout) if alt_tiles else [])]
            for lin in range(6) for lout in range(6)}
    for lin in range(6):
        for lout in range(6):
            hs = cj.specialize(cj.K_LTIMES, dt, layout_a=lin, layout_b=lout, m=M, d=D)
            hg = cj.specialize(cj.K_LTIMES, dt, layout_a=lin, layout_b=lout, m=M, d=D, flags=cj.FLAG_GENERIC)
            fs = lambda: cj.launch_ltimes(hs, Lt, xin[lin], o, G, Z, stream=stream)
            fg = lambda: cj.launch_ltimes(hg, Lt, xin[lin], o, G, Z, stream=stream)
            _events(torch, stream, fs, 1)
            ms_s = _events(torch, stream, fs, reps)
            e_s = err_of(lout)
            _events(torch, stream, fg, 1)
            ms_g = _events(torch, stream, fg, reps)
            e_g = err_of(lout)
            worst = max(worst, e_s, e_g)
            row = {"in": synth.LAYOUT_NAMES[lin], "out": synth.LAYOUT_NAMES[lout].replace("D", "M"),
                   "spec_ms": ms_s, "generic_ms": ms_g, "spec_gbs": byt / ms_s / 1e6,
                   "speedup_vs_generic": ms_g / ms_s, "spec_rel_err": e_s, "tile": _key_tile(hs)}
            for name, ha in alts[(lin, lout)]:
                ha.wait()
                fa = lambda: cj.launch_ltimes(ha, Lt, xin[lin], o, G, Z, stream=stream)
                _events(torch, stream, fa, 1)
                row[name + "_ms"] = _events(torch, stream, fa, reps)
                row[name + "_rel_err"] = e_a = err_of(lout)
                worst = max(worst, e_a)
            rows.append(row)
            tot_s += ms_s
            tot_g += ms_g
    wait_timeouts = cj.stats()["wait_timeouts"] - wt0
    del xin, o
    # Compute bound of the default kernel: FP32 runs 3xTF32 on the tensor
    # cores (tile modes 4-6: three TF32 products per multiply-add, TF32 peak
    # = measured bf16 x the nominal 1.1 / 2.25 ratio); FP64 runs on the
    # FP64 pipe at its nominal rate.
    tc = dt == cj.F32 and all(((r["tile"][3] >> 16) & 0xF) in (4, 5, 6) for r in rows)
    if tc:
        peak = measured_peak("bf16_tflops", 1800.0) * 1.1 / 2.25
        t_alu = 3 * f / (peak * 1e12) * 1e3
    else:
        peak = PEAK_TFLOPS[dtype]
        t_alu = f / (peak * 1e12) * 1e3
    t_hbm = byt / (hbm_peak_gbs() * 1e9) * 1e3
    mean_ms = tot_s / 36
    bound = "tensor" if tc and t_alu >= t_hbm else "alu" if t_alu >= t_hbm else "hbm"
    rf = {"bound": bound, "roofline_ms": max(t_alu, t_hbm), "mean_ms": mean_ms,
          "frac": max(t_alu, t_hbm) / mean_ms, "compute_frac": t_alu / mean_ms, "hbm_frac": t_hbm / mean_ms,
          "compute_peak_tflops": peak, "compute_unit": "TF32 tensor (3 passes)" if tc else dtype + " pipe",
          "hbm_gbs": hbm_peak_gbs()}
    if bound == "hbm":
        rf.update({"achieved": byt / mean_ms / 1e6, "peak": hbm_peak_gbs(), "unit": "GB/s",
                   "algorithmic_bytes": byt})
    else:
        rf.update({"achieved": f / mean_ms / 1e9, "peak": peak, "unit": "TFLOP/s"})
    return {"value": 36 * f / tot_s / 1e6, "dtype": dtype, "mean_ms": mean_ms,
            "generic": {"value": 36 * f / tot_g / 1e6, "unit": "GFLOP/s", "mean_ms": tot_g / 36},
            "speedup_vs_generic": tot_g / tot_s,
            "min_speedup_vs_generic": min(r["speedup_vs_generic"] for r in rows),
            "max_rel_frobenius_error_vs_oracle": worst,
            "error_sample": f"{samples} seeded (g, z) columns x all 36 moments, every order pair, every kernel timed",
            "wait_timeouts": wait_timeouts, "valid": wait_timeouts == 0,
            "roofline": rf, "per_pair": rows,
            "config": {"workload": f"LTimes out[m][g][z] = sum_d L[m][d] in[d][g][z], M=36 D=96 G=32 Z={Z}, "
                                   f"all 36 (in, out) storage orders, {dtype} (seed 0xC1A3)"}}


# The paper's Laghos figure (Sec. 5): 2-D, 10,000 elements, runs labelled dNqM
# with N dofs and M quadrature points per dimension.
MASS_PAPER_CASES = ((2, 4), (2, 2), (4, 8), (2, 8), (4, 2), (4, 4), (8, 4), (8, 2))
# Throughput cases: the 2-D instantiations of the paper's Laghos listing, and
# 3-D ones, each about 2 GB of x, op and y.
MASS_CASES = ((2, 2, 2), (2, 2, 4), (2, 3, 4), (2, 3, 6), (2, 4, 6), (2, 4, 8), (2, 5, 8),
              (3, 2, 4), (3, 3, 4), (3, 3, 6), (3, 4, 6), (3, 4, 8), (3, 5, 8))


def mass_flops(dim, D, Q):
    """Sum-factorized flops per element: one 1-D contraction per dimension to
    the quadrature points and back (2 flops per multiply-add), plus the
    pointwise scaling."""
    if dim == 2:
        return 2.0 * 2 * (Q * D * D + Q * Q * D) + Q * Q
    return 2.0 * 2 * (Q * D ** 3 + Q * Q * D * D + Q ** 3 * D) + Q ** 3


def _mass_case(torch, cj, stream, oracle, dt, tdt, es, dim, D, Q, ne, K, W, samples=256):
    B1, op, x = synth.mass_inputs_torch(synth.SEED_MASS, dim, D, Q, ne, "cuda")
    op, x = op.to(tdt), x.to(tdt)
    Bt = torch.from_numpy(B1).to("cuda", tdt)
    y = torch.empty_like(x)
    f = mass_flops(dim, D, Q) * ne
    row = {"dim": dim, "D": D, "Q": Q, "elements": ne, "laghos_key": hex((dim << 16) | ((D - 1) << 8) | (Q >> 1))}
    worst = 0.0
    forms = [("spec", 0), ("generic", cj.FLAG_GENERIC), ("staged", 0)]
    if dim == 2 and D * Q + D * D <= 80:
        forms.append(("thread", 0))
    for name, fl in forms:
        # staged: the default tile's elements per block on the persistent kernel with staged loads;
        # thread: 2-D, one thread per element (128 per block)
        tile = ((row["tile"][0], 1, 0, 0) if name == "staged" else (128, 2, 0, 0) if name == "thread"
                else (0, 0, 0, 0))
        h = cj.specialize(cj.K_MASS, dt, n=D, m=Q, d=dim, flags=fl, tile=tile)
        h.wait()
        fn = lambda h=h: cj.launch_mass(h, Bt, op, x, y, ne, stream=stream)
        _events(torch, stream, fn, W)
        ms = _events(torch, stream, fn, K)
        stream.synchronize()
        rng = np.random.default_rng(dim * 100 + D * 10 + Q)
        it = torch.from_numpy(np.unique(rng.integers(0, ne, samples))).cuda()
        ref = oracle.mass(Bt.double().cpu().numpy(), op[it].double().cpu().numpy(), x[it].double().cpu().numpy(), dim)
        got = y[it].double().cpu().numpy()
        err = float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))
        worst = max(worst, err)
        row.update({name + "_us": ms * 1e3, name + "_gflops": f / ms / 1e6, name + "_regs": h.regs()[0],
                    name + "_rel_err": err})
        if name == "spec":
            row["tile"] = _key_tile(h)
    row["speedup_vs_generic"] = row["generic_us"] / row["spec_us"]
    row["staged_speedup"] = row["spec_us"] / row["staged_us"]
    if "thread_us" in row:
        row["thread_speedup"] = row["spec_us"] / row["thread_us"]
    return row, f, worst


def run_mass_workload(torch, cj, stream, dtype, K, W):
    """Mass operator of tensor-product elements (the Laghos kernel, Sec. 5):
    (1) the paper's figure cases, 2-D, 10,000 elements, specialized against
    generic (the paper reports this ratio); (2) throughput cases of about
    2 GB each, with the roofline max(FP pipe, HBM) time per case.  Every
    timed output is checked against the oracle on 256 sampled elements."""
    import oracle
    dt = cj.F64 if dtype == "f64" else cj.F32
    tdt = torch.float64 if dt == cj.F64 else torch.float32
    es = 8 if dt == cj.F64 else 4
    peak = PEAK_TFLOPS[dtype]
    worst = 0.0
    paper = []
    for D, Q in MASS_PAPER_CASES:
        row, _, w = _mass_case(torch, cj, stream, oracle, dt, tdt, es, 2, D, Q, 10000, max(K, 20), W)
        row["run"] = f"d{D}q{Q}"
        paper.append(row)
        worst = max(worst, w)
    rows, tot_f, tot_s, tot_g, tot_roof = [], 0.0, 0.0, 0.0, 0.0
    for dim, D, Q in MASS_CASES:
        ne = (1 << 31) // ((2 * D ** dim + Q ** dim) * es)
        row, f, w = _mass_case(torch, cj, stream, oracle, dt, tdt, es, dim, D, Q, ne, K, W)
        worst = max(worst, w)
        byt = float(es) * (2 * D ** dim + Q ** dim) * ne
        t_alu, t_hbm = f / (peak * 1e12) * 1e3, byt / (hbm_peak_gbs() * 1e9) * 1e3
        row.update({"roofline_ms": max(t_alu, t_hbm), "frac": max(t_alu, t_hbm) / (row["spec_us"] * 1e-3),
                    "bound": "alu" if t_alu >= t_hbm else "hbm", "spec_gbs": byt / (row["spec_us"] * 1e-3) / 1e6})
        rows.append(row)
        tot_f += f
        tot_s += row["spec_us"] * 1e-3
        tot_g += row["generic_us"] * 1e-3
        tot_roof += max(t_alu, t_hbm)
    return {"value": tot_f / tot_s / 1e6, "dtype": dtype,
            "generic": {"value": tot_f / tot_g / 1e6, "unit": "GFLOP/s"},
            "speedup_vs_generic": tot_g / tot_s, "min_speedup_vs_generic": min(r["speedup_vs_generic"] for r in rows),
            "paper_figure_cases": paper,
            "max_rel_frobenius_error_vs_oracle": worst, "per_case": rows,
            "roofline": {"bound": "max(pipe, hbm) per case", "frac": tot_roof / tot_s, "peak_tflops": peak,
                         "hbm_gbs": hbm_peak_gbs()},
            "config": {"workload": "mass operator y = B^T diag(op) B x of tensor-product elements: the paper's figure "
                                   f"runs {['d%dq%d' % c for c in MASS_PAPER_CASES]} (2-D, 10,000 elements) and "
                                   f"throughput cases (dim, D, Q) in {list(MASS_CASES)} of about 2 GB, {dtype} "
                                   "(seed 0xC1A6)",
                       "flops_per_element": "sum factorized: 2D 4(QD^2+Q^2D)+Q^2, 3D 4(QD^3+Q^2D^2+Q^3D)+Q^3"}}


def uneven_reference(dtypes):
    """Oracle X of the 10,000-instance uneven batch: from the FP64 pool, and
    from the pool rounded to FP32 (what the FP32 and BF16 plans read)."""
    import oracle
    n, t = synth.uneven_sizes(synth.SEED_UNEVEN, 10000)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN, n)
    cores = os.cpu_count() or 1
    ref = {"n": n, "t": t, "pool": pool, "off": off}
    if "f64" in dtypes:
        ref["f64"] = oracle.update_chain_uneven(n, t, off, pool, nthreads=cores)
    if "f32" in dtypes or "bf16" in dtypes:
        ref["f32"] = oracle.update_chain_uneven(n, t, off, pool.astype(np.float32).astype(np.float64),
                                                nthreads=cores)
    return ref


def _uneven_errors(got, ref, n, off):
    errs = np.empty(len(n))
    for nn in np.unique(n):
        idx = np.nonzero(n == nn)[0]
        rows = off[idx][:, None] + np.arange(nn * nn)[None, :]
        errs[idx] = np.linalg.norm(got[rows] - ref[rows], axis=1) / np.linalg.norm(ref[rows], axis=1)
    return errs


def run_config4(torch, cj, stream, dtype, K, W, ref):
    """The 10,000-instance uneven batch through grouped plans: default tiles,
    tiles and launch form chosen by the plan's autotuner, and the generic
    kernels.  Every form is timed -- the plan's one-launch dispatcher and one
    kernel per group, each as a CUDA graph and issued directly -- and every
    instance of each autotuned-plan form's output is checked against the
    oracle.  `value` is the autotuned plan as a user launches it (the form its
    autotuner kept; graph or direct, the faster)."""
    dt = {"f64": cj.F64, "f32": cj.F32, "bf16": cj.BF16}[dtype]
    tdt = torch.float64 if dt == cj.F64 else torch.float32
    n, t, pool, off = ref["n"], ref["t"], ref["pool"], ref["off"]
    A = torch.from_numpy(pool).to("cuda", tdt)
    X = torch.empty_like(A)
    f = float(np.sum(t * (2.0 * n ** 3 + 2.0 * n ** 2)))
    reps = max(K, 10)
    modes, changed, errs, disp = {}, 0, None, {}
    forms = {"dispatch_graph": (True, False), "dispatch_direct": (False, False),
             "per_group_graph": (True, True), "per_group_streams": (False, True)}
    for name, fl in (("default_tiles", 0), ("spec", 0), ("generic", cj.FLAG_GENERIC)):
        plan = cj.GroupPlan(dt, n, t, flags=fl)
        plan.wait()                     # every group's instantiation and the dispatcher compiled
        if name == "spec":
            # the plan's tiles chosen by its own autotuner (every candidate of the
            # 16 most expensive groups timed on the group's own work list), then
            # the faster launch form
            changed = plan.autotune(A, X, stream=stream, max_groups=16, reps=3)
            disp = plan.dispatcher()
        for form, (use_graph, per_group) in forms.items():
            if fl == cj.FLAG_GENERIC and not per_group:
                continue                # a generic plan has no dispatcher
            fn = lambda: plan.launch(A, X, stream=stream, use_graph=use_graph, per_group=per_group)
            _events(torch, stream, fn, W)
            modes[(name, form)] = _events(torch, stream, fn, reps)
            if name == "spec":
                stream.synchronize()
                e = _uneven_errors(X.double().cpu().numpy(), ref["f64" if dt == cj.F64 else "f32"], n, off)
                errs = e if errs is None else np.maximum(errs, e)
        plan.destroy()
    # every dispatcher variant pinned in turn (its tiles come from the
    # dispatcher's own rule, not from the groups' autotuned tiles), as a graph
    variants_ms = {}
    plan = cj.GroupPlan(dt, n, t)
    plan.wait()
    for v in range(plan.use_dispatcher()):
        plan.use_dispatcher(v)
        fn = lambda: plan.launch(A, X, stream=stream, use_graph=True)
        _events(torch, stream, fn, W)
        d = plan.dispatcher()
        variants_ms[f"{v} (blocks/SM {d['blocks_per_sm']})"] = _events(torch, stream, fn, reps)
        stream.synchronize()
        e = _uneven_errors(X.double().cpu().numpy(), ref["f64" if dt == cj.F64 else "f32"], n, off)
        errs = np.maximum(errs, e)
    plan.destroy()
    del A, X
    kept = "dispatch" if disp.get("state") == "ready" else "per_group"
    spec_ms = min(modes[("spec", kept + "_graph")], modes[("spec", kept + ("_direct" if kept == "dispatch" else "_streams"))])
    def best(name):
        return min(v for (k, _), v in modes.items() if k == name)
    peak = measured_peak("bf16_tflops", 1800.0) if dtype == "bf16" else PEAK_TFLOPS[dtype]
    if dtype == "bf16":
        err = {"max_rel_frobenius_error_vs_oracle_n_ge_16": float(errs[n >= 16].max()),
               "max_rel_frobenius_error_vs_oracle_n_lt_16_fp32": float(errs[n < 16].max())}
    else:
        err = {"max_rel_frobenius_error_vs_oracle": float(errs.max())}
    return {"value": f / spec_ms / 1e6, "dtype": dtype, **err,
            "error_sample": "every instance, every launch form of the autotuned plan and every dispatcher variant",
            "launch_form_kept": kept, "dispatcher": disp, "dispatcher_variants_ms": variants_ms,
            "dispatch_gflops": f / min(modes[("spec", "dispatch_graph")], modes[("spec", "dispatch_direct")]) / 1e6,
            "per_group_gflops": f / min(modes[("spec", "per_group_graph")], modes[("spec", "per_group_streams")]) / 1e6,
            "generic": {"value": f / best("generic") / 1e6, "unit": "GFLOP/s", "ms": best("generic")},
            "default_tiles": {"value": f / best("default_tiles") / 1e6, "unit": "GFLOP/s",
                              "ms": best("default_tiles")},
            "autotuned_groups_changed": changed,
            "launch_ms": {f"{k}_{form}": v for (k, form), v in modes.items()},
            "hw_queues": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8"),
            "ms_per_launch": spec_ms, "speedup_vs_generic": best("generic") / spec_ms,
            "roofline": {"bound": "alu" if dtype != "bf16" else "tensor", "peak": peak, "unit": "TFLOP/s",
                         "frac": f / spec_ms / 1e9 / peak},
            "config": {"workload": "uneven batch: 10,000 update chains, N log-uniform in [2,64], "
                                   "T uniform in [16,128] (seed 0xC1A4), one grouped plan, autotuned tiles and "
                                   f"launch form, {dtype}",
                       "flops": f, "groups": int(len(np.unique(n)))}}


def pch_workload(args):
    """JIT compile latency with and without NVRTC's automatic precompiled
    headers (-pch), over the FP64 sweep's nine instantiations (default
    tiles), compiled from the library's embedded kernel sources with the
    library's own options.  Needs no GPU.  Reports p50/p95 per setting and
    whether files appeared under the temporary directory (the library's
    requirement is that run-time compilation touches no file)."""
    import glob
    import tempfile
    from cuda.bindings import nvrtc
    from paper_1904_08555_b300 import build, cj
    kdir = build.KDIR
    hdr_names = ["geometry.h", "update_chain.cuh", "ltimes.cuh"]
    hdrs = [open(os.path.join(kdir, h)).read().encode() for h in hdr_names]
    exprs = []
    for n in SWEEP_N:
        tiles = cj.candidates(cj.K_UPDATE_CHAIN, dtype=cj.F64, n=n, layout_a=0)
        d = next(t for t in tiles if cj.featurize(cj.K_UPDATE_CHAIN, cj.F64, batch=synth.chain_batch(n), steps=T_STEPS,
                                                   tile=t, n=n, layout_a=0)[31] == 1.0)
        exprs.append(f"cj::update_chain<double, {n}, 0, {d[0]}, {d[1]}>")
    base = [b"-arch=sm_103a", b"-std=c++17", b"-lineinfo", b"--no-cache"]
    tmp = tempfile.gettempdir()

    def compile_all(opts):
        ms = []
        for e in exprs:
            t0 = time.perf_counter()
            _, prog = nvrtc.nvrtcCreateProgram(b'#include "update_chain.cuh"\n', b"cj_instantiation.cu", 3, hdrs,
                                               [h.encode() for h in hdr_names])
            nvrtc.nvrtcAddNameExpression(prog, e.encode())
            (rc,) = nvrtc.nvrtcCompileProgram(prog, len(opts), opts)
            if rc == nvrtc.nvrtcResult.NVRTC_SUCCESS:
                _, size = nvrtc.nvrtcGetCUBINSize(prog)
                buf = b" " * size
                nvrtc.nvrtcGetCUBIN(prog, buf)
            nvrtc.nvrtcDestroyProgram(prog)
            ms.append((time.perf_counter() - t0) * 1e3)
            assert rc == nvrtc.nvrtcResult.NVRTC_SUCCESS, e
        return ms

    compile_all(base)                       # warm NVRTC (first use)
    before = set(glob.glob(os.path.join(tmp, "*nvrtc*")))
    res = {}
    for name, opts in (("no_pch", base), ("auto_pch", base + [b"-pch"])):
        ms = []
        for _ in range(args.steps):
            ms += compile_all(opts)
        res[name] = {"p50_ms": float(np.percentile(ms, 50)), "p95_ms": float(np.percentile(ms, 95)),
                     "mean_ms": float(np.mean(ms)), "compiles": len(ms)}
    after = set(glob.glob(os.path.join(tmp, "*nvrtc*")))
    out = {"metric": "JIT compile ms (NVRTC to sm_103a CUBIN), with and without automatic PCH",
           "value": res["no_pch"]["p50_ms"], "unit": "ms", "higher_is_better": False, "n_gpus": 0,
           "steps": args.steps, "warmup": 1, "dtype": "f64", "data": "synthetic", "result": res,
           "files_created_under_tmp_by_pch": sorted(after - before),
           "config": {"workload": "the FP64 sweep's 9 instantiations (default tiles), compiled from the embedded "
                                  "sources; no_pch is the library's configuration"}}
    print(json.dumps(out), flush=True)


def secondary(args):
    if args.workload == "pch":
        return pch_workload(args)
    import torch
    from paper_1904_08555_b300 import cj
    torch.cuda.set_device(0)
    if args.workload == "costmodel":
        cj.init(sync=False, compile_threads=os.cpu_count() or 4)
    else:
        cj.init(sync=True, compile_threads=4)
    stream = torch.cuda.Stream()
    sampler = ClockSampler(0)
    sampler.start()
    out = {"metric": METRIC, "unit": "GFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    K, W = args.steps, args.warmup
    if args.workload == "small":
        out.update(run_config1(torch, cj, stream, W))
    elif args.workload == "sweep32":
        dt, tdt = cj.F32, torch.float32
        rows, tot_f, tot_spec, tot_gen = [], 0.0, 0.0, 0.0
        for n in SWEEP_N:
            b = synth.chain_batch(n)
            A = synth.uniform_torch(synth.SEED_CHAIN_SWEEP, synth.STREAM_A, b * n * n, "cuda").view(b, n, n).to(tdt)
            X = torch.empty_like(A)
            f = chain_flops(b, n, T_STEPS)
            row = {"N": n, "batch": b}
            variants = [("jit", cj.FLAG_NO_AOT, (0, 0, 0, 0)), ("generic", cj.FLAG_GENERIC, (0, 0, 0, 0))]
            if n in AOT_N:
                variants.append(("aot", 0, (0, 0, 0, 0)))
            if n % 4 == 0 and n >= 8:
                variants.append(("regblock", 0, (5, max(1, 256 // ((n // 4) ** 2)), 0, 0)))
            if n <= 32:
                variants.append(("tworow", 0, (6, max(1, 256 // ((n + 1) // 2)), 0, 0)))
                variants.append(("tworow128", 0, (6, max(1, 128 // ((n + 1) // 2)), 0, 0)))
            for name, fl, tile in variants:
                h = cj.specialize(cj.K_UPDATE_CHAIN, dt, n=n, flags=fl, tile=tile)
                fn = lambda h=h: cj.launch_update_chain(h, A, X, T_STEPS, stream=stream)
                _events(torch, stream, fn, W)
                ms = _events(torch, stream, fn, K)
                row[name + "_us"] = ms * 1e3
                row[name + "_gflops"] = f / ms / 1e6
                row[name + "_regs"] = h.regs()[0]
            row["speedup_vs_generic"] = row["generic_us"] / row["jit_us"]
            rows.append(row)
            tot_f += f
            tot_spec += row["jit_us"]
            tot_gen += row["generic_us"]
            del A, X
        peak = PEAK_TFLOPS["f32"]
        out.update({"value": tot_f / tot_spec / 1e3, "dtype": "f32",
                    "generic": {"value": tot_f / tot_gen / 1e3, "unit": "GFLOP/s"},
                    "speedup_vs_generic": tot_gen / tot_spec, "per_n": rows,
                    "roofline": {"bound": "alu", "peak": peak, "unit": "TFLOP/s",
                                 "frac": tot_f / tot_spec / 1e6 / peak},
                    "config": {"workload": "update chain FP32 size sweep, same sizes as the FP64 sweep"}})
    elif args.workload == "ltimes":
        out.update(run_config3(torch, cj, stream, args.dtype, args.ltimes_z, K, alt_tiles=args.lt_alt_tiles))
    elif args.workload == "uneven":
        ref = uneven_reference((args.dtype,))
        out.update(run_config4(torch, cj, stream, args.dtype, K, W, ref))
    elif args.workload == "kernel":
        # one kernel on a small case (inputs above L2), for profiler captures
        dt = {"f64": cj.F64, "f32": cj.F32, "bf16": cj.BF16}[args.dtype]
        tdt = torch.float64 if dt == cj.F64 else torch.float32     # bf16 chains keep fp32 state
        generic = args.kernel.endswith("-generic")
        fl = cj.FLAG_GENERIC if generic else cj.FLAG_NO_AOT
        if args.kernel.startswith("eigen"):
            n, b = args.n, args.batch
            M0 = synth.uniform_torch(synth.SEED_CHAIN_SWEEP, synth.STREAM_A, b * n * n, "cuda").to(tdt)
            Mo = torch.empty_like(M0)
            h = cj.specialize(cj.K_EIGEN_RECURRENCE, dt, n=n, flags=cj.FLAG_GENERIC if generic else 0,
                              tile=tuple(args.tile) if args.tile else (0, 0, 0, 0))
            fn = lambda: cj.launch_eigen(h, M0, Mo, T_STEPS, 5e-5, batch=b, stream=stream)
            f = float(b) * T_STEPS * (2.0 * n ** 3 + 3.0 * n ** 2)
            desc = f"Eigen recurrence N={n} batch={b} repeats={T_STEPS} {args.dtype} {'generic' if generic else 'jit'}"
        elif args.kernel.startswith("chain"):
            n, b = args.n, args.batch
            A = synth.uniform_torch(synth.SEED_CHAIN_SWEEP, synth.STREAM_A, b * n * n, "cuda").view(b, n, n).to(tdt)
            X = torch.empty_like(A)
            h = cj.specialize(cj.K_UPDATE_CHAIN, dt, n=n, flags=fl, tile=tuple(args.tile) if args.tile else (0, 0, 0, 0))
            fn = lambda: cj.launch_update_chain(h, A, X, T_STEPS, stream=stream)
            f = chain_flops(b, n, T_STEPS)
            desc = f"update chain N={n} batch={b} T={T_STEPS} {args.dtype} {'generic' if generic else 'jit'}"
        else:
            M, D, G, Z = 36, 96, 32, args.ltimes_z
            L, _ = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, 1, 1)
            Lt = torch.from_numpy(L).to("cuda", tdt)
            x = synth.uniform_torch(synth.SEED_LTIMES, synth.STREAM_A, D * G * Z, "cuda").view(D, G, Z)
            xin = x.permute(*synth.LAYOUT_PERMS[args.layout_in]).contiguous().view(-1).to(tdt)
            del x
            o = torch.empty(M * G * Z, device="cuda", dtype=tdt)
            h = cj.specialize(cj.K_LTIMES, dt, layout_a=args.layout_in, layout_b=args.layout_out, m=M, d=D, flags=fl,
                              tile=tuple(args.tile) if args.tile else (0, 0, 0, 0))
            fn = lambda: cj.launch_ltimes(h, Lt, xin, o, G, Z, stream=stream)
            f = 2.0 * M * D * G * Z
            desc = (f"LTimes M=36 D=96 G=32 Z={Z} in {synth.LAYOUT_NAMES[args.layout_in]} out order "
                    f"{args.layout_out} {args.dtype} {'generic' if generic else 'jit'}")
        _events(torch, stream, fn, W)
        ms = _events(torch, stream, fn, K)
        out.update({"value": f / ms / 1e6, "dtype": args.dtype, "ms_per_launch": ms, "regs": h.regs()[0],
                    "config": {"workload": desc}})
    elif args.workload == "mass":
        out.update(run_mass_workload(torch, cj, stream, args.dtype if args.dtype != "bf16" else "f64", K, W))
    elif args.workload == "eigen":
        # the paper's literal Eigen recurrence (Listing eigen1), batched: random
        # starts in [-1, 1), c = 5e-5, 64 repeats, batch = 2^24 / N^2 per size
        dt = cj.F64 if args.dtype == "f64" else cj.F32
        tdt = torch.float64 if dt == cj.F64 else torch.float32
        rep, c = 64, 5e-5
        rows, tot_f, tot_s, tot_g = [], 0.0, 0.0, 0.0
        for n in range(1, 17):
            b = (1 << 24) // (n * n)
            M0 = synth.uniform_torch(synth.SEED_CHAIN_SWEEP, synth.STREAM_A, b * n * n, "cuda").to(tdt)
            M = torch.empty_like(M0)
            f = float(b) * rep * (2.0 * n ** 3 + 3.0 * n ** 2)
            row = {"N": n, "batch": b}
            for name, fl in (("spec", 0), ("generic", cj.FLAG_GENERIC)):
                h = cj.specialize(cj.K_EIGEN_RECURRENCE, dt, n=n, flags=fl)
                fn = lambda h=h: cj.launch_eigen(h, M0, M, rep, c, batch=b, stream=stream)
                _events(torch, stream, fn, W)
                ms = _events(torch, stream, fn, K)
                row.update({name + "_ms": ms, name + "_gflops": f / ms / 1e6, name + "_regs": h.regs()[0]})
            row["speedup_vs_generic"] = row["generic_ms"] / row["spec_ms"]
            rows.append(row)
            tot_f += f
            tot_s += row["spec_ms"]
            tot_g += row["generic_ms"]
            del M0, M
        peak = PEAK_TFLOPS[args.dtype]
        out.update({"value": tot_f / tot_s / 1e6, "dtype": args.dtype,
                    "generic": {"value": tot_f / tot_g / 1e6, "unit": "GFLOP/s"},
                    "speedup_vs_generic": tot_g / tot_s,
                    "min_speedup_vs_generic": min(r["speedup_vs_generic"] for r in rows),
                    "per_n": rows,
                    "roofline": {"bound": "alu", "peak": peak, "unit": "TFLOP/s",
                                 "frac": tot_f / tot_s / 1e9 / peak},
                    "config": {"workload": "Eigen literal recurrence M = Ones + 5e-5 (M + M M) (Listing eigen1), "
                                           f"N = 1..16, 64 repeats, batch 2^24/N^2, random starts, {args.dtype}",
                               "flops_per_instance_step": "2 N^3 + 3 N^2"}})
    elif args.workload == "costmodel":
        from paper_1904_08555_b300 import costmodel
        res = costmodel.run(n_heldout=args.heldout, train_steps=args.train_steps, log=lambda m: print(m, file=sys.stderr))
        rg = res["regret"]
        out.update({"metric": "cost-model regret t(chosen)/t(best exhaustive) - 1, geometric mean over held-out requests",
                    "value": rg["model"]["geomean"], "unit": "fraction", "higher_is_better": False,
                    "dtype": "f32 (network); f64/f32 kernels", "result": res,
                    "config": {"workload": f"{res['heldout_requests']} unseen specialization requests (seed 0xC1A5): "
                                           "chain/LTimes 50/50; chain N uniform over the sizes in [2,64] not trained "
                                           "on, f64/f32 (+bf16 at N >= 16); LTimes over the 18 order pairs not "
                                           "trained on, f64/f32; chain batch 2^22/N^2, T 64; LTimes M 36 D 96 G 32 "
                                           "Z 2^16"}})
    out["clocks"] = sampler.stop()
    st = cj.stats()
    out["jit_compile_ms_p50"] = st["compile_ms_p50"]
    out["jit_compile_ms_p95"] = st["compile_ms_p95"]
    print(json.dumps(out), flush=True)
    cj.shutdown()


if __name__ == "__main__":
    main()
