"""Benchmark: detector-sampling throughput of the GPU Pauli-frame sampler.

One step = one ``tmcs_sample`` call over the whole workload (every layer of
the compiled circuit for every shot: frame updates, noise streams,
measurement records, detector/observable parities and their HBM stores).
Default workload: distance-29 surface-code non-local CNOT, 29 rounds before
and after, p = 1e-3, p_ebit = 1e-2, 1e7 shots, seed 1 (synthetic circuit; the
paper's workloads are circuits fully defined by their parameters).

Prints ONE JSON line (rank 0). ``--impl reference`` times the CPU oracle
(the project's plain one-shot frame simulator) instead, on the host cores.

Under torchrun (N > 1) each rank samples its own disjoint range of 64-shot
chunks (weak scaling, no data-path collective; outputs are keyed by global
chunk index, so the union equals one big run).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "detector-shot bits/sec and shots/sec (d=29 surface CNOT, BB teleport) vs roofline"
UNIT = "detector-shot bits/s"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_rate(circ, seed: int, budget_s: float, threads: int):
    """Oracle shots/s on a bounded sample (whole 64-shot chunks spread over
    the chunk range, one per thread per round)."""
    import oracle
    m = oracle.Marshalled(circ)
    chunks = threads
    t0 = time.perf_counter()
    oracle.sample(circ, 64 * chunks, seed, first_chunk=0, threads=threads, marshalled=m)
    dt = time.perf_counter() - t0
    shots = 64 * chunks
    rounds = max(0, int(budget_s / max(dt, 1e-9)) - 1)
    if rounds:
        t0 = time.perf_counter()
        oracle.sample(circ, 64 * chunks * rounds, seed, first_chunk=chunks, threads=threads, marshalled=m)
        dt += time.perf_counter() - t0
        shots += 64 * chunks * rounds
    return shots / dt, shots, dt


def reference_arm(args, workload, circ, rank, world):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    import oracle
    oracle.lib()
    per_step = []
    shots_done = 0
    for step in range(args.warmup + args.steps):
        chunks = threads
        t0 = time.perf_counter()
        oracle.sample(circ, 64 * chunks, workload.seed, first_chunk=step * chunks, threads=threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            per_step.append(dt)
            shots_done += 64 * chunks
    total = sum(per_step)
    shots_s = shots_done / total
    value = shots_s * circ.n_det
    sample_desc = (f"{args.steps} steps x {threads} chunks x 64 shots of {workload.name} "
                   f"(global chunks from 0), one-shot-at-a-time oracle, {threads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "shots_per_s": shots_s,
        "config": {"workload": workload.name, "shots_per_step": 64 * threads, "seed": workload.seed},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nl_sc29")
    ap.add_argument("--shots", type=int, default=0, help="override the workload's shot count")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=120, help="serve: number of requests")
    ap.add_argument("--batch-mix", default="config", choices=["config", "small"], help="batch64: job mix")
    ap.add_argument("--load", type=float, default=0.7, help="serve: offered load / solo capacity")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (64-job mix) and served (Poisson requests) measurements that the "
                         "default single-GPU run appends to its line")
    args = ap.parse_args()

    from paper_2504_05611_gb300 import circuits
    if args.workload == "batch64":
        batch_bench(args)
        return
    if args.workload == "serve":
        serve_bench(args)
        return
    if args.workload == "peaks":
        peaks_bench(args)
        return
    workload = circuits.WORKLOADS[args.workload]
    if args.shots:
        workload = circuits.Workload(workload.name, workload.code, workload.op, workload.rounds_before,
                                     workload.rounds_after, workload.p, workload.p_ebit, args.shots,
                                     workload.seed)
    circ = workload.circuit()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, workload, circ, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    from paper_2504_05611_gb300 import build as lib_build
    lib_build.build()
    from paper_2504_05611_gb300 import tmcs

    shots = workload.shots
    cols = (shots + 63) // 64
    from paper_2504_05611_gb300.shard import max_over_ranks, rank_chunk_range
    first_chunk, _ = rank_chunk_range(rank, world, shots)  # weak scaling: disjoint global chunk ranges
    sampler = tmcs.Sampler(circ)
    info = sampler.info
    stats = sampler.stats()
    det = torch.empty((info["n_det"], cols), dtype=torch.int64, device=dev)
    obs = torch.empty((max(info["n_obs"], 1), cols), dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def step():
        tmcs.tmcs_sample_range(sampler.handle, first_chunk, shots, workload.seed, det, obs, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    # device-timed steps: one kernel launch per step, CUDA events on its stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    ms_local = total_ms / args.steps
    ms_step = max_over_ranks(ms_local, dev)
    total_shots = shots * world
    shots_s = total_shots / (ms_step / 1e3)
    value = shots_s * info["n_det"]

    out_bytes = (info["n_det"] + info["n_obs"]) * cols * 8
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    peak, peak_kind = measured_peaks()
    achieved = out_bytes / avg_launch_s / 1e9
    # the kernel the autotuner picked for this workload, and its DRAM traffic
    # per launch from an ncu capture of the same kernel build, if committed
    shape = tmcs.tmcs_launch_shape(sampler.handle)
    kernel = shape["kernel"] or "autotuner not run (call below its size threshold)"
    traffic = None
    sha = _kernel_sha(kernel)
    for fn in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        if not fn.endswith("_traffic.json"):
            continue
        with open(os.path.join(ROOT, "profiles", fn)) as f:
            p = json.load(f)
        if p.get("workload") == workload.name and p.get("kernel") == kernel and p.get("kernel_sha") == sha:
            traffic = p.get("dram_bytes_per_launch")

    # end-to-end through the public API with host buffers: per step, sample
    # the workload in slices and stream each slice's detector/observable words
    # to pinned host memory (double-buffered); inputs are the compiled circuit
    # (resident) and the seed.
    e2e = None
    if args.e2e_steps > 0:
        slice_cols = max(1, min(cols, (1 << 28) // max(8 * (info["n_det"] + info["n_obs"]), 1)))
        nslices = (cols + slice_cols - 1) // slice_cols
        dbuf = [torch.empty((info["n_det"], slice_cols), dtype=torch.int64, device=dev) for _ in range(2)]
        obuf = [torch.empty((max(info["n_obs"], 1), slice_cols), dtype=torch.int64, device=dev) for _ in range(2)]
        hd = [torch.empty((info["n_det"], slice_cols), dtype=torch.int64, pin_memory=True) for _ in range(2)]
        ho = [torch.empty((max(info["n_obs"], 1), slice_cols), dtype=torch.int64, pin_memory=True) for _ in range(2)]
        copy_stream = torch.cuda.Stream(device=dev)
        done = [torch.cuda.Event() for _ in range(2)]
        sampled = [torch.cuda.Event() for _ in range(2)]

        def e2e_step():
            d2h = 0
            for s in range(nslices):
                b = s % 2
                c0 = s * slice_cols
                n = min(slice_cols, cols - c0)
                nshots = min(64 * n, shots - 64 * c0)
                stream.wait_event(done[b])
                tmcs.tmcs_sample_range(sampler.handle, first_chunk + c0, nshots, workload.seed,
                                       dbuf[b], obuf[b], stream)
                sampled[b].record(stream)
                copy_stream.wait_event(sampled[b])
                with torch.cuda.stream(copy_stream):
                    # the call writes rows of n words (row stride n), so a
                    # short last slice is the first n_det * n words
                    nd, no = info["n_det"] * n, max(info["n_obs"], 1) * n
                    hd[b].view(-1)[:nd].copy_(dbuf[b].view(-1)[:nd], non_blocking=True)
                    ho[b].view(-1)[:no].copy_(obuf[b].view(-1)[:no], non_blocking=True)
                done[b].record(copy_stream)
                d2h += (info["n_det"] + info["n_obs"]) * n * 8
            return d2h

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        w0 = time.perf_counter()
        d2h_bytes = 0
        for _ in range(args.e2e_steps):
            d2h_bytes = e2e_step()
        torch.cuda.synchronize()
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - w0) / args.e2e_steps, dev)
        # the device-to-host copy rate alone (one full slice, best of 3), the
        # ceiling of this end-to-end path
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        link_ms = []
        for _ in range(3):
            c0.record(copy_stream)
            with torch.cuda.stream(copy_stream):
                hd[0].copy_(dbuf[0], non_blocking=True)
            c1.record(copy_stream)
            c1.synchronize()
            link_ms.append(c0.elapsed_time(c1))
        e2e = {"value": total_shots * info["n_det"] / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": d2h_bytes, "shots_per_s": total_shots / e2e_s,
               "launches_per_step": nslices,
               "d2h_copy_gbs": hd[0].numel() * 8 / (min(link_ms) * 1e-3) / 1e9}

    # batched and served throughput on the same GPU, stated against the
    # single-circuit kernel (1 GPU only; the outputs of the headline run are
    # released first)
    extras = {}
    if world == 1 and not args.no_extras and not args.shots:
        del det, obs
        if args.e2e_steps > 0:
            del dbuf, obuf, hd, ho
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        b = batch_measure(args, 3)
        b["vs_single_circuit_shots_per_s"] = b["shots_per_s"] / shots_s
        extras["batch"] = b
        sv = serve_measure(args, args.requests, args.load)
        sv["vs_single_circuit_shots_per_s"] = sv["shots_per_s"] / shots_s
        extras["serve"] = sv

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, n_shots, secs = oracle_rate(circ, workload.seed, args.cpu_budget, threads)
        rate1, n1, secs1 = oracle_rate(circ, workload.seed, args.cpu_budget / 4, 1)
        cpu = {"value": rate * info["n_det"], "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{n_shots} shots ({n_shots // 64} chunks) of {workload.name} in {secs:.1f} s, "
                         f"one-shot-at-a-time oracle on {threads} threads; single thread: {n1} shots "
                         f"in {secs1:.1f} s",
               "shots_per_s": rate, "shots_per_s_1_thread": rate1}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "shots_per_s": shots_s,
            "config": {"workload": workload.name, "code": workload.code, "op": workload.op,
                       "rounds": [workload.rounds_before, workload.rounds_after], "p": workload.p,
                       "p_ebit": workload.p_ebit, "shots_per_gpu": shots, "seed": workload.seed,
                       "detectors": info["n_det"], "observables": info["n_obs"],
                       "slots": stats["n_slots"], "layers": stats["n_layers"],
                       "l2": f"output {out_bytes / 1e9:.1f} GB per step >> 129 MB L2 (no flush needed); "
                             f"compiled program {info['device_bytes'] / 1e6:.1f} MB stays resident",
                       "parallelism": f"chunk-range shards x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                         else "fallback 6.8 TB/s",
                         "algorithmic_bytes_per_launch": out_bytes, "avg_launch_ms": avg_launch_s * 1e3,
                         "kernel": kernel},
            "clocks": clk,
            "gpu_launches": args.steps,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    sampler.close()
    if world > 1:
        dist.destroy_process_group()


def batch_measure(args, steps):
    """Batched launch over the seeded 64-job mix (uneven circuits and shot
    counts) against the same jobs sampled one call each on the same stream;
    returns the batched, graph-replay and solo times and throughput."""
    import torch
    from paper_2504_05611_gb300 import circuits, tmcs
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.batch_mix == "small":
        # many small jobs (SC d = 3..9, 1e4..1e5 shots): solo launches underfill the GPU
        rng = __import__("numpy").random.default_rng(3)
        jobs = []
        for j in range(64):
            d = int(rng.choice([3, 5, 7, 9]))
            p = float(rng.choice([1e-4, 3e-4, 1e-3]))
            jobs.append(circuits.Workload(f"small{j}", f"sc{d}", ("nl", "teleport")[j % 2], d, d, p, 10 * p,
                                          int(round(10 ** rng.uniform(4, 5))), seed=j + 1))
    else:
        jobs = circuits.batch_mix(64, seed=1)
    cache = {}
    samplers, outs, total_det_bits, total_shots = [], [], 0, 0
    for w in jobs:
        key = (w.code, w.op, w.rounds_before, w.p)
        if key not in cache:
            cache[key] = tmcs.Sampler(w.circuit())
        s = cache[key]
        samplers.append(s)
        cols = (w.shots + 63) // 64
        outs.append((torch.empty((s.info["n_det"], cols), dtype=torch.int64, device=dev),
                     torch.empty((max(s.info["n_obs"], 1), cols), dtype=torch.int64, device=dev)))
        total_det_bits += s.info["n_det"] * w.shots
        total_shots += w.shots
    stream = torch.cuda.Stream(device=dev)
    jl = [(s.handle, w.shots, w.seed, d, o if s.info["n_obs"] else None)
          for s, w, (d, o) in zip(samplers, jobs, outs)]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    n_large = sum(1 for s, w in zip(samplers, jobs)
                  if (w.shots + 63) // 64 >= 16 * sms and tmcs.tmcs_circuit_stats(s.handle)["sig_ok"])

    def timed(fn, steps):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    def batched():
        tmcs.tmcs_batch_sample(jl, stream)

    def solo():
        for (h, n, seed, d, o) in jl:
            tmcs.tmcs_sample(h, n, seed, d, o, stream)

    for _ in range(max(1, args.warmup)):
        batched()
        solo()
    torch.cuda.synchronize()
    # a CUDA graph of the batched launch
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            batched()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    ms_batch = timed(batched, steps)

    def replay():
        with torch.cuda.stream(stream):
            g.replay()

    ms_graph = timed(replay, steps)
    clk = clocks.stop()
    ms_solo = timed(solo, max(1, steps // 2))
    value = total_det_bits / (min(ms_batch, ms_graph) / 1e3)
    del g
    for s in cache.values():
        s.close()
    return {
        "value": value, "shots_per_s": total_shots / (min(ms_batch, ms_graph) / 1e3), "total_shots": total_shots,
        "jobs": len(jobs), "distinct_circuits": len(cache), "batched_ms": ms_batch, "graph_replay_ms": ms_graph,
        "solo_calls_ms": ms_solo, "batched_vs_solo": ms_solo / min(ms_batch, ms_graph), "clocks": clk,
        "gpu_launches": n_large + (1 if n_large < len(jobs) else 0), "n_large": n_large,
        "mix": "circuits.batch_mix(64, seed=1)" if args.batch_mix != "small" else
               "64 SC d=3..9 NL/teleport jobs, 1e4..1e5 shots (seed 3)",
    }


def batch_bench(args):
    """--workload batch64: the batched measurement as its own JSON line."""
    import torch
    from paper_2504_05611_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)
    r = batch_measure(args, args.steps)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": min(r["batched_ms"], r["graph_replay_ms"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "shots_per_s": r["shots_per_s"],
        "config": {"workload": "batch64", "jobs": r["jobs"], "distinct_circuits": r["distinct_circuits"],
                   "total_shots": r["total_shots"], "mix": r["mix"]},
        "batched_ms": r["batched_ms"], "graph_replay_ms": r["graph_replay_ms"], "solo_calls_ms": r["solo_calls_ms"],
        "batched_vs_solo": r["batched_vs_solo"], "clocks": r["clocks"],
        # jobs of at least 16 chunks per SM run as their own tuned launch;
        # the others share one persistent launch per size class (1 or 2)
        "gpu_launches": r["gpu_launches"],
        "gpu_launches_note": f"{r['n_large']} GPU-filling jobs as single launches + the shared launches "
                             "(1 per size class)",
    }
    print(json.dumps(line), flush=True)


def serve_requests(n, seed):
    """Seeded request stream of the batched family: SC d = 3..29 (odd) and
    BB[[144,12,12]], NL or teleport, p in {1e-4, 3e-4, 1e-3} with p_ebit =
    10 p, shots log-uniform in [1e4, 1e7]."""
    from paper_2504_05611_gb300 import circuits
    return circuits.batch_mix(n, seed=seed)


def serve_measure(args, n_requests, load):
    """Poisson arrivals into the continuous-batching server at a fixed
    fraction of the measured solo capacity; returns throughput and latency."""
    import threading
    import numpy as np
    import torch
    from paper_2504_05611_gb300 import tmcs
    dev = torch.device("cuda", torch.cuda.current_device())
    reqs = serve_requests(n_requests, seed=7)
    cache, handles = {}, []
    for w in reqs:
        key = (w.code, w.op, w.rounds_before, w.p)
        if key not in cache:
            cache[key] = tmcs.Sampler(w.circuit())
        handles.append(cache[key])
    det_bits = sum(h.info["n_det"] * w.shots for h, w in zip(handles, reqs))
    shots_total = sum(w.shots for w in reqs)
    # solo capacity: every request as one tmcs_sample call, back to back
    words = max((h.info["n_det"] + h.info["n_obs"]) * ((w.shots + 63) // 64) for h, w in zip(handles, reqs))
    scratch = torch.empty(words, dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def solo_pass():
        for h, w in zip(handles, reqs):
            cols = (w.shots + 63) // 64
            d = scratch[: h.info["n_det"] * cols]
            o = scratch[h.info["n_det"] * cols: (h.info["n_det"] + h.info["n_obs"]) * cols]
            tmcs.tmcs_sample(h.handle, w.shots, w.seed, d, o if h.info["n_obs"] else None, stream)

    solo_pass()                      # uploads and autotunes every circuit
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solo_pass()
    torch.cuda.synchronize()
    solo_s = time.perf_counter() - t0
    del scratch
    torch.cuda.empty_cache()
    mean_gap = solo_s / len(reqs) / load
    rng = np.random.default_rng(11)
    gaps = rng.exponential(mean_gap, size=len(reqs))
    srv = tmcs.Server(n_streams=4)
    ids = [None] * len(reqs)
    submitted = threading.Event()

    def client():
        t = time.perf_counter()
        for i, (h, w) in enumerate(zip(handles, reqs)):
            t += gaps[i]
            delay = t - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids[i] = srv.submit(h, w.shots, w.seed)
        submitted.set()

    clocks = ClockSampler(dev.index)
    clocks.start()
    start = time.perf_counter()
    th = threading.Thread(target=client)
    th.start()
    done = 0
    while done < len(reqs):
        while ids[done] is None:
            time.sleep(0.0005)
        srv.release(ids[done])
        done += 1
    th.join()
    makespan = time.perf_counter() - start
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    for h in cache.values():
        h.close()
    return {"value": det_bits / makespan, "shots_per_s": shots_total / makespan, "makespan_s": makespan,
            "requests": len(reqs), "offered_load": load, "latency_p50_s": st["latency_p50_s"],
            "latency_p99_s": st["latency_p99_s"], "latency_mean_s": st["latency_mean_s"],
            "solo_capacity_s": solo_s, "solo_shots_per_s": shots_total / solo_s,
            "served_vs_solo_throughput": solo_s / makespan, "completed": st["completed"], "failed": st["failed"],
            "clocks": clk}


def serve_bench(args):
    """--workload serve: the serving measurement as its own JSON line."""
    import torch
    from paper_2504_05611_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)
    r = serve_measure(args, args.requests, args.load)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": r["makespan_s"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic", "shots_per_s": r["shots_per_s"],
        "config": {"workload": "serve", "requests": r["requests"], "offered_load": r["offered_load"],
                   "arrivals": "Poisson", "family": "circuits.batch_mix(n, seed=7)", "n_streams": 4},
        "latency_p50_s": r["latency_p50_s"], "latency_p99_s": r["latency_p99_s"],
        "latency_mean_s": r["latency_mean_s"], "solo_capacity_s": r["solo_capacity_s"],
        "served_vs_solo_throughput": r["served_vs_solo_throughput"], "completed": r["completed"],
        "failed": r["failed"], "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)


def peaks_bench(args):
    """Measured non-HBM ceilings of this GPU (shared-memory loads, shared
    atomics, LOP3), the denominators of the kernels' shared-memory and
    integer-pipe fractions; one JSON line."""
    import torch
    from paper_2504_05611_gb300 import build as lib_build
    lib_build.build()
    from paper_2504_05611_gb300 import tmcs
    torch.cuda.set_device(0)
    runs = [tmcs.tmcs_measure_peaks() for _ in range(3)]
    best = {k: max(r[k] for r in runs) for k in runs[0]}
    print(json.dumps({"metric": "device peaks (microbenchmarks)", "smem_load_TBps": best["smem_load_bytes_per_s"] / 1e12,
                      "smem_wavefronts_per_s": best["smem_load_wavefronts_per_s"],
                      "smem_atomic_lanes_per_s": best["smem_atomic_lanes_per_s"],
                      "lop3_lanes_per_s": best["lop3_lanes_per_s"], "lop3_warp_inst_per_s": best["lop3_warp_inst_per_s"],
                      "sms": best["sms"], "sm_clock_mhz_attribute": best["sm_clock_mhz"], "runs": 3}), flush=True)


def _strip_comments(src: str) -> str:
    """C/C++/CUDA source without // and /* */ comments (string and character
    literals kept) and without whitespace."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return re.sub(r"\s+", "", "".join(out))


def _kernel_sha(kernel=None):
    """Hash of the sources that define a kernel (its device code, the device
    primitives it uses and the program layout it reads), comments and
    whitespace excluded: a committed traffic figure stays attached to the
    kernel build it was measured on."""
    import hashlib
    h = hashlib.sha256()
    if kernel and kernel.startswith("flow_kernel"):
        files = ("tmcs_flow.cu", "tmcs_device.cuh", "tmcs_internal.h", "tmcs_signature.cpp")
    else:
        files = ("tmcs_sample.cu", "tmcs_device.cuh", "tmcs_internal.h", "tmcs_host.cpp", "tmcs_signature.cpp")
    for f in files:
        with open(os.path.join(ROOT, "paper_2504_05611_gb300", "csrc", f)) as fh:
            h.update(_strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
