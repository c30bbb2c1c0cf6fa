#!/usr/bin/env python
"""EMPC benchmark: rollout state-steps/s of full EMPC solves on one GB300.

A step is one EMPC solve: G generations of breed + knot expansion + rollout +
cost + elite selection over the whole population, starting cold (the same
work every step).  Default workload: the 24-DoF coupled chain (n=48, m=24,
T=100, 5 knots, P=4096, E=128, G=30), FP32.

  python bench.py [--gpus N --steps K --warmup W] [--workload c1|c2|c5]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas, one
problem per rank (weak scaling, no collective on the data path).
"""
import argparse
import datetime as dt
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

L2_FLUSH_BYTES = 256 << 20
METRIC = "EMPC rollout state-steps/s"
UNIT = "state-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload_desc(wl):
    return (f"{wl.name}: {wl.dof}-DoF chain (n={wl.n}, m={wl.m}), T={wl.T}, p={wl.p}, "
            f"P={wl.P}, E={wl.E}, G={wl.G}, sigma={wl.sigma}, dt={wl.dt}")


def alg_flops_per_candidate(wl):
    """Algorithmic FLOPs of one candidate's rollout and cost in one generation:
    per step 2n^2 (D x) + 6n (knot lerp 3n, increment n, stage cost 2n... see
    the design doc), plus 2pnm for the knot forces B U_j and 3mp for the input cost."""
    n, m, T, p = wl.n, wl.m, wl.T, wl.p
    return T * (2 * n * n + 6 * n) + 2 * p * n * m + 3 * m * p


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        idx = vis.split(",")[local_rank] if vis else str(local_rank)
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", idx, f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                ts = dt.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm = float(f[1].split()[0])
                smax = float(f[2].split()[0])
            except ValueError:
                continue
            rows.append((ts, sm, smax, f[5:9]))
        inside = [r for r in rows if t0 - 0.25 <= r[0] <= t1 + 0.25] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v == "Active"})
        sms = [r[1] for r in inside]
        return {"sm_mhz": float(np.median(sms)) if sms else None,
                "sm_max_mhz": max(r[2] for r in inside) if inside else None,
                "samples": len(inside), "reasons": reasons}


def traffic_record(kernel_file):
    """DRAM bytes per launch from a committed ncu summary, valid only while the
    kernel source is unchanged (its sha256 is stored beside the figure)."""
    path = os.path.join(ROOT, "profiles", "rollout_traffic.json")
    src = os.path.join(ROOT, "paper_2001_04931_gb300", "csrc", kernel_file)
    try:
        rec = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        return rec if rec.get("source_sha256") == sha else None
    except (OSError, ValueError):
        return None


def cpu_baseline(wl, seconds):
    """The oracle (FP64, as it stands) running Algorithm 1 on the full
    population on the host cores until `seconds` pass or G generations end."""
    import oracle as O
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    b = wl.bounds()
    M = O.Model(A, B, wl.Q(), wl.R(), b[:, 0], b[:, 1], wl.T, wl.p)
    ga = O.EMPC(M, wl.P, wl.E, seed=1, sigma=wl.sigma)
    x0, g = wl.start_goal()
    t0 = time.perf_counter()
    gens = 0
    while gens < wl.G and (gens == 0 or time.perf_counter() - t0 < seconds):
        ga.generation(x0, g)
        gens += 1
    el = time.perf_counter() - t0
    return {"value": wl.P * wl.T * gens / el, "unit": UNIT, "cores": O.num_threads(),
            "kind": "oracle",
            "sample": f"{gens} of {wl.G} generations of the full {wl.P}-candidate population "
                      f"({workload_desc(wl)}), FP64 C oracle, OpenMP over candidates",
            "seconds": el}


def run_reference(args, wl):
    """The oracle as the reference arm: each step is one generation of Algorithm
    1 on a sub-population sized so the whole run takes about two minutes."""
    import oracle as O
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    b = wl.bounds()
    M = O.Model(A, B, wl.Q(), wl.R(), b[:, 0], b[:, 1], wl.T, wl.p)
    x0, g = wl.start_goal()
    # calibrate the sample size on one small generation
    probe = O.EMPC(M, 64, min(wl.E, 8), seed=1, sigma=wl.sigma)
    t0 = time.perf_counter()
    probe.generation(x0, g)
    per_cand = (time.perf_counter() - t0) / 64
    budget = 120.0 / max(1, args.steps + args.warmup)
    S = int(max(64, min(wl.P, budget / max(per_cand, 1e-9))))
    E = max(1, min(wl.E, S // 16))
    ga = O.EMPC(M, S, E, seed=1, sigma=wl.sigma)
    for _ in range(args.warmup):
        ga.generation(x0, g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ga.generation(x0, g)
    el = time.perf_counter() - t0
    value = S * wl.T * args.steps / el
    sample = (f"one generation of Algorithm 1 per step on {S} of {wl.P} candidates "
              f"({workload_desc(wl)}), FP64 C oracle, OpenMP over candidates")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(wl), "sample_candidates": S},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, wl, rank, world, local_rank):
    import torch
    import paper_2001_04931_gb300 as E

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    wl = W.config(wl.name, seed=rank)  # one independent problem per rank
    A, B = E.discretize_zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    prob = E.Problem(A, B, wl.Q(), wl.R(), wl.bounds(), wl.T, wl.p, wl.P, seed=1 + rank,
                     elite=wl.E, sigma=wl.sigma)
    stream = torch.cuda.Stream()
    prob.set_stream(stream.cuda_stream)
    x0, g = wl.start_goal()
    x0d = torch.tensor(x0, dtype=torch.float32, device="cuda")
    gd = torch.tensor(g, dtype=torch.float32, device="cuda")
    kd = torch.empty(wl.m * wl.p, device="cuda")
    cd = torch.empty(1, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")

    def solve_step():
        prob.reset()
        prob.solve_device(x0d, gd, wl.G, kd, cd)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            solve_step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        sampler = ClockSampler(local_rank)
        time.sleep(0.5)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall0 = time.time()
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            solve_step()
            e1.record(stream)
        torch.cuda.synchronize()
        t_wall1 = time.time()
        if dist:
            dist.barrier()
        clocks = sampler.stop(t_wall0, t_wall1)
        total_ms = sum(a.elapsed_time(b) for a, b in ev)
        if dist:
            t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        ms_step = total_ms / args.steps
        units = wl.P * wl.T * wl.G
        value = units * world / (ms_step * 1e-3)

        # per-kernel durations, CUDA events around each launch on this stream
        roll_us, sel_us = prob.time_generation(20)

    # end to end through the public API with host buffers
    n_e2e = max(1, min(args.e2e_steps, args.steps))
    e2e_t = []
    for i in range(n_e2e + 3):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.reset()
        prob.solve(x0, g, wl.G)
        if i >= 3:
            e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_t))
    if dist:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    props = torch.cuda.get_device_properties(local_rank)
    sms = props.multi_processor_count
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak_derived = sms * 128 * 2 * sm_max * 1e6 / 1e12
    try:
        peak_measured = E.measure_fp32_peak()
    except E.EmpcError:
        peak_measured = None
    flops = alg_flops_per_candidate(wl) * wl.P
    achieved = flops / (roll_us * 1e-6) / 1e12
    tr = traffic_record("rollout.cu")
    info = prob.info()
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "ms_per_problem": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded mass-spring-damper chain, ZOH-discretized, x0/goal U[-1,1]",
        "config": {"workload": workload_desc(wl),
                   "l2": f"flushed before every timed step ({L2_FLUSH_BYTES >> 20} MB write)",
                   "tile": {"nx": info.tile_nx, "rows": info.tile_rows,
                            "cands": info.tile_cands, "groups": info.tile_groups,
                            "threads": info.threads_per_cta, "ctas": info.ctas},
                   "replicas": world},
        "roofline": {"bound": "alu", "kernel": "rollout_kernel (fused breed+rollout+cost)",
                     "achieved": achieved, "peak": peak_derived, "unit": "TFLOP/s",
                     "frac": achieved / peak_derived,
                     "peak_basis": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                     "measured_fp32_peak": peak_measured,
                     "frac_of_measured": (achieved / peak_measured) if peak_measured else None,
                     "flops_per_launch": flops, "launch_us": roll_us, "select_us": sel_us,
                     "traffic": tr["dram_bytes_per_launch"] if tr else None},
        "e2e": {"value": units / e2e_s, "unit": UNIT, "ms_per_problem": 1e3 * e2e_s,
                "h2d_bytes_per_step": 2 * 4 * wl.n,
                "d2h_bytes_per_step": 4 * (wl.m * wl.p + 2)},
        "gpu_launches": args.steps * wl.G * 2,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    wl = W.config(args.workload)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return
    run_gpu(args, wl, rank, world, local_rank)


if __name__ == "__main__":
    main()
