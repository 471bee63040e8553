#!/usr/bin/env python
"""kMC events/s of the sequential-update parallel kMC hot path on GB300.

Default workload (one bench step = the whole configuration):
  1024x1024 periodic 2D Ising, J=1, h=0, L_d=32 (32x32 domains, 4 colours),
  T in {1.5, 2.269, 3.0}, random and all-up starts, k in {1, 4, 16} steps per
  domain visit, 1e4 palindromic schedules per run, energy/magnetisation every
  10 schedules.  The three temperatures of one (k, start) run as one batch of
  three replicas, so a step is six runs = 18 lattice trajectories.

An event is one uniformised domain step (the unit k counts); real flips are
reported beside it.  `value` times the device work with inputs resident in
HBM (CUDA events on the launch stream, L2 flushed between steps); `e2e`
times the same work through the public API with host buffers: pinned host ->
device copy of the initial spins, the run, device -> host copy of the final
spins and observables.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload ising1024|ising8192|batched]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "kMC events/s on 1 GB300 (plain vs batched+grad), % of roofline, bit-exact"
UNIT = "events/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ising1024", choices=["ising1024", "ising8192", "batched"])
    ap.add_argument("--schedules", type=int, default=0, help="override schedules per run (0 = workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workloads: list of runs (L list, L_d, k, betas, hs, seeds, init, schedules, obs_every)
# ---------------------------------------------------------------------------
def workload_runs(name: str, rank: int, sched_override: int):
    from paper_1403_4674_gb300 import workloads as wl
    runs = []
    if name == "ising1024":
        Ts = [1.5, 2.269, 3.0]
        for k in (1, 4, 16):
            seeds = wl.replica_seeds(1024 * 1000 + 17 * k + 7919 * rank, 3)
            for init in (0, 1):
                runs.append(dict(L=[1024] * 3, Ld=32, k=k, beta=[1 / T for T in Ts], h=[0.0] * 3,
                                 seeds=seeds, init=init, schedules=10000, obs_every=10))
        desc = ("1024x1024 periodic Ising, J=1, h=0, L_d=32, T in {1.5,2.269,3.0} x {random, all-up} "
                "x k in {1,4,16}, 1e4 palindromic schedules per run, obs every 10")
    elif name == "ising8192":
        w = wl.lattice_8192(seed=8192 + rank)
        runs.append(dict(L=w.L, Ld=w.L_d, k=w.k, beta=w.beta, h=w.h, seeds=w.seeds, init=0,
                         schedules=w.schedules, obs_every=0))
        desc = "8192x8192 periodic Ising, T=2.269, h=0.01, L_d=64, k=8, 2000 palindromic schedules"
    else:
        w = wl.batched_replicas(512, master=512 + rank)
        runs.append(dict(L=w.L, Ld=w.L_d, k=w.k, beta=w.beta, h=w.h, seeds=w.seeds, init=0,
                         schedules=200, obs_every=10))
        desc = ("512 replicas, L=16*round(exp(U[ln32,ln512])/16), T~U[1.5,3.5], h~U[-0.1,0.1], "
                "L_d=8, k=8, 200 palindromic schedules, obs every 10")
    if sched_override > 0:
        for r in runs:
            r["schedules"] = sched_override
        desc += " (schedules overridden to %d)" % sched_override
    return runs, desc


def run_events(run) -> int:
    return int(sum(2 * (L // run["Ld"]) ** 2 * run["k"] for L in run["L"]) * run["schedules"])


def visit_bytes(Ld: int, k: int) -> int:
    """Algorithmic HBM bytes of one domain visit: the domain plus its halo read
    once ((L_d+2)^2 - 4 bytes of int8 state), write-back of at most k dirty 32-byte
    sectors and 4*L_d bytes of edge buffers."""
    return (Ld + 2) ** 2 - 4 + 32 * k + 4 * Ld


def run_algorithmic_bytes(run) -> int:
    visits = sum(2 * (L // run["Ld"]) ** 2 for L in run["L"]) * run["schedules"]
    return visits * visit_bytes(run["Ld"], run["k"])


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="kmc_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# oracle CPU baseline (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def oracle_sample(runs, budget_s: float):
    """Time the CPU oracle, single-threaded, on a bounded sample: for each
    distinct k, replica 0 of the random-start run for as many schedules as fit
    in budget_s / (#k values).  Returns (events/s, description, events, seconds)."""
    from oracle import oracle as orc
    by_k = {}
    for r in runs:
        if r["init"] == 0 and r["k"] not in by_k:
            by_k[r["k"]] = r
    per = budget_s / max(1, len(by_k))
    ev = 0
    secs = 0.0
    parts = []
    for k, r in sorted(by_k.items()):
        L, Ld = r["L"][0], r["Ld"]
        rep = orc.Replica(L=L, Ld=Ld, k=k, seed=r["seeds"][0], beta=r["beta"][0], h=r["h"][0])
        steps_per_sched = 2 * (L // Ld) ** 2 * k
        t0 = time.perf_counter()
        rep.run(1)
        one = time.perf_counter() - t0
        n = max(1, int(per / max(one, 1e-6)))
        t0 = time.perf_counter()
        rep.run(n)
        dt = time.perf_counter() - t0
        ev += n * steps_per_sched
        secs += dt
        parts.append("L=%d k=%d T=%.4g: %d schedules" % (L, k, 1 / r["beta"][0], n))
    return ev / secs, "; ".join(parts), ev, secs


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    runs, desc = workload_runs(args.workload, 0, args.schedules)
    budget = 8.0
    for _ in range(args.warmup):
        oracle_sample(runs, 1.0)
    vals, evs, secs = [], 0, 0.0
    for _ in range(args.steps):
        v, sample, e, s = oracle_sample(runs, budget)
        vals.append(v)
        evs += e
        secs += s
    value = evs / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": desc, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: " + sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # the CPU baseline runs before any CUDA work (rank 0, N = 1 only)
    runs, desc = workload_runs(args.workload, rank, args.schedules)
    cpu = None
    if world == 1 and not args.no_cpu:
        v, sample, e, s = oracle_sample(runs, 12.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%s; %d events in %.1f s, single thread" % (sample, e, s)}

    import torch
    import paper_1403_4674_gb300 as kmc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()

    # one context and one stream per run, created outside the timed region.  The
    # runs of a step are independent trajectories, so they are launched
    # concurrently (longest first) and the step ends when all have finished.
    runs.sort(key=lambda r: -r["k"])
    for r in runs:
        r["stream"] = torch.cuda.Stream()
        with torch.cuda.stream(r["stream"]):
            r["lat"] = kmc.Lattice(r["L"], r["Ld"], r["k"], r["seeds"], init=r["init"])
            r["lat"].profile(True)
    ctxs = {id(r): r["lat"] for r in runs}

    def step():
        start = torch.cuda.Event()
        start.record(stream)
        done = []
        for r in runs:
            r["stream"].wait_event(start)
            with torch.cuda.stream(r["stream"]):
                lat = r["lat"]
                lat.reset(r["init"])
                lat.set_rates(r["beta"], r["h"])
                r["obs"] = lat.run(r["schedules"], obs_every=r["obs_every"])
                ev = torch.cuda.Event()
                ev.record(r["stream"])
                done.append(ev)
        for ev in done:
            stream.wait_event(ev)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for lat in ctxs.values():
        lat.profile_read()  # discard warm-up timings
    launches0 = sum(lat.kernel_launches() for lat in ctxs.values())

    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush between timed steps (outside the event pair)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = sum(lat.kernel_launches() for lat in ctxs.values()) - launches0

    for r in runs:
        with torch.cuda.stream(r["stream"]):
            r["lat"].sync()
    run_ms, run_n = 0.0, 0
    for lat in ctxs.values():
        ms, n = lat.profile_read()
        run_ms += ms
        run_n += n

    events_step = sum(run_events(r) for r in runs)
    bytes_step = sum(run_algorithmic_bytes(r) for r in runs)
    dev_s = sum(step_ms) / 1000.0
    if dist is not None:
        t = torch.tensor([dev_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_s = float(t.item())
    value = events_step * args.steps * world / dev_s

    # real flips of the last step (reported beside events)
    flips = 0
    for r in runs:
        with torch.cuda.stream(r["stream"]):
            flips += int(r["lat"].observables()["flips"].sum())

    # end-to-end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host_in = {}
        for r in runs:
            with torch.cuda.stream(r["stream"]):
                lat = r["lat"]
                lat.reset(r["init"])
                lat.sync()
                host_in[id(r)] = lat.spins.cpu().pin_memory()
        host_out = {id(r): torch.empty_like(host_in[id(r)]).pin_memory() for r in runs}
        h2d = sum(host_in[id(r)].numel() for r in runs)
        d2h = 0

        def e2e_step():
            """Host buffers in, public API, host buffers out; runs concurrent as above."""
            nonlocal d2h
            d2h = 0
            outs = []
            for r in runs:
                with torch.cuda.stream(r["stream"]):
                    lat = r["lat"]
                    lat.spins.copy_(host_in[id(r)], non_blocking=True)
                    lat.reset(kmc.KMC_INIT_KEEP)
                    lat.set_rates(r["beta"], r["h"])
                    obs = lat.run(r["schedules"], obs_every=r["obs_every"])
                    host_out[id(r)].copy_(lat.spins, non_blocking=True)
                    d2h += lat.spins.numel()
                    if obs is not None:
                        o = torch.empty(obs.shape, dtype=obs.dtype, pin_memory=True)
                        o.copy_(obs, non_blocking=True)
                        d2h += obs.numel() * 8
                        outs.append(o)
            torch.cuda.synchronize()
            return outs

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        e2e_s = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": events_step * args.steps * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    avg_run_s = (run_ms / 1000.0) / max(run_n, 1)
    # The run kernels of a step overlap in time (one stream per run), so the
    # device-level rate divides the algorithmic bytes of all of them by the
    # step time; the per-launch rate divides one launch's bytes by its own
    # event time.
    achieved = (bytes_step * args.steps) / dev_s / 1e9 if dev_s > 0 else 0.0
    per_launch = (bytes_step * args.steps) / (run_ms / 1000.0) / 1e9 if run_ms > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None,
                "kernel": "kmcdev::run_kernel", "peak_source": peak_src,
                "per_launch_achieved": per_launch,
                "run_kernel_ms_avg": 1000 * avg_run_s, "run_kernel_launches": run_n,
                "run_kernel_busy_over_step": (run_ms / 1000.0) / dev_s if dev_s > 0 else None}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": {"workload": desc, "events_per_step": events_step,
                           "real_flips_per_step": flips,
                           "real_flips_per_s": flips * world / (dev_s / args.steps),
                           "l2": "flushed between timed steps (512 MB write outside the event pair)",
                           "parallelism": ("replicas only" if world > 1 else "1 GPU") +
                                          ", %d independent runs per step on concurrent streams" % len(runs),
                           "launch": [list(lat.launch()) for lat in ctxs.values()],
                           "wall_s": wall},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    for lat in ctxs.values():
        lat.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
