#!/usr/bin/env python
"""kMC events/s of the sequential-update parallel kMC hot path on GB300.

Default workload (one bench step = the whole configuration):
  1024x1024 periodic 2D Ising, J=1, h=0, L_d=32 (32x32 domains, 4 colours),
  T in {1.5, 2.269, 3.0}, random and all-up starts, k in {1, 4, 16} steps per
  domain visit, 1e4 palindromic schedules, energy/magnetisation every 10
  schedules.  All 18 trajectories (T x start x k) are replicas of one context
  with per-replica k and start, so a step is one run-kernel launch; its launch
  plan is measured and chosen before the timed region.

An event is one uniformised domain step (the unit k counts); real flips are
reported beside it.  `value` times the device work with inputs resident in
HBM (CUDA events on the launch stream, L2 flushed between steps); `e2e`
times the same work through the public API with host buffers: pinned host ->
device copy of the initial spins, the run, device -> host copy of the final
spins and observables.

`variants` adds, at N = 1, the batched configuration (512 uneven replicas,
domain side, k and plan autotuned per group, one CUDA graph per step), the
gradient configuration (256 x 256^2 with likelihood-ratio scores), one
8192^2 lattice (L_d = 64, k = 8), the paper's 1D experiment (the 8-spin
ring of Sec. 3.1 over its whole N_D x N_I grid, 768000 trajectories) and its
2D experiments (12^2 and 100^2 in stripes and blocks, Sec. 3.2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload ising1024|ising8192] [--no-variants]
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
L2_FLUSH_FLOATS = 512 * 1024 * 1024 // 4  # a 512 MB buffer written between timed steps (L2 is 129 MB)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ising1024", choices=["ising1024", "ising8192"])
    ap.add_argument("--schedules", type=int, default=0, help="override schedules per run (0 = workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the batched and gradient variants")
    ap.add_argument("--plan", default="", help="launch plan mode,size,warps (skips the plan tuning)")
    ap.add_argument("--batch-k", type=int, default=32, help="steps per visit of the batch with --plan (profiling)")
    ap.add_argument("--part-streams", type=int, default=1,
                    help="streams the 12^2 settings of the 2D experiments are dealt over (0 = one stream each)")
    ap.add_argument("--only", default="", choices=["", "batched", "grad", "lattice8192", "ring8", "partitions2d",
                                                    "pollcost", "chain"],
                    help="time one variant alone and print its JSON object (profiling runs; not the contract line)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def main_workload(name: str, rank: int, sched_override: int):
    """The timed workload of the JSON line (one context, one run-kernel launch per step)."""
    from paper_1403_4674_gb300 import workloads as wl
    if name == "ising1024":
        w = wl.ising1024_all(seed_master=1024 + 7919 * rank)
        desc = ("1024x1024 periodic Ising, J=1, h=0, L_d=32, T in {1.5,2.269,3.0} x {random, all-up} "
                "x k in {1,4,16} (18 replicas in one launch), 1e4 palindromic schedules, obs every 10")
    elif name == "ising8192":
        w = wl.lattice_8192(seed=8192 + rank)
        desc = "8192x8192 periodic Ising, T=2.269, h=0.01, L_d=64, k=8, 2000 palindromic schedules"
    else:
        raise ValueError(name)
    if sched_override > 0:
        w.schedules = sched_override
        desc += " (schedules overridden to %d)" % sched_override
    return w, desc


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: int, steps: int, world: int, max_seconds: float) -> float:
    """Units of every rank over the slowest rank's time (weak scaling: each
    rank runs its own replicas of the same workload)."""
    return units_per_rank_step * steps * world / max_seconds


def visit_bytes(Ld: int, k: int) -> int:
    """Algorithmic HBM bytes of one domain visit: the domain plus its halo read
    once ((L_d+2)^2 - 4 bytes of int8 state), write-back of at most k dirty 32-byte
    sectors and 4*L_d bytes of edge buffers."""
    return (Ld + 2) ** 2 - 4 + 32 * k + 4 * Ld


def schedule_bytes(L, Ld: int, ks) -> int:
    """Algorithmic bytes of one palindromic schedule (two visits per domain)."""
    return int(sum(2 * (x // Ld) ** 2 * visit_bytes(Ld, k) for x, k in zip(L, ks)))


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
def oracle_sample(w, budget_s: float):
    """Time the CPU oracle, single-threaded, on a bounded sample: for each
    distinct k and temperature, the first random-start replica of that pair
    for as many schedules as fit in budget_s / (#pairs).  Returns
    (events/s, description, events, seconds)."""
    from oracle import oracle as orc
    by_kT = {}
    for r in range(len(w.L)):
        key = (w.k_of(r), round(1 / w.beta[r], 4))
        if w.init_of(r) == 0 and key not in by_kT:
            by_kT[key] = r
    per = budget_s / max(1, len(by_kT))
    ev = 0
    secs = 0.0
    parts = []
    for (k, T), r in sorted(by_kT.items()):
        L, Ld = w.L[r], w.L_d
        rep = orc.Replica(L=L, Ld=Ld, k=k, seed=w.seeds[r], beta=w.beta[r], h=w.h[r])
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
        parts.append("L=%d k=%d T=%.4g: %d schedules" % (L, k, T, n))
    return ev / secs, "; ".join(parts), ev, secs


def _oracle_job(job):
    """One oracle replica for a bounded time (module level: runs in a spawned
    worker).  job = (L, L_d, k, seed, beta, h, scores, budget_s); returns
    (uniformised steps run, seconds)."""
    from oracle import oracle as orc
    L, Ld, k, seed, beta, h, scores, budget = job
    rep = orc.Replica(L=L, Ld=Ld, k=k, seed=seed, beta=beta, h=h)
    if scores:
        rep.enable_score()
    steps_per_sched = 2 * (L // Ld) ** 2 * k
    t0 = time.perf_counter()
    rep.run(1)
    one = time.perf_counter() - t0
    n = max(0, int((budget - one) / max(one, 1e-6)))
    if n > 0:
        rep.run(n)
    return (n + 1) * steps_per_sched, time.perf_counter() - t0


def oracle_parallel(jobs, label: str):
    """Run oracle jobs on all host cores (one single-threaded oracle process
    per job at a time, spawned); events/s = all jobs' steps / wall time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    workers = min(cores, len(jobs))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(_oracle_job, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    ev = sum(e for e, _ in res)
    return {"value": ev / wall, "unit": UNIT, "cores": workers, "host_cores": cores, "kind": "oracle",
            "sample": "%s: %d oracle processes at a time, %d events in %.1f s wall" % (label, workers, ev, wall)}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, desc = main_workload(args.workload, 0, args.schedules)
    budget = 8.0
    for _ in range(args.warmup):
        oracle_sample(w, 1.0)
    evs, secs = 0, 0.0
    sample = ""
    for _ in range(args.steps):
        _, sample, e, s_ = oracle_sample(w, budget)
        evs += e
        secs += s_
    value = evs / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": desc, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": "per step: " + sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# Counters of the timed run-kernel launches from one ncu capture each
# (profiles/run_kernel_issue_and_polls.md): warp instructions
# (smsp__inst_executed.sum), uniformised steps and halo-poll iterations
# (kmc_profile_polls) of one launch, DRAM bytes read + written, and the
# instructions of one poll iteration (a launch whose every wait runs out:
# `bench.py --only pollcost`; per warp iteration for the warp kernels, per
# thread iteration for the thread-per-domain kernel).  Each kernel's counts
# hold for the sources it is compiled from with these SHA-256 values and are
# left out of the line once those sources change.
KERNEL_SOURCES = {"run_kernel": ("kmc_kernels.cuh",), "tpd_kernel": ("kmc_kernels.cuh", "kmc_tpd.cuh"),
                  "tpdr_kernel": ("kmc_kernels.cuh", "kmc_tpdr.cuh"),
                  "tpdr64_kernel": ("kmc_kernels.cuh", "kmc_tpdr.cuh", "kmc_tpdr64.cuh")}
NCU_KERNEL_SHA256 = {
    "run_kernel": "90af89946413baa798ef8f01d0c7ce7e5b89bd1e0fd3acf67e20162380c30ad6",
    "tpd_kernel": "5ab1c616b84c8ddd0b73b5d36543cc05ac331f4a3fd1470c4adebfb01c54cb6b",
    "tpdr_kernel": "1c3f3576cd4a8b8ff68d0f0762f1031a3aaaa29eaceace994b1a14a8ede61ed8",
    "tpdr64_kernel": "6b404b82601f0094f4f12fc6fe54ed1788cea73a5585c71dbbe6715c588f5699",
}
# instructions of one poll iteration: per warp iteration for the warp kernels
# and the shared-memory thread kernel, per thread re-read for the 8x8 one
INST_PER_POLL = {"run_kernel": 22.24, "tpd_kernel": 0.85, "tpdr_kernel": 28.38, "tpdr64_kernel": 32.44}
NCU_COUNTS = {
    # (workload, kernel): (warp instructions, steps, poll iterations or None, DRAM bytes) of one launch
    ("ising1024", "tpdr_kernel/rr"): (105701953345, 2580480000, 359845347, 6919936),
    ("ising1024", "run_kernel"): (424586232478, 2580480000, 1572988655, 6585856),
    ("grad", "tpdr_kernel"): (38819166107, 1310720000, 238780472, 5571840),
    ("lattice8192", "tpdr64_kernel"): (18400662534, 524288000, 59494537, 11306240),
    ("batched", "tpd_kernel/k16"): (37003135232, 2636876800, 160081004, 7619467264),
    ("batched", "tpd_kernel/k32"): (73589388272, 5273753600, 637452521, 6709346304),
}
ISSUE_PER_SM_CYCLE = 4  # one warp instruction per scheduler per cycle, four schedulers


def run_kernel_name(lat) -> str:
    """The persistent kernel a lattice's plan launches."""
    if lat.launch()[0] == 3:
        return {8: "tpd_kernel", 64: "tpdr64_kernel"}.get(lat.L_d, "tpdr_kernel")
    return "run_kernel"


def counts_kernel(lat, plan) -> str:
    """The name the ncu counts of a launch are keyed by: the kernel, marked
    "/rr" on a thread plan that deals several replicas round-robin over the
    warps (the same kernel on another domain order, with other counts)."""
    k = run_kernel_name(lat)
    if k in ("tpdr_kernel", "tpdr64_kernel") and plan is not None and len(plan) > 1 and plan[0] == 3 \
            and plan[1] == 2 and lat.n_replicas > 1:
        k += "/rr"
    return k


def ncu_counts(workload: str, kernel: str):
    """The workload's ncu counters on that kernel, if taken on the current kernel source."""
    base = kernel.split("/")[0]
    want = NCU_KERNEL_SHA256.get(base)
    if want is None or want != kernel_source_sha256(base):
        return None
    return NCU_COUNTS.get((workload, kernel))


def launch_traffic(workload: str, kernel: str):
    """DRAM bytes (read + write) of one timed launch from the workload's ncu capture, or None."""
    cnt = ncu_counts(workload, kernel)
    return None if cnt is None else cnt[3]


def issue_roofline(workload: str, kernel: str, steps_per_s: float, sm_mhz: float, polls_per_step=None):
    """Issue-rate view: warp instructions per second against 4 per SM cycle x
    the SMs x the SM clock.  Gross counts every instruction, halo polls
    included; net leaves out the poll iterations (busy-waiting, not work).
    With polls_per_step (this run's own count) the gross figure uses it, else
    the capture's."""
    import torch
    cnt = ncu_counts(workload, kernel)
    ipp = INST_PER_POLL.get(kernel.split("/")[0])
    if cnt is None or ipp is None:
        return None
    inst, steps, polls, _ = cnt
    if polls is None and polls_per_step is None:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = ISSUE_PER_SM_CYCLE * sms * sm_mhz * 1e6
    # the capture's polls where it counted them, else this run's
    work = inst / steps - (polls / steps if polls is not None else polls_per_step) * ipp
    pps = polls / steps if polls_per_step is None else polls_per_step
    gross = work + pps * ipp
    return {"bound": "issue", "unit": "warp-inst/s", "peak": peak,
            "achieved": gross * steps_per_s, "frac": gross * steps_per_s / peak,
            "achieved_net": work * steps_per_s, "frac_net": work * steps_per_s / peak,
            "inst_per_step": gross, "inst_per_step_net": work, "polls_per_step": pps,
            "inst_per_poll": ipp,
            "source": "ncu smsp__inst_executed of one timed launch, less its halo-poll iterations x instructions "
                      "per poll iteration; peak = 4 warp instructions per SM cycle x %d SMs x %.0f MHz" % (sms, sm_mhz)}


def kernel_source_sha256(kernel: str = "") -> str:
    """SHA-256 over the device code of one run kernel (its sources in
    KERNEL_SOURCES), or of all of them, comments and blank lines left out, so
    that a comment edit keeps counters taken on the same code."""
    import hashlib
    import re
    h = hashlib.sha256()
    names = KERNEL_SOURCES[kernel] if kernel else ("kmc_kernels.cuh", "kmc_tpd.cuh", "kmc_tpdr.cuh", "kmc_tpdr64.cuh")
    for name in names:
        with open(os.path.join(ROOT, "paper_1403_4674_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()


def device_time(step, steps: int, warmup: int, flush, stream):
    """Per-step device milliseconds (CUDA events on `stream`, L2 flushed before
    each timed step outside the event pair)."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    out = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def roofline(bytes_per_launch: float, launch_s: float, peaks: dict, traffic=None):
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_per_launch / launch_s / 1e9 if launch_s > 0 else 0.0
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "traffic": traffic, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------
def variant_batched(args, peaks, flush, stream):
    """512 uneven replicas: domain side, k and launch plan per group chosen by
    the autotuner; one CUDA graph per step (all groups concurrent)."""
    import torch
    from paper_1403_4674_gb300 import autotune, workloads as wl
    w = wl.batched_replicas(512, master=512)
    n_sched, obs_every = (args.schedules if args.schedules > 0 else 200), 10  # shorter only for profiling captures
    t0 = time.perf_counter()
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    if args.plan:
        # profiling runs: the whole batch as one group at L_d = 8 and k = --batch-k on the given plan
        choices = [autotune.GroupChoice(replicas=list(range(len(w.L))), L_d=8, k=args.batch_k,
                                        plan=tuple(int(x) for x in args.plan.split(",")), events_per_s=0.0)]
    else:
        plans = [(0, 0, 16), (3, 0, 4), (3, 3 * sm, 4), (3, 6 * sm, 2), (1, 4, 16), (1, 16, 16), (1, 16, 8),
                 (2, sm, 16), (2, 2 * sm, 12), (2, 3 * sm, 8)]
        choices = autotune.tune_batch(w.L, w.beta, w.h, w.seeds, k_candidates=(4, 8, 16, 32),
                                      Ld_candidates=(8, 16, 32, 64), plans=plans, trial_schedules=20)
    tune_s = time.perf_counter() - t0
    # oracle on a 64-replica subset, each with its group's domain side and k
    grp = {}
    for ch in choices:
        for i in ch.replicas:
            grp[i] = (ch.L_d, ch.k)
    sub = list(range(0, len(w.L), max(1, len(w.L) // 64)))[:64]
    cpu = None if args.no_cpu else oracle_parallel(
        [(w.L[i], grp[i][0], grp[i][1], w.seeds[i], w.beta[i], w.h[i], False, 1.5) for i in sub],
        "64 of the 512 replicas with their tuned L_d and k, about 1.5 s each")
    batch = autotune.Batch(w.L, w.beta, w.h, w.seeds, choices)
    graph = batch.capture(n_sched, obs_every, reset=0)
    ms = device_time(graph.replay, args.steps, args.warmup, flush, stream)
    ev = batch.events_per_schedule() * n_sched
    # the ncu counters were taken on the whole batch as one group at L_d = 8
    # on a thread-per-domain plan (its state stays in L2 on any such plan),
    # per k
    one_thread_group = len(choices) == 1 and choices[0].L_d == 8 and choices[0].plan[0] == 3
    ckern = "tpd_kernel/k%d" % choices[0].k
    polls = None
    if args.plan:
        # profiling runs: one more step outside the graph, profiled, for its halo-poll count
        for lat in batch.lattices:
            lat.profile(True)
        batch.run(n_sched, obs_every, reset=0)
        batch.sync()
        polls = sum(lat.profile_polls() for lat in batch.lattices)
    by = sum(schedule_bytes(lat.L, lat.L_d, lat.ks) for lat in batch.lattices) * n_sched
    dev_s = sum(ms) / 1000.0
    out = {"value": ev * args.steps / dev_s, "unit": UNIT, "ms_per_step": statistics.mean(ms),
           "workload": "512 replicas, L=16*round(exp(U[ln32,ln512])/16), T~U[1.5,3.5], h~U[-0.1,0.1], "
                       "%d palindromic schedules, obs every %d; L_d, k and plan autotuned per group; "
                       "one CUDA graph per step" % (n_sched, obs_every),
           "groups": [{"replicas": len(ch.replicas), "L_d": ch.L_d, "k": ch.k, "plan": list(ch.plan),
                       "tuned_events_per_s": ch.events_per_s} for ch in choices],
           "tune_s": tune_s, "events_per_step": ev, "polls_per_launch": polls,
           "roofline": roofline(by, dev_s / args.steps, peaks,
                                launch_traffic("batched", ckern) if one_thread_group else None),
           "cpu_baseline": cpu}
    out["roofline"]["note"] = "step-level: the groups' run kernels overlap on concurrent streams"
    iss = issue_roofline("batched", ckern, ev * args.steps / dev_s, float(peaks.get("sm_max_mhz", 2070.0))) \
        if one_thread_group else None
    if iss is not None:
        iss["note"] = "counts of the single-context configuration of the same batch; steps/s of the whole step"
        out["roofline"]["issue"] = iss
    batch.close()
    return out


def variant_grad(args, peaks, flush, stream):
    """256 x 256^2 at T=2.4, h=0.02, k=8, 5000 schedules with FP64 score
    accumulation, then LR estimates of d<e>/d(beta,h) and d<m>/d(beta,h)."""
    import torch
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import autotune, workloads as wl
    w = wl.grad_replicas(256, seed_master=256, k=8)
    cpu = None if args.no_cpu else oracle_parallel(
        [(w.L[i], w.L_d, w.k, w.seeds[i], w.beta[i], w.h[i], True, 4.0) for i in range(16)],
        "16 of the 256 replicas with scores, about 4 s each")
    lat = kmc.Lattice(w.L, w.L_d, w.k, w.seeds, init=0)
    lat.set_rates(w.beta, w.h)
    lat.enable_grad(True)
    if args.plan:
        plan = tuple(int(x) for x in args.plan.split(","))
        lat.set_launch(*plan)
    else:
        plan, _ = autotune.tune_plan(lat, w.beta, w.h, trial_schedules=100)
    lat.profile(True)
    n = args.schedules if args.schedules > 0 else w.schedules  # a shorter run only for profiling captures
    out_obs = torch.empty((1, lat.n_replicas, 6), dtype=torch.float64, device="cuda")
    grads = {}

    def step():
        lat.reset(kmc.KMC_INIT_RANDOM)
        lat.run(n, obs_every=n, out=out_obs)
        grads["e"] = lat.lr_estimate(out_obs[0, :, 0])
        grads["m"] = lat.lr_estimate(out_obs[0, :, 1])

    ms = device_time(step, args.steps, args.warmup, flush, stream)
    lat.sync()
    lat.profile_read()
    lat.profile_polls()
    step()
    run_ms, run_n = lat.profile_read()
    polls = lat.profile_polls()
    ev = lat.events_per_schedule() * n
    by = schedule_bytes(lat.L, lat.L_d, lat.ks) * n
    dev_s = sum(ms) / 1000.0
    ge, gm = grads["e"].cpu().numpy(), grads["m"].cpu().numpy()
    out = {"value": ev * args.steps / dev_s, "unit": UNIT, "ms_per_step": statistics.mean(ms),
           "workload": "256 x 256^2 Ising, T=2.4, h=0.02, L_d=32, k=8, %d palindromic schedules, FP64 scores, "
                       "LR gradients of <e> and <m> w.r.t. (beta, h) per step" % n,
           "plan": list(plan), "launch": list(lat.launch()),
           "lr_grad_e_beta_h": [float(ge[0]), float(ge[1])], "lr_grad_m_beta_h": [float(gm[0]), float(gm[1])],
           "events_per_step": ev, "cpu_baseline": cpu, "polls_per_launch": polls / max(run_n, 1),
           "roofline": roofline(by, (run_ms / 1000.0) / max(run_n, 1), peaks,
                                launch_traffic("grad", counts_kernel(lat, plan)))}
    iss = issue_roofline("grad", counts_kernel(lat, plan), ev * max(run_n, 1) / (run_ms / 1000.0) if run_ms > 0 else 0.0,
                         float(peaks.get("sm_max_mhz", 2070.0)), polls / max(ev * max(run_n, 1), 1))
    if iss is not None:
        out["roofline"]["issue"] = iss
    lat.close()
    return out


def variant_lattice8192(args, peaks, flush, stream):
    """One 8192^2 lattice (67M sites), T=2.269, h=0.01, L_d=64, k=8, 2000
    palindromic schedules, plan tuned."""
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import autotune, workloads as wl
    w = wl.lattice_8192(seed=8192)
    cpu = None
    if not args.no_cpu:
        cpu = oracle_parallel([(w.L[0], w.L_d, w.k, w.seeds[0], w.beta[0], w.h[0], False, 0.0)],
                              "one schedule of the 8192^2 lattice (one process: a single lattice)")
    lat = kmc.Lattice(w.L, w.L_d, w.k, w.seeds, init=0)
    lat.set_rates(w.beta, w.h)
    if args.plan:
        plan = tuple(int(x) for x in args.plan.split(","))
        lat.set_launch(*plan)
    else:
        plan, _ = autotune.tune_plan(lat, w.beta, w.h, trial_schedules=20)
    lat.profile(True)
    n = args.schedules if args.schedules > 0 else w.schedules  # a shorter run only for profiling captures

    def step():
        lat.reset(kmc.KMC_INIT_RANDOM)
        lat.run(n)

    ms = device_time(step, args.steps, args.warmup, flush, stream)
    lat.sync()
    lat.profile_read()
    lat.profile_polls()
    step()
    run_ms, run_n = lat.profile_read()
    polls = lat.profile_polls()
    ev = lat.events_per_schedule() * n
    by = schedule_bytes(lat.L, lat.L_d, lat.ks) * n
    dev_s = sum(ms) / 1000.0
    out = {"value": ev * args.steps / dev_s, "unit": UNIT, "ms_per_step": statistics.mean(ms),
           "workload": "8192x8192 periodic Ising (67M sites), T=2.269, h=0.01, L_d=64, k=8, %d palindromic "
                       "schedules" % n,
           "plan": list(plan), "launch": list(lat.launch()), "events_per_step": ev, "cpu_baseline": cpu,
           "polls_per_launch": polls / max(run_n, 1),
           "roofline": roofline(by, (run_ms / 1000.0) / max(run_n, 1), peaks,
                                launch_traffic("lattice8192", counts_kernel(lat, plan)))}
    rate = ev * max(run_n, 1) / (run_ms / 1000.0) if run_ms > 0 else 0.0
    iss = issue_roofline("lattice8192", counts_kernel(lat, plan), rate, float(peaks.get("sm_max_mhz", 2070.0)),
                         polls / max(ev * max(run_n, 1), 1))
    if iss is not None:
        out["roofline"]["issue"] = iss
    lat.close()
    return out


def variant_ring(args, peaks, flush, stream):
    """The paper's 1D experiment (Sec. 3.1) as one step: the 8-spin ring at
    beta J = 0.5, Barker, its 8 pair-of-up-spins ICs x 6000 trajectories for
    every N_D in {1, 2, 4, 8} and N_I in {1, 2, 5, 10}: S = 800 steps per
    trajectory in random domain orders per sweep, ensemble sums after every
    domain process.  16 contexts (one per setting, 48000 trajectories each)
    on 16 streams; each timed step continues every trajectory by S steps."""
    import torch
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    NS, S, per_ic = 8, 800, 6000
    ics = [(1 << i) | (1 << ((i + 1) % 8)) for i in (6, 5, 4, 3, 2, 1, 0, 7)]
    runs = []
    for a, ND in enumerate((1, 2, 4, 8)):
        for b, NI in enumerate((1, 2, 5, 10)):
            n = 8 * per_ic
            ring = kmc.Ring(NS, NS // ND, NI, wl.replica_seeds(800 + 4 * a + b, n), [ics[i % 8] for i in range(n)])
            ring.set_rates([0.5] * n, [0.0] * n, law=kmc.KMC_RATE_BARKER)
            n_sched = S // (NI * ND)
            n_rec = ring.n_records(n_sched, kmc.KMC_SCHEDULE_RANDOM_PERM, 1)
            ens = torch.empty((n_rec, 4 + NS), dtype=torch.int64, device="cuda")
            runs.append((ring, n_sched, ens, torch.cuda.Stream()))

    def step():
        main = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(main)
        for ring, n_sched, ens, st in runs:
            st.wait_event(start)
            with torch.cuda.stream(st):
                ring.run(n_sched, schedule=kmc.KMC_SCHEDULE_RANDOM_PERM, obs_every=1, records=False,
                         ensemble=True, out=(None, None, ens))
                ev = torch.cuda.Event()
                ev.record(st)
            main.wait_event(ev)

    ms = device_time(step, args.steps, args.warmup, flush, stream)
    ev = sum(r.n_traj for r, _, _, _ in runs) * S
    dev_s = sum(ms) / 1000.0
    # <H>/N_S at the last record of the N_D = 4, N_I = 5 setting (equilibrium: -0.465649)
    ens = runs[10][2][-1].cpu().numpy()
    out = {"value": ev * args.steps / dev_s, "unit": UNIT, "ms_per_step": statistics.mean(ms),
           "workload": "8-spin ring (Sec. 3.1), beta J = 0.5, Barker, 8 ICs x 6000 trajectories for each of "
                       "N_D in {1,2,4,8} x N_I in {1,2,5,10}, S = 800 steps per trajectory, random domain order "
                       "per sweep, ensemble sums after every domain process",
           "events_per_step": ev, "launches_per_step": len(runs),
           "energy_per_site_ND4_NI5": float(-ens[0] / (runs[10][0].n_traj * NS))}
    for r, _, _, _ in runs:
        r.close()
    return out


def part_settings(stripes, blocks):
    """The 28 settings (L, n_traj, S, kind, N_D, N_I) of the paper's 2D
    experiments (Sec. 3.2), S the steps per trajectory of one timed step."""
    settings = []
    for L, n_traj, S, parts in [(12, 500, 16000, [(stripes, 2), (stripes, 4), (blocks, 4)]),
                                (100, 50, 160000, [(stripes, 2), (stripes, 4), (blocks, 4), (blocks, 16)])]:
        for kind, ND in parts:
            for NI in (1, 2, 5, 10):
                settings.append((L, n_traj, S, kind, ND, NI))
    return settings


def part_launch_groups(settings, blocks, n_streams):
    """Launch groups of the 2D experiments' settings (L, n_traj, S, kind, N_D,
    N_I): each group is a list of setting indices run one after another on
    one stream, the groups launched in list order.

    The longest chains first: the settings with the most steps per trajectory
    (100^2: 1.6e5) start at once, one stream each, ordered by expected length
    (smallest N_I first, then blocks before stripes and more domains first) so
    that the longest chains take SMs of their own before the shorter ones
    double up on SMs.  The shorter settings (12^2) follow, smallest N_I first,
    dealt round-robin over `n_streams` streams (0: one stream each).  One
    stream (500 trajectories at a time beside the 800 of 100^2) crowds the
    100^2 warps least: 124.7 ms per step against 126.8 on two streams and
    129.9 with all twelve at once."""
    S_max = max(s[2] for s in settings)
    long_ = sorted((i for i in range(len(settings)) if settings[i][2] == S_max),
                   key=lambda i: (settings[i][5], settings[i][3] != blocks, -settings[i][4]))
    short = sorted((i for i in range(len(settings)) if settings[i][2] < S_max), key=lambda i: settings[i][5])
    n_sh = min(n_streams, len(short)) if n_streams > 0 else len(short)
    return [[i] for i in long_] + [short[c::n_sh] for c in range(n_sh)]


def variant_part(args, peaks, flush, stream):
    """The paper's 2D experiments (Sec. 3.2) as one step: 12^2 x 500 and
    100^2 x 50 trajectories at T = 2.4, Barker, from the all-up state, in
    vertical stripes (N_D = 2, 4) and square blocks (N_D = 4; 16 for 100^2),
    N_I in {1, 2, 5, 10}, the random domain order per sweep; per timed step
    every trajectory advances 1.6e4 (12^2) or 1.6e5 (100^2) steps with 64
    energy records.  28 contexts; see `--part-streams` for their streams."""
    import torch
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    B_ = kmc.KMC_PART_BLOCKS
    settings = part_settings(kmc.KMC_PART_STRIPES, B_)
    runs = []
    for i, (L, n_traj, S, kind, ND, NI) in enumerate(settings):
        g = kmc.Partitioned(L, kind, ND, NI, wl.replica_seeds(1200 + i, n_traj))
        g.set_rates([1 / 2.4] * n_traj, law=kmc.KMC_RATE_BARKER)
        n_sched = S // (ND * NI)
        obs_every = max(1, n_sched * ND // 64)
        obs = torch.empty((g.n_records(n_sched, kmc.KMC_SCHEDULE_RANDOM_PERM, obs_every), n_traj, 4),
                          dtype=torch.float64, device="cuda")
        runs.append((g, n_sched, obs_every, obs, torch.cuda.Stream(), n_traj * S))

    groups = [(runs[members[0]][4], members) for members in part_launch_groups(settings, B_, args.part_streams)]

    def step():
        main = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(main)
        for st, members in groups:
            st.wait_event(start)
            with torch.cuda.stream(st):
                for g, n_sched, obs_every, obs, _, _ in (runs[i] for i in members):
                    g.run(n_sched, schedule=kmc.KMC_SCHEDULE_RANDOM_PERM, obs_every=obs_every, out=obs)
                ev = torch.cuda.Event()
                ev.record(st)
            main.wait_event(ev)

    ms = device_time(step, args.steps, args.warmup, flush, stream)
    ev = sum(r[5] for r in runs)
    dev_s = sum(ms) / 1000.0
    # mean energy per site over the last records of the 12^2, 4-stripe, N_I = 5 setting
    e12 = float(runs[6][3][-16:, :, 0].mean().item())
    out = {"value": ev * args.steps / dev_s, "unit": UNIT, "ms_per_step": statistics.mean(ms),
           "workload": "Sec. 3.2 grid: 12^2 x 500 and 100^2 x 50 trajectories, T = 2.4, Barker, stripes N_D in "
                       "{2,4}, blocks N_D = 4 (and 16 for 100^2), N_I in {1,2,5,10}, random domain order per "
                       "sweep; per step 1.6e4 (12^2) / 1.6e5 (100^2) steps per trajectory",
           "events_per_step": ev, "launches_per_step": len(runs), "streams": len(groups),
           "energy_per_site_12x12_stripes4_NI5": e12}
    for r in runs:
        r[0].close()
    return out


def variant_chain(args, peaks, flush, stream):
    """Latency of one domain's chain: a 64^2 lattice at L_d = 32 (four
    domains, one per colour) at beta = 0, where every uniformised step is a
    real event (Metropolis), so that one palindromic schedule is a chain of
    6k events and four colour hand-offs (colours 1 and 2 run side by side).
    Launch times at k = 4 and k = 16 give the time per event (their
    difference over 72 events) and per hand-off, for the thread plan and a
    warp plan.  This is the floor under the 1024^2 workload's launch time:
    its k = 16, T = 3 replicas run about 70 real events per schedule on
    their critical path."""
    import paper_1403_4674_gb300 as kmc
    n = 2000
    out = {"workload": "64x64, L_d = 32, beta = 0, k in {4, 16}, %d palindromic schedules per launch" % n}
    for name, plan in (("thread", (3, 0, 1)), ("warp", (2, 4, 4))):
        per = {}
        for k in (4, 16):
            lat = kmc.Lattice([64], 32, k, [7])
            lat.set_launch(*plan)
            lat.set_rates([0.0], [0.0])
            lat.run(2)
            lat.sync()
            lat.profile(True)
            lat.profile_read()
            lat.run(n)
            lat.sync()
            ms, runs = lat.profile_read()
            per[k] = ms * 1e6 / max(runs, 1) / n  # ns per schedule
            lat.close()
        ev = (per[16] - per[4]) / (6 * 12)
        hop = (per[4] - 6 * 4 * ev) / 4
        out[name] = {"plan": list(plan), "ns_per_schedule": {str(k): v for k, v in per.items()},
                     "ns_per_event": ev, "ns_per_handoff": hop}
    return out


def variant_pollcost(args, peaks, flush, stream):
    """Instructions of one halo-poll iteration, for the net issue rate: one
    launch of the default workload's context and plan in which every visit
    waits for one neighbour visit more than will ever come
    (kmc_debug_barrier), so each warp polls until the 20 ms limit and the
    launch's instructions are almost all poll iterations.  Prints the poll
    count; `ncu --metrics smsp__inst_executed.sum -k regex:run_kernel` of the
    same command gives the instructions, and their ratio is the cost of one
    iteration.  The context is checked to be usable afterwards."""
    import torch
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    w, desc = main_workload("ising1024", 0, 0)
    ks = [w.k_of(r) for r in range(len(w.L))]
    inits = [w.init_of(r) for r in range(len(w.L))]
    lat = kmc.Lattice(w.L, w.L_d, ks[0], w.seeds, init=inits[0])
    lat.set_replica_params(k=ks, init=inits)
    lat.reset(kmc.KMC_INIT_PER_REPLICA)
    lat.set_rates(w.beta, w.h)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    plan = tuple(int(x) for x in args.plan.split(",")) if args.plan else (2, 5 * sm, 4)
    lat.set_launch(*plan)
    limit_ns = 20_000_000
    kmc.kmc_debug_barrier(lat.ctx, 1, limit_ns)
    lat.profile(True)
    lat.run(1)
    try:
        lat.sync()
        status = 0
    except kmc.KmcError as e:
        status = e.status
    polls = lat.profile_polls()
    kmc.kmc_debug_barrier(lat.ctx, 0, 0)
    lat.reset(kmc.KMC_INIT_PER_REPLICA)
    lat.run(1)
    lat.sync()
    out = {"workload": desc, "plan": list(plan), "launch": list(lat.launch()), "limit_ns": limit_ns,
           "status_after_timeout": status, "polls": polls}
    if status != -5:
        raise RuntimeError("expected KMC_ETIMEOUT from the waits that run out, got %d" % status)
    # the same workload on the shared-memory thread-per-domain kernel (its
    # count is per warp poll round)
    lat.set_launch(3, 0, 1)
    kmc.kmc_debug_barrier(lat.ctx, 1, limit_ns)
    lat.profile_polls()
    lat.run(1)
    try:
        lat.sync()
        status = 0
    except kmc.KmcError as e:
        status = e.status
    out["thread_rows"] = {"launch": list(lat.launch()), "status_after_timeout": status, "polls": lat.profile_polls()}
    kmc.kmc_debug_barrier(lat.ctx, 0, 0)
    lat.close()
    # the 64x64 thread kernel (count per warp poll round): the 8192^2 lattice
    w64 = wl.lattice_8192(seed=8192)
    lat = kmc.Lattice(w64.L, w64.L_d, w64.k, w64.seeds)
    lat.set_rates(w64.beta, w64.h)
    lat.set_launch(3, 1, 4)
    kmc.kmc_debug_barrier(lat.ctx, 1, limit_ns)
    lat.profile(True)
    lat.run(1)
    try:
        lat.sync()
        status = 0
    except kmc.KmcError as e:
        status = e.status
    out["thread_rows64"] = {"workload": "8192^2, L_d = 64, k = 8", "launch": list(lat.launch()),
                            "status_after_timeout": status, "polls": lat.profile_polls()}
    kmc.kmc_debug_barrier(lat.ctx, 0, 0)
    lat.close()
    if status != -5:
        raise RuntimeError("expected KMC_ETIMEOUT from the 64x64 thread plan's waits, got %d" % status)
    # the same for the thread-per-domain kernel (its count is per thread): the
    # batched workload's 512 replicas at L_d = 8, k = 16 on the library's plan
    wb = wl.batched_replicas(512, master=512)
    lat = kmc.Lattice(wb.L, 8, 16, wb.seeds)
    lat.set_rates(wb.beta, wb.h)
    kmc.kmc_debug_barrier(lat.ctx, 1, limit_ns)
    lat.profile(True)
    lat.run(1)
    try:
        lat.sync()
        status = 0
    except kmc.KmcError as e:
        status = e.status
    out["threads"] = {"workload": "512 batched replicas, L_d = 8, k = 16", "launch": list(lat.launch()),
                      "status_after_timeout": status, "polls": lat.profile_polls()}
    kmc.kmc_debug_barrier(lat.ctx, 0, 0)
    lat.close()
    if status != -5:
        raise RuntimeError("expected KMC_ETIMEOUT from the thread plan's waits, got %d" % status)
    return out


VARIANTS = {"batched": "variant_batched", "grad": "variant_grad", "lattice8192": "variant_lattice8192",
            "ring8": "variant_ring", "partitions2d": "variant_part", "pollcost": "variant_pollcost",
            "chain": "variant_chain"}


def only_variant(args):
    import torch
    torch.cuda.set_device(0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    flush = torch.empty(L2_FLUSH_FLOATS, dtype=torch.float32, device="cuda")
    out = globals()[VARIANTS[args.only]](args, peaks, flush, torch.cuda.current_stream())
    print(json.dumps({"variant": args.only, **out}))


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.only:
        return only_variant(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # the CPU baseline runs before any CUDA work (rank 0, N = 1 only)
    w, desc = main_workload(args.workload, rank, args.schedules)
    cpu = None
    if world == 1 and not args.no_cpu:
        v, sample, e, s = oracle_sample(w, 12.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": "%s; %d events in %.1f s, single thread" % (sample, e, s)}
        # the same replicas on every host core, one oracle process per replica
        jobs = [(w.L[r], w.L_d, w.k_of(r), w.seeds[r], w.beta[r], w.h[r], False, 5.0)
                for r in range(len(w.L)) if w.init_of(r) == 0]
        cpu["all_cores"] = oracle_parallel(jobs, "the %d random-start replicas (k x T), about 5 s each" % len(jobs))

    import torch
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import autotune

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass

    # one context for the whole workload, created and tuned outside the timed region
    ks = [w.k_of(r) for r in range(len(w.L))]
    inits = [w.init_of(r) for r in range(len(w.L))]
    lat = kmc.Lattice(w.L, w.L_d, ks[0], w.seeds, init=inits[0])
    per_replica = len(set(ks)) > 1 or len(set(inits)) > 1
    if per_replica:
        lat.set_replica_params(k=ks, init=inits)
    reset_mode = kmc.KMC_INIT_PER_REPLICA if per_replica else inits[0]
    lat.reset(reset_mode)
    lat.set_rates(w.beta, w.h)
    t0 = time.perf_counter()
    if args.plan:
        plan = tuple(int(x) for x in args.plan.split(","))
        lat.set_launch(*plan)
    else:
        plan, _ = autotune.tune_plan(lat, w.beta, w.h, trial_schedules=200 if w.L[0] <= 1024 else 2)
    tune_s = time.perf_counter() - t0
    lat.profile(True)
    n_obs = w.schedules // w.obs_every if w.obs_every > 0 else 0
    obs_buf = (torch.empty((n_obs, lat.n_replicas, 4), dtype=torch.float64, device="cuda") if n_obs > 0 else None)

    def step():
        lat.reset(reset_mode)
        lat.run(w.schedules, obs_every=w.obs_every, out=obs_buf)

    flush = torch.empty(L2_FLUSH_FLOATS, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    lat.profile_read()  # discard warm-up timings
    lat.profile_polls()
    launches0 = lat.kernel_launches()

    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    step_ms = device_time(step, args.steps, 0, flush, stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = lat.kernel_launches() - launches0
    run_ms, run_n = lat.profile_read()
    polls = lat.profile_polls()

    # the timed step's final state and records, for the bit-exactness check below
    dev_spins = lat.spins.clone()
    dev_obs = obs_buf.clone() if obs_buf is not None else None
    events_step = lat.events_per_schedule() * w.schedules
    bytes_step = schedule_bytes(lat.L, lat.L_d, lat.ks) * w.schedules
    dev_s = max_over_ranks(sum(step_ms) / 1000.0, dist, "cuda")
    value = whole_job_rate(events_step, args.steps, world, dev_s)
    flips = int(lat.observables()["flips"].sum())

    # end-to-end through the public API with host buffers
    e2e = None
    bit_exact = None
    if not args.no_e2e:
        lat.reset(reset_mode)
        lat.sync()
        host_in = lat.spins.cpu().pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        host_obs = torch.empty(obs_buf.shape, dtype=torch.float64).pin_memory() if obs_buf is not None else None
        d2h = host_out.numel() + (host_obs.numel() * 8 if host_obs is not None else 0)

        def e2e_step():
            lat.spins.copy_(host_in, non_blocking=True)
            lat.reset(kmc.KMC_INIT_KEEP)
            lat.run(w.schedules, obs_every=w.obs_every, out=obs_buf)
            host_out.copy_(lat.spins, non_blocking=True)
            if host_obs is not None:
                host_obs.copy_(obs_buf, non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": whole_job_rate(events_step, args.steps, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(host_in.numel()), "d2h_bytes_per_step": int(d2h)}
        # every step restarts from the same state and Philox position, so the
        # end-to-end run must reproduce the device-timed run bit for bit
        # (parity with the oracle in these launch configurations is checked by
        # tests/test_gpu_bench_configs.py)
        # (the clock column sums the domains' FP64 clock advances with atomics,
        # in no fixed order: equal to 1e-12 relative, the oracle tolerance)
        bit_exact = {"e2e_spins_equal_device_run": bool(torch.equal(host_out, dev_spins.cpu()))}
        if host_obs is not None:
            do = dev_obs.cpu()
            bit_exact["e2e_records_e_m_em_equal_device_run"] = bool(torch.equal(host_obs[..., :3], do[..., :3]))
            bit_exact["e2e_records_clock_rel_diff_max"] = float(
                ((host_obs[..., 3] - do[..., 3]).abs() / do[..., 3].abs().clamp_min(1e-300)).max().item())

    full = args.schedules == 0
    kern = run_kernel_name(lat)
    ckern = counts_kernel(lat, plan)
    traffic = launch_traffic(args.workload, ckern) if full else None
    avg_run_s = (run_ms / 1000.0) / max(run_n, 1)
    roof = roofline(bytes_step, avg_run_s, peaks, traffic)
    roof.update({"kernel": "kmcdev::" + kern, "run_kernel_ms_avg": 1000 * avg_run_s,
                 "run_kernel_launches": run_n, "algorithmic_bytes_per_launch": bytes_step,
                 "step_level_achieved": bytes_step * args.steps / dev_s / 1e9,
                 "polls_per_launch": polls / max(run_n, 1)})
    # the bound this kernel actually meets: instruction issue
    if full and clk.get("sm_mhz") and avg_run_s > 0:
        iss = issue_roofline(args.workload, ckern, events_step / avg_run_s, clk["sm_mhz"],
                             polls / max(events_step * max(run_n, 1), 1))
        if iss is not None:
            roof["issue"] = iss

    variants = None
    if world == 1 and not args.no_variants and args.workload == "ising1024":
        variants = {"batched": variant_batched(args, peaks, flush, stream),
                    "grad": variant_grad(args, peaks, flush, stream),
                    "lattice8192": variant_lattice8192(args, peaks, flush, stream),
                    "ring8": variant_ring(args, peaks, flush, stream),
                    "partitions2d": variant_part(args, peaks, flush, stream)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": {"workload": desc, "events_per_step": events_step,
                           "real_flips_per_step": flips,
                           "real_flips_per_s": flips * world / (dev_s / args.steps),
                           "l2": "flushed between timed steps (512 MB write outside the event pair)",
                           "parallelism": ("replicas only, %d ranks" % world if world > 1 else "1 GPU") +
                                          ", one run-kernel launch per step",
                           "plan": list(plan), "launch": list(lat.launch()), "tune_s": tune_s,
                           "threads_per_domain": (("one thread per domain, 32 domains per warp, state in shared "
                                                   "memory" if kern in ("tpdr_kernel", "tpdr64_kernel")
                                                   else "one thread per domain")
                                                  if kern != "run_kernel" else "one warp per domain") +
                                                 (", replicas dealt round-robin over the warps"
                                                  if ckern.endswith("/rr") else "") +
                                                 " (the tuner's choice between thread and warp plans)",
                           "wall_s": wall},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "bit_exact": bit_exact,
                "clocks": clk, "variants": variants}
        print(json.dumps(line), flush=True)
    lat.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
