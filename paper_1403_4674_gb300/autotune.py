"""Measured choice of launch plan, domain side and steps per visit.

Nothing here changes what a replica computes for a given (L_d, k): the launch
plan only decides which CTA runs which domain, and the library's results do
not depend on it.  The domain side L_d and the steps per visit k do change
the dynamics (the paper's N_D and N_I, Sec. 3) but not the stationary
distribution (Eqs. 9-10).  Every uniformised step advances its domain's clock
by the same expected 1/(n_d nu) per site, so events per second is a fair
figure of merit across L_d and k: it is simulated time per second times the
number of sites.  Tune L_d and k only where equilibrium sampling is the goal,
and pass a single value otherwise.

A context has one L_d, and a replica of side L needs L to be a multiple of
2 L_d (an even number of domains per side keeps the 2x2 colouring valid under
periodic wrap).  `tune_batch` therefore splits a batch into groups by the
largest valid L_d and tunes each group; `Batch` runs the groups concurrently,
one stream each, and can capture a whole batch step in one CUDA graph.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from .api import (KMC_INIT_PER_REPLICA, KMC_INIT_RANDOM, KMC_LAUNCH_AUTO, KMC_LAUNCH_CLUSTER,
                  KMC_LAUNCH_GRID, KMC_LAUNCH_THREADS, KmcError, Lattice)

DOMAIN_SIDES = (8, 16, 32, 64)
Plan = Tuple[int, int, int]  # (mode, size, warps per CTA) as for kmc_set_launch


def max_domain_side(L: int, candidates: Sequence[int] = DOMAIN_SIDES) -> int:
    best = 0
    for Ld in candidates:
        if L % (2 * Ld) == 0:
            best = max(best, Ld)
    if best == 0:
        raise ValueError("no domain side in %s divides L = %d into an even count" % (tuple(candidates), L))
    return best


def plan_candidates(sm_count: int, L_d: Optional[int] = None) -> List[Plan]:
    """Launch plans worth measuring: the library default, clusters of every
    size (the library packs as many replicas per cluster as fit), and
    cooperative grids of one to six CTAs per SM with 20-24 resident warps
    where the kernel's registers allow (small CTAs spread the cost-balanced
    colour chunks over more, shorter lists; the library rejects shapes that
    do not fit), and the thread-per-domain plans of the domain side."""
    out: List[Plan] = [(KMC_LAUNCH_AUTO, 0, 16)]
    out += [(KMC_LAUNCH_CLUSTER, c, 16) for c in (1, 2, 4, 8, 16)]
    out += [(KMC_LAUNCH_CLUSTER, c, 8) for c in (4, 16)]
    out += [(KMC_LAUNCH_GRID, sm_count, 16), (KMC_LAUNCH_GRID, 2 * sm_count, 8),
            (KMC_LAUNCH_GRID, 2 * sm_count, 10), (KMC_LAUNCH_GRID, 2 * sm_count, 12),
            (KMC_LAUNCH_GRID, 3 * sm_count, 8), (KMC_LAUNCH_GRID, 4 * sm_count, 5),
            (KMC_LAUNCH_GRID, 5 * sm_count, 4), (KMC_LAUNCH_GRID, 6 * sm_count, 4)]
    # one thread per domain: for 8x8 domains the library's balanced grid and
    # grids of fixed size; 16x16, 32x32 and 64x64 ones take one domain per
    # thread, their size choosing the order of the domains over the warps (1:
    # replica after replica, 2: round-robin over the replicas)
    if L_d in (16, 32, 64):
        out += [(KMC_LAUNCH_THREADS, o, w) for o in (1, 2) for w in (4, 1)]
    elif L_d in (None, 8):
        out += [(KMC_LAUNCH_THREADS, 0, 4), (KMC_LAUNCH_THREADS, 0, 1)]
        out += [(KMC_LAUNCH_THREADS, m * sm_count, w) for m, w in ((3, 4), (2, 4), (4, 2), (6, 2))]
    return out


@dataclass
class Trial:
    L_d: int
    k: int
    plan: Plan
    events_per_s: float = 0.0
    launch: Optional[tuple] = None
    error: Optional[str] = None


def _timed_events_per_s(lat: Lattice, n_sched: int, stream: torch.cuda.Stream) -> float:
    with torch.cuda.stream(stream):
        lat.run(2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.run(n_sched)
        e1.record(stream)
    e1.synchronize()
    lat.sync()
    return lat.events_per_schedule() * n_sched / (e0.elapsed_time(e1) / 1000.0)


def measure(L: Sequence[int], L_d: int, ks: Sequence[int], seeds: Sequence[int], beta: Sequence[float],
            h: Sequence[float], plans: Sequence[Plan], trial_schedules: int = 50, law: int = 0,
            grad: bool = False) -> List[Trial]:
    """Events/s of one group geometry under each plan, on a scratch context
    (the caller's lattices are not touched); grad measures the score-carrying
    kernels."""
    stream = torch.cuda.Stream()
    trials: List[Trial] = []
    with torch.cuda.stream(stream):
        try:
            lat = Lattice(L, L_d, ks[0], seeds, init=KMC_INIT_RANDOM)
        except KmcError as exc:
            return [Trial(L_d, ks[0], p, error=str(exc)) for p in plans]
        try:
            if any(k != ks[0] for k in ks):
                lat.set_replica_params(k=list(ks))
            lat.set_rates(list(beta), list(h), law=law)
            if grad:
                lat.enable_grad(True)
            for p in plans:
                t = Trial(L_d, max(ks), p)
                try:
                    lat.set_launch(*p)
                except KmcError as exc:
                    t.error = str(exc)
                    trials.append(t)
                    continue
                t.launch = lat.launch()
                t.events_per_s = _timed_events_per_s(lat, trial_schedules, stream)
                trials.append(t)
        finally:
            lat.close()
    return trials


def tune_plan(lat: Lattice, beta: Sequence[float], h: Sequence[float], plans: Optional[Sequence[Plan]] = None,
              trial_schedules: int = 50, law: int = 0) -> Tuple[Plan, List[Trial]]:
    """Measure the plans on a scratch copy of `lat`'s geometry and install
    the fastest on `lat`."""
    if plans is None:
        plans = plan_candidates(torch.cuda.get_device_properties(lat.spins.device).multi_processor_count, lat.L_d)
    trials = measure(lat.L, lat.L_d, lat.ks, lat.seeds, beta, h, plans, trial_schedules, law,
                     grad=lat.grad_enabled)
    ok = [t for t in trials if t.error is None]
    if not ok:
        raise KmcError(-1, "no launch plan runs: " + "; ".join(str(t.error) for t in trials))
    best = max(ok, key=lambda t: t.events_per_s)
    lat.set_launch(*best.plan)
    return best.plan, trials


@dataclass
class GroupChoice:
    replicas: List[int]  # indices into the batch
    L_d: int
    k: int
    plan: Plan
    events_per_s: float
    trials: List[Trial] = field(default_factory=list)


def tune_batch(L: Sequence[int], beta: Sequence[float], h: Sequence[float], seeds: Sequence[int],
               k_candidates: Sequence[int] = (8,), Ld_candidates: Sequence[int] = DOMAIN_SIDES,
               plans: Optional[Sequence[Plan]] = None, trial_schedules: int = 20,
               law: int = 0) -> List[GroupChoice]:
    """Group replicas by their largest valid domain side, then pick (L_d, k,
    plan) per group by measured events/s."""
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count

    def plans_for(Ld: int) -> Sequence[Plan]:
        return plans if plans is not None else plan_candidates(sm, Ld)
    groups: Dict[int, List[int]] = {}
    for i, x in enumerate(L):
        groups.setdefault(max_domain_side(x, Ld_candidates), []).append(i)
    out: List[GroupChoice] = []
    for gmax, idx in sorted(groups.items()):
        Lg = [L[i] for i in idx]
        sides = [x for x in Ld_candidates if x <= gmax and all(y % (2 * x) == 0 for y in Lg)]
        trials: List[Trial] = []
        for Ld in sides:
            for k in k_candidates:
                trials += measure(Lg, Ld, [k] * len(idx), [seeds[i] for i in idx], [beta[i] for i in idx],
                                  [h[i] for i in idx], plans_for(Ld), trial_schedules, law)
        ok = [t for t in trials if t.error is None]
        if not ok:
            errs = sorted({str(t.error) for t in trials})[:3]
            raise KmcError(-1, "no configuration runs for a group of %d replicas (largest L = %d): %s"
                           % (len(idx), max(Lg), "; ".join(errs)))
        best = max(ok, key=lambda t: t.events_per_s)
        out.append(GroupChoice(idx, best.L_d, best.k, best.plan, best.events_per_s, trials))
    # Groups that chose the same (L_d, k) can share one context; groups tuned
    # alone may compete for SMs when run side by side (cooperative grids wait
    # for a whole GPU).  Keep whichever partition runs the whole batch faster.
    keys = {}
    for ch in out:
        keys.setdefault((ch.L_d, ch.k), []).append(ch)
    if any(len(v) > 1 for v in keys.values()):
        merged: List[GroupChoice] = []
        for (Ld, k), chs in keys.items():
            if len(chs) == 1:
                merged.append(chs[0])
                continue
            idx = sorted(i for ch in chs for i in ch.replicas)
            trials = measure([L[i] for i in idx], Ld, [k] * len(idx), [seeds[i] for i in idx],
                             [beta[i] for i in idx], [h[i] for i in idx], plans_for(Ld), trial_schedules, law)
            okm = [t for t in trials if t.error is None]
            if not okm:
                merged = []
                break
            best = max(okm, key=lambda t: t.events_per_s)
            merged.append(GroupChoice(idx, Ld, k, best.plan, best.events_per_s, trials))
        if merged and batch_events_per_s(L, beta, h, seeds, merged, trial_schedules, law) > \
                batch_events_per_s(L, beta, h, seeds, out, trial_schedules, law):
            out = merged
    return out


def batch_events_per_s(L, beta, h, seeds, choices: List[GroupChoice], n_sched: int, law: int = 0) -> float:
    """Measured events/s of a whole batch step (all groups concurrently)."""
    batch = Batch(L, beta, h, seeds, choices, law=law)
    try:
        batch.run(2)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.run(n_sched)
        e1.record()
        e1.synchronize()
        return batch.events_per_schedule() * n_sched / (e0.elapsed_time(e1) / 1000.0)
    finally:
        batch.close()


class Batch:
    """A tuned batch: one context and stream per group, run concurrently."""

    def __init__(self, L: Sequence[int], beta: Sequence[float], h: Sequence[float], seeds: Sequence[int],
                 choices: List[GroupChoice], init: int = KMC_INIT_RANDOM, law: int = 0):
        self.L, self.beta, self.h, self.seeds = list(L), list(beta), list(h), list(seeds)
        self.choices = choices
        self.init = init
        self.streams = [torch.cuda.Stream() for _ in choices]
        self.lattices: List[Lattice] = []
        for ch, st in zip(choices, self.streams):
            with torch.cuda.stream(st):
                lat = Lattice([L[i] for i in ch.replicas], ch.L_d, ch.k, [seeds[i] for i in ch.replicas], init=init)
                lat.set_launch(*ch.plan)
                lat.set_rates([beta[i] for i in ch.replicas], [h[i] for i in ch.replicas], law=law)
            self.lattices.append(lat)
        self.outs: List[Optional[torch.Tensor]] = [None] * len(self.lattices)

    def events_per_schedule(self) -> int:
        return sum(lat.events_per_schedule() for lat in self.lattices)

    def enable_grad(self, enable: bool = True):
        for lat in self.lattices:
            lat.enable_grad(enable)

    def _alloc_obs(self, n_sched: int, obs_every: int):
        for i, lat in enumerate(self.lattices):
            if obs_every > 0 and n_sched // obs_every > 0:
                width = 6 if lat.grad_enabled else 4
                shape = (n_sched // obs_every, lat.n_replicas, width)
                o = self.outs[i]
                if o is None or tuple(o.shape) != shape:
                    self.outs[i] = torch.empty(shape, dtype=torch.float64, device=lat.spins.device)
            else:
                self.outs[i] = None

    def step(self, n_sched: int, obs_every: int = 0, reset: Optional[int] = None):
        """Enqueue (optionally reset and) n_sched schedules on every group,
        concurrently; the current stream waits for all of them.  Returns the
        per-group observation buffers (reused between calls)."""
        main = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(main)
        for lat, st, o in zip(self.lattices, self.streams, self.outs):
            st.wait_event(start)
            with torch.cuda.stream(st):
                if reset is not None:
                    lat.reset(reset)
                lat.run(n_sched, obs_every=obs_every, out=o)
                ev = torch.cuda.Event()
                ev.record(st)
            main.wait_event(ev)
        return self.outs

    def run(self, n_sched: int, obs_every: int = 0, reset: Optional[int] = None):
        self._alloc_obs(n_sched, obs_every)
        return self.step(n_sched, obs_every, reset)

    def capture(self, n_sched: int, obs_every: int = 0, reset: int = KMC_INIT_RANDOM) -> "BatchGraph":
        """One CUDA graph for a whole batch step (reset, then n_sched
        schedules on every group).  Buffers are sized by an eager step first;
        replaying the graph repeats the same trajectories from the reset."""
        self.run(n_sched, obs_every, reset)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cap):
            with torch.cuda.graph(g, stream=cap):
                self.step(n_sched, obs_every, reset)
        torch.cuda.current_stream().wait_stream(cap)
        return BatchGraph(g, "kmc batch step: %d replicas in %d groups, %d schedules"
                          % (sum(len(l.L) for l in self.lattices), len(self.lattices), n_sched))

    def sync(self):
        for lat, st in zip(self.lattices, self.streams):
            with torch.cuda.stream(st):
                lat.sync()

    def close(self):
        for lat in self.lattices:
            lat.close()
        self.lattices = []


class BatchGraph:
    """A captured batch step; each replay is one NVTX range (Nsight Systems)."""

    def __init__(self, graph: torch.cuda.CUDAGraph, name: str):
        self.graph = graph
        self.name = name

    def replay(self):
        torch.cuda.nvtx.range_push(self.name)
        try:
            self.graph.replay()
        finally:
            torch.cuda.nvtx.range_pop()


__all__ = ["DOMAIN_SIDES", "Batch", "GroupChoice", "Trial", "max_domain_side", "measure", "plan_candidates",
           "tune_batch", "tune_plan", "KMC_INIT_PER_REPLICA", "BatchGraph"]
