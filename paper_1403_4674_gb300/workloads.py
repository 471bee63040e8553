"""Seeded synthetic workloads (shapes and parameters only, no kMC arithmetic).

Both the CUDA path and the CPU oracle take their inputs from here: lattice
sides, temperatures, fields and per-replica seeds.  The method's own random
numbers (Philox4x32-10 keyed by the replica seed) are drawn inside each
implementation.  The paper's workloads are Ising lattices it builds itself
(Sec. 3); there is no external dataset.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Workload:
    name: str
    L: List[int]
    L_d: int
    k: int
    beta: List[float]
    h: List[float]
    seeds: List[int]
    init: int = 0            # 0 random, 1 all up
    schedules: int = 1
    obs_every: int = 0
    J: float = 1.0
    nu: float = 1.0
    law: int = 0             # Metropolis
    note: str = ""
    ks: Optional[List[int]] = None     # per-replica k (default: k for all)
    inits: Optional[List[int]] = None  # per-replica start (default: init for all)

    def k_of(self, r: int) -> int:
        return self.ks[r] if self.ks is not None else self.k

    def init_of(self, r: int) -> int:
        return self.inits[r] if self.inits is not None else self.init

    @property
    def sites(self) -> int:
        return int(sum(x * x for x in self.L))

    def steps_per_schedule(self) -> int:
        """Uniformised steps of one palindromic schedule (two visits per domain)."""
        return int(sum(2 * (x // self.L_d) ** 2 * self.k_of(r) for r, x in enumerate(self.L)))


def replica_seeds(master: int, n: int) -> List[int]:
    rng = np.random.default_rng(master)
    return [int(s) for s in rng.integers(1, 2**63 - 1, size=n, dtype=np.int64)]


def small_64(seed: int = 1) -> Workload:
    """64x64, J=1, h=0, T=2.5, L_d=16, k=1, palindrome, 1000 schedules."""
    return Workload("ising64_T2.5_Ld16_k1", [64], 16, 1, [1 / 2.5], [0.0], [seed],
                    schedules=1000, note="64^2 periodic, random +-1 start")


def lattice_1024(T: float, k: int, init: int = 0, seed: int = 7) -> Workload:
    """1024x1024, L_d=32, k in {1,4,16}, T in {1.5, 2.269, 3.0}, obs every 10 schedules."""
    return Workload("ising1024_T%g_k%d_%s" % (T, k, "up" if init else "rand"), [1024], 32, k,
                    [1 / T], [0.0], [seed], init=init, schedules=10000, obs_every=10)


def batch_1024(k: int, seed_master: int = 1024) -> Workload:
    """The six 1024^2 lattices of one k: T in {1.5, 2.269, 3.0} x {random, all-up} as one batch.

    Random-start and all-up replicas differ only in the initial state; they are
    run as two batches (init is per call), each of three temperatures.
    """
    Ts = [1.5, 2.269, 3.0]
    seeds = replica_seeds(seed_master + k, 3)
    return Workload("ising1024x3_k%d" % k, [1024] * 3, 32, k, [1 / T for T in Ts], [0.0] * 3, seeds,
                    schedules=10000, obs_every=10)


def ising1024_all(seed_master: int = 1024) -> Workload:
    """Every 1024^2 trajectory of the T x start x k grid as one batch of 18
    replicas: T in {1.5, 2.269, 3.0}, random and all-up starts, k in {1, 4, 16},
    1e4 palindromic schedules, observables every 10 schedules."""
    Ts = [1.5, 2.269, 3.0]
    L, ks, inits, beta, seeds = [], [], [], [], []
    for k in (1, 4, 16):
        sk = replica_seeds(seed_master + k, 3)
        for init in (0, 1):
            for T, sd in zip(Ts, sk):
                L.append(1024)
                ks.append(k)
                inits.append(init)
                beta.append(1 / T)
                seeds.append(sd)
    return Workload("ising1024x18", L, 32, 1, beta, [0.0] * len(L), seeds, schedules=10000, obs_every=10,
                    ks=ks, inits=inits)


def lattice_8192(seed: int = 8192) -> Workload:
    """8192x8192 (67M sites), T=2.269, h=0.01, L_d=64, k=8, 2000 schedules."""
    return Workload("ising8192_T2.269_h0.01_Ld64_k8", [8192], 64, 8, [1 / 2.269], [0.01], [seed],
                    schedules=2000)


def batched_replicas(n: int = 512, master: int = 512, L_d: int = 8, k: int = 8) -> Workload:
    """n replicas, L = 16*round(exp(U[ln 32, ln 512])/16), T ~ U[1.5, 3.5], h ~ U[-0.1, 0.1]."""
    rng = np.random.default_rng(master)
    L = (16 * np.round(np.exp(rng.uniform(np.log(32), np.log(512), size=n)) / 16)).astype(int)
    L = np.maximum(L, 2 * L_d)
    T = rng.uniform(1.5, 3.5, size=n)
    h = rng.uniform(-0.1, 0.1, size=n)
    return Workload("batched%d" % n, [int(x) for x in L], L_d, k, [float(1 / t) for t in T],
                    [float(x) for x in h], replica_seeds(master + 1, n))


def grad_replicas(n: int = 256, seed_master: int = 256, k: int = 8) -> Workload:
    """n replicas of 256x256 at T=2.4, h=0.02 for likelihood-ratio gradients."""
    return Workload("grad%dx256" % n, [256] * n, 32, k, [1 / 2.4] * n, [0.02] * n,
                    replica_seeds(seed_master, n), schedules=5000)
