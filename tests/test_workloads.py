"""The seeded synthetic workloads match their stated recipes (host only).

They hold shapes, temperatures, fields and seeds and none of the method's
arithmetic; the benchmark and the GPU tests build their inputs from them."""
import numpy as np

from paper_1403_4674_gb300 import workloads as wl


def test_ising1024_grid_of_trajectories():
    w = wl.ising1024_all()
    assert w.L == [1024] * 18 and w.L_d == 32 and w.schedules == 10000 and w.obs_every == 10
    combos = {(w.k_of(r), w.init_of(r), round(1 / w.beta[r], 3)) for r in range(18)}
    assert combos == {(k, i, T) for k in (1, 4, 16) for i in (0, 1) for T in (1.5, 2.269, 3.0)}
    assert all(h == 0.0 for h in w.h)
    # the random and all-up trajectories of one (k, T) share a seed; the k differ
    assert len(set(w.seeds)) == 9
    # uniformised steps per schedule: two visits of k steps per domain
    assert w.steps_per_schedule() == 2 * 1024 * 6 * (1 + 4 + 16)
    assert w.steps_per_schedule() * w.schedules == 2580480000


def test_batched_replicas_recipe():
    w = wl.batched_replicas()
    L = np.array(w.L)
    assert len(L) == 512 and np.all(L % 16 == 0) and L.min() >= 32 and L.max() <= 512
    T = 1 / np.array(w.beta)
    assert T.min() >= 1.5 and T.max() <= 3.5
    assert min(w.h) >= -0.1 and max(w.h) <= 0.1
    assert len(set(w.seeds)) == 512
    # log-uniform sides: the median side is near the geometric mean sqrt(32 * 512) = 128
    assert 100 <= np.median(L) <= 160
    # deterministic from the master seed, different for another master
    assert wl.batched_replicas().L == w.L and wl.batched_replicas(master=7).L != w.L


def test_other_workloads():
    g = wl.grad_replicas()
    assert g.L == [256] * 256 and g.schedules == 5000 and g.k == 8
    assert np.allclose(1 / np.array(g.beta), 2.4) and np.allclose(g.h, 0.02)
    b = wl.lattice_8192()
    assert b.L == [8192] and b.L_d == 64 and b.k == 8 and b.h == [0.01] and b.schedules == 2000
    s = wl.small_64()
    assert s.L == [64] and s.L_d == 16 and s.k == 1 and s.schedules == 1000
    seeds = wl.replica_seeds(5, 100)
    assert seeds == wl.replica_seeds(5, 100) and len(set(seeds)) == 100 and all(0 < x < 2 ** 63 for x in seeds)
