"""Parity in the launch configurations the benchmark times: the workloads'
own contexts, plans and parameters, a few schedules, against the oracle (all
replicas where the oracle is quick, a seeded sample otherwise)."""
import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sm():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def _check(spins_of, obs, idx, n, L, Ld, ks, seeds, beta, h, inits, scores=None, obs_every=1):
    """spins_of(r) -> device spins of replica r; obs[rec, r, :]; idx: replicas to check."""
    for r in idx:
        ref = orc.Replica(L=L[r], Ld=Ld, k=ks[r], seed=seeds[r], beta=beta[r], h=h[r], init=inits[r])
        if scores is not None:
            ref.enable_score()
        robs = ref.run(n, obs_every=obs_every)
        assert np.array_equal(spins_of(r), ref.spins), "replica %d: spins differ" % r
        assert np.array_equal(obs[:, r, :3], robs[:, :3]), "replica %d: e, m, e*m differ" % r
        np.testing.assert_allclose(obs[:, r, 3], robs[:, 3], rtol=1e-12, atol=0)
        if scores is not None:
            np.testing.assert_allclose(scores[r], ref.score.sum(axis=0), rtol=1e-12, atol=1e-12)
            if obs.shape[2] >= 6:
                np.testing.assert_allclose(obs[:, r, 4:6], robs[:, 4:6], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("plan", ["grid_5x4", "grid_2x10", "grid_3x8", "grid_1x16", "cluster_16", "threads_1",
                                  "threads_rr_1", "threads_rr_4"])
def test_ising1024_all_replicas(plan):
    """The 18 replicas of 1024^2 (T x start x k) in one context and launch,
    per-replica k and start, profiling on, as the benchmark runs them."""
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    w = wl.ising1024_all()
    n = len(w.L)
    ks = [w.k_of(r) for r in range(n)]
    inits = [w.init_of(r) for r in range(n)]
    lat = kmc.Lattice(w.L, w.L_d, ks[0], w.seeds, init=inits[0])
    lat.set_replica_params(k=ks, init=inits)
    lat.reset(kmc.KMC_INIT_PER_REPLICA)
    lat.set_rates(w.beta, w.h)
    sm = _sm()
    lat.set_launch(*{"grid_5x4": (2, 5 * sm, 4), "grid_2x10": (2, 2 * sm, 10), "grid_3x8": (2, 3 * sm, 8),
                     "grid_1x16": (2, sm, 16), "cluster_16": (1, 16, 16), "threads_1": (3, 1, 1),
                     "threads_rr_1": (3, 2, 1), "threads_rr_4": (3, 2, 4)}[plan])
    lat.profile(True)
    obs = lat.run(3, obs_every=1).cpu().numpy()
    lat.sync()
    _check(lambda r: lat.replica_spins(r).cpu().numpy(), obs, range(n), 3, w.L, w.L_d, ks, w.seeds, w.beta,
           w.h, inits)
    lat.close()


def test_batched_512_autotuned_graph_sample():
    """The 512 uneven replicas grouped and planned by the autotuner with the
    benchmark's candidates, one CUDA graph per step (reset, then schedules on
    every group concurrently); six replicas of every group checked, the
    largest and smallest among them."""
    import torch
    from paper_1403_4674_gb300 import autotune, workloads as wl
    w = wl.batched_replicas(512, master=512)
    sm = _sm()
    plans = [(0, 0, 16), (1, 4, 16), (1, 16, 16), (1, 16, 8), (2, sm, 16), (2, 2 * sm, 12), (2, 3 * sm, 8)]
    choices = autotune.tune_batch(w.L, w.beta, w.h, w.seeds, k_candidates=(4, 8, 16, 32),
                                  Ld_candidates=(8, 16, 32, 64), plans=plans, trial_schedules=4)
    assert sorted(i for ch in choices for i in ch.replicas) == list(range(len(w.L)))
    batch = autotune.Batch(w.L, w.beta, w.h, w.seeds, choices)
    graph = batch.capture(2, 1, reset=0)
    graph.replay()
    graph.replay()  # a replay repeats the trajectories from the reset
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    for ch, lat, o in zip(choices, batch.lattices, batch.outs):
        Lg = [w.L[i] for i in ch.replicas]
        sub = {int(np.argmax(Lg)), int(np.argmin(Lg))}
        sub |= set(rng.choice(len(Lg), min(4, len(Lg)), replace=False).tolist())
        _check(lambda j: lat.replica_spins(j).cpu().numpy(), o.cpu().numpy(), sorted(sub), 2, Lg, ch.L_d,
               [ch.k] * len(Lg), [w.seeds[i] for i in ch.replicas], [w.beta[i] for i in ch.replicas],
               [w.h[i] for i in ch.replicas], [0] * len(Lg))
    batch.close()


def test_grad_256_replicas_sample():
    """256 x 256^2 with scores, one 16-warp CTA per SM on the grid plan;
    two schedules, eight replicas' spins, records and scores checked."""
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    w = wl.grad_replicas(256, seed_master=256, k=8)
    n = len(w.L)
    lat = kmc.Lattice(w.L, w.L_d, w.k, w.seeds)
    lat.set_rates(w.beta, w.h)
    lat.enable_grad(True)
    lat.set_launch(2, _sm(), 16)
    obs = lat.run(2, obs_every=1).cpu().numpy()
    scores = lat.score().cpu().numpy()
    _check(lambda r: lat.replica_spins(r).cpu().numpy(), obs, [0, 37, 101, 128, 177, 200, 254, 255], 2,
           w.L, w.L_d, [w.k] * n, w.seeds, w.beta, w.h, [0] * n, scores=scores)
    lat.close()


@pytest.mark.parametrize("plan", [(2, 0, 16), (3, 1, 4), (3, 1, 1)])
def test_lattice8192_one_schedule(plan):
    """8192^2 at L_d = 64, k = 8 on the 16-warp grid and on the thread plan:
    one schedule, checked on every site against the oracle (one replica; the
    C oracle runs it in seconds)."""
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    w = wl.lattice_8192()
    lat = kmc.Lattice(w.L, w.L_d, w.k, w.seeds)
    lat.set_rates(w.beta, w.h)
    lat.set_launch(plan[0], plan[1] or _sm(), plan[2])
    assert lat.launch()[0] == plan[0]
    obs = lat.run(1, obs_every=1).cpu().numpy()
    lat.sync()
    _check(lambda r: lat.replica_spins(r).cpu().numpy(), obs, [0], 1, w.L, w.L_d, [w.k], w.seeds, w.beta, w.h,
           [0])
    lat.close()


def test_ising1024_full_timed_length_sampled_replica():
    """The benchmark's timed launch itself: all 18 replicas of 1024^2 in one
    context for the full 1e4 schedules with records every 10, on the plans
    the tuner chooses between (the warp kernel's grid of five CTAs of 4
    warps per SM, and the thread kernel with the replicas dealt round-robin
    over the warps); all 18 replicas' spins and records identical on both;
    replica 2 (k = 1, T = 3.0, random start: the most real events per step)
    checked against the oracle over the whole run (about a minute of CPU)."""
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    w = wl.ising1024_all()
    n = len(w.L)
    ks = [w.k_of(r) for r in range(n)]
    inits = [w.init_of(r) for r in range(n)]
    runs = []
    for plan in ((2, 5 * _sm(), 4), (3, 2, 1)):
        lat = kmc.Lattice(w.L, w.L_d, ks[0], w.seeds, init=inits[0])
        lat.set_replica_params(k=ks, init=inits)
        lat.reset(kmc.KMC_INIT_PER_REPLICA)
        lat.set_rates(w.beta, w.h)
        lat.set_launch(*plan)
        obs = lat.run(w.schedules, obs_every=w.obs_every).cpu().numpy()
        lat.sync()
        assert lat.launch()[0] == plan[0]
        runs.append((lat.spins.cpu().numpy(), obs, lat.replica_spins(2).cpu().numpy()))
        lat.close()
    (s0, o0, r0), (s1, o1, r1) = runs
    assert np.array_equal(s0, s1), "the plans' final spins differ"
    assert np.array_equal(o0[..., :3], o1[..., :3]), "the plans' records differ"
    np.testing.assert_allclose(o0[..., 3], o1[..., 3], rtol=1e-12, atol=0)
    _check(lambda r: r1, o1, [2], w.schedules, w.L, w.L_d, ks, w.seeds, w.beta, w.h, inits, obs_every=w.obs_every)


def _oracle_grad_replica(args):
    """One oracle replica with scores (module level: runs in a spawned worker)."""
    L, Ld, k, seed, beta, h, n = args
    ref = orc.Replica(L=L, Ld=Ld, k=k, seed=seed, beta=beta, h=h)
    ref.enable_score()
    robs = ref.run(n, obs_every=n)
    return ref.spins, robs, ref.score.sum(axis=0)


def test_grad_full_timed_length_sampled_replicas():
    """The gradient benchmark's timed launch at its full length: 256 x 256^2
    with scores, 5000 schedules (5.1e6 steps per replica), one record at the
    end, on both plans the tuner chooses between (the 16-warp grid of the
    warp kernel and the thread kernel, one domain per lane); four replicas'
    spins, records and scores checked against the oracle (run in parallel
    worker processes), the scores to 1e-12 relative."""
    import multiprocessing as mp
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    w = wl.grad_replicas(256, seed_master=256, k=8)
    idx = [0, 1, 2, 131]
    jobs = [(w.L[r], w.L_d, w.k, w.seeds[r], w.beta[r], w.h[r], w.schedules) for r in idx]
    # the oracle workers start before this test's first GPU call, by spawn
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        pending = pool.map_async(_oracle_grad_replica, jobs)
        runs = []
        for plan in ((2, _sm(), 16), (3, 0, 1)):
            lat = kmc.Lattice(w.L, w.L_d, w.k, w.seeds)
            lat.set_rates(w.beta, w.h)
            lat.enable_grad(True)
            lat.set_launch(*plan)
            obs = lat.run(w.schedules, obs_every=w.schedules).cpu().numpy()
            assert lat.launch()[0] == plan[0]
            runs.append((plan, obs, lat.score().cpu().numpy(), [lat.replica_spins(r).cpu().numpy() for r in idx]))
            lat.close()
        results = pending.get()
    for plan, obs, scores, spins in runs:
        for r, sp, (rspins, robs, rscore) in zip(idx, spins, results):
            msg = "plan %s replica %d" % (plan, r)
            assert np.array_equal(sp, rspins), msg + ": spins differ"
            assert np.array_equal(obs[:, r, :3], robs[:, :3]), msg + ": e, m, e*m differ"
            np.testing.assert_allclose(obs[:, r, 3], robs[:, 3], rtol=1e-12, atol=0)
            np.testing.assert_allclose(scores[r], rscore, rtol=1e-12, atol=1e-12, err_msg=msg)
            np.testing.assert_allclose(obs[:, r, 4:6], robs[:, 4:6], rtol=1e-12, atol=1e-12, err_msg=msg)


def test_batched_512_full_step_sample():
    """The batched benchmark's timed step itself: the tuned groups, one CUDA
    graph of reset + 200 schedules with records every 10, replayed; the
    largest, the smallest and one more replica of every group against the
    oracle over the whole step."""
    import torch
    from paper_1403_4674_gb300 import autotune, workloads as wl
    w = wl.batched_replicas(512, master=512)
    sm = _sm()
    plans = [(0, 0, 16), (1, 4, 16), (1, 16, 16), (1, 16, 8), (2, sm, 16), (2, 2 * sm, 12), (2, 3 * sm, 8)]
    choices = autotune.tune_batch(w.L, w.beta, w.h, w.seeds, k_candidates=(4, 8, 16, 32),
                                  Ld_candidates=(8, 16, 32, 64), plans=plans, trial_schedules=20)
    batch = autotune.Batch(w.L, w.beta, w.h, w.seeds, choices)
    graph = batch.capture(200, 10, reset=0)
    graph.replay()
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for ch, lat, o in zip(choices, batch.lattices, batch.outs):
        Lg = [w.L[i] for i in ch.replicas]
        sub = {int(np.argmax(Lg)), int(np.argmin(Lg)), int(rng.integers(len(Lg)))}
        _check(lambda j: lat.replica_spins(j).cpu().numpy(), o.cpu().numpy(), sorted(sub), 200, Lg, ch.L_d,
               [ch.k] * len(Lg), [w.seeds[i] for i in ch.replicas], [w.beta[i] for i in ch.replicas],
               [w.h[i] for i in ch.replicas], [0] * len(Lg), obs_every=10)
    batch.close()


@pytest.mark.parametrize("plan", [(2, 0, 16), (3, 1, 4)])
def test_lattice8192_full_length_properties(plan):
    """The 8192^2 benchmark launch at its full 2000 schedules (too long for
    the oracle), checked by properties that hold at any size: the records,
    built on the device from per-visit changes, equal e and m recomputed from
    the final spins on the host; every domain made exactly 2 k steps per
    schedule; two runs of 1000 schedules reproduce one of 2000 bit for bit."""
    import torch
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    w = wl.lattice_8192()
    L, n = w.L[0], w.schedules
    lat = kmc.Lattice(w.L, w.L_d, w.k, w.seeds)
    lat.set_rates(w.beta, w.h)
    lat.set_launch(plan[0], plan[1] or _sm(), plan[2])
    assert lat.launch()[0] == plan[0]
    obs = lat.run(n, obs_every=n // 2).cpu().numpy()
    s = lat.spins.view(L, L).to(torch.int32)
    bonds = int((s * (torch.roll(s, -1, 1) + torch.roll(s, -1, 0))).sum().item())
    mag = int(s.sum().item())
    N = float(L) * float(L)
    e = (-w.J * float(bonds) - w.h[0] * float(mag)) / N
    m = float(mag) / N
    assert obs[-1, 0, 0] == e and obs[-1, 0, 1] == m and obs[-1, 0, 2] == e * m
    ob = lat.observables()
    assert int(ob["steps"][0]) == (L // w.L_d) ** 2 * 2 * w.k * n
    final = lat.spins.clone()
    lat.reset(kmc.KMC_INIT_RANDOM)
    lat.run(n // 2)
    lat.run(n // 2)
    torch.cuda.synchronize()
    assert torch.equal(final, lat.spins)
    lat.close()
