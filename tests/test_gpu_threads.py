"""The thread-per-domain plan (KMC_LAUNCH_THREADS, 8x8 domains): one thread
runs a whole domain process (Sec. 2.2) in a 64-bit word.  Checked against the
oracle element by element, as the warp plans are: spins, per-domain
real-event counts and event hashes bit-exact, e, m, e*m bit-exact, clocks to
1e-12; and against the warp plans on the same seeds."""
import numpy as np
import pytest

from gpu_helpers import assert_parity, run_both
from oracle import oracle as orc

pytestmark = pytest.mark.gpu

THREADS = 3


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sm():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_default_plans():
    """One thread per domain for every domain side; with scores on, 16x16
    and 32x32 domains keep it (their thread kernel carries scores) and 8x8
    and 64x64 domains take a warp plan."""
    import paper_1403_4674_gb300 as kmc
    for Ld in (8, 16, 32, 64):
        lat = kmc.Lattice([4 * Ld, 2 * Ld], Ld, 4, [1, 2])
        assert lat.launch()[0] == THREADS
        lat.enable_grad(True)
        assert (lat.launch()[0] == THREADS) == (Ld in (16, 32))
        lat.close()
    lat = kmc.Lattice([128], 64, 4, [1])
    lat.set_launch(2, _sm(), 8)
    with pytest.raises(kmc.KmcError):
        lat.set_launch(THREADS, _sm(), 4)  # a CTA count is no domain order: refused, previous plan kept
    assert lat.launch()[0] == 2
    lat.close()


@pytest.mark.parametrize("k", [1, 5, 16, 40])
@pytest.mark.parametrize("time_mode", [0, 1])
def test_parity_steps_and_clocks(k, time_mode):
    """k past 32 and fused same-colour phases; exponential and expected clocks."""
    sm = _sm()
    gpu, ref = run_both([32, 64, 96], 8, k, [11, 12, 13], [0.45, 0.3, 0.6], [0.0, 0.05, -0.1], 4,
                        time_mode=time_mode, obs_every=1, launch=(THREADS, 2 * sm, 4))
    assert_parity(gpu, ref, 3)


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
@pytest.mark.parametrize("schedule", [0, 1])
def test_laws_and_schedules(law, schedule):
    gpu, ref = run_both([64], 8, 3, [7], [0.44], [0.02], 5, law=law, schedule=schedule, obs_every=2,
                        launch=(THREADS, 64, 2))
    assert_parity(gpu, ref, 1)


@pytest.mark.parametrize("every", [1, 3])
def test_colour_pass_records(every):
    """Register-shifted endpoints: a record after every obs_every-th colour pass."""
    gpu, ref = run_both([48, 32], 8, 4, [5, 6], [0.4, 0.5], [0.0, 0.03], 3, obs_every=every, obs_per_pass=True,
                        launch=(THREADS, 16, 1))
    assert_parity(gpu, ref, 2)


def test_uneven_batch_per_replica_k_and_start_few_threads():
    """More domains than threads (each thread visits several domains per
    colour), per-replica k and start, resumed across calls."""
    L = [16, 32, 48, 64, 80, 96, 128, 256]
    seeds = [int(s) for s in np.random.default_rng(9).integers(1, 2**62, size=len(L))]
    beta = list(np.linspace(1 / 3.5, 1 / 1.5, len(L)))
    h = list(np.linspace(-0.1, 0.1, len(L)))
    ks = [1, 4, 16, 2, 8, 3, 16, 5]
    inits = [0, 1, 0, 1, 0, 1, 0, 1]
    gpu, ref = run_both(L, 8, ks, seeds, beta, h, 6, init=inits, obs_every=2, chunks=[2, 3, 1],
                        launch=(THREADS, 3, 1))
    assert_parity(gpu, ref, len(L))


def test_thread_and_warp_plans_agree():
    """Same seeds under the thread plan and a warp grid plan: identical
    trajectories and records, clocks to 1e-12 (they multiply the clock
    variates in a different order)."""
    import paper_1403_4674_gb300 as kmc
    L, seeds = [64, 128, 256], [31, 32, 33]
    out = []
    for plan in ((THREADS, 3 * _sm(), 4), (2, 2 * _sm(), 8)):
        lat = kmc.Lattice(L, 8, 16, seeds)
        lat.set_launch(*plan)
        lat.set_rates([0.42, 0.35, 0.5], [0.0, 0.01, -0.02])
        obs = lat.run(20, obs_every=5).cpu().numpy()
        h, f, t = lat.domain_state()
        out.append((lat.spins.cpu().numpy(), h, f, t, obs))
        lat.close()
    (s0, h0, f0, t0, o0), (s1, h1, f1, t1, o1) = out
    assert np.array_equal(s0, s1) and np.array_equal(h0, h1) and np.array_equal(f0, f1)
    assert np.array_equal(o0[..., :3], o1[..., :3])
    np.testing.assert_allclose(t0, t1, rtol=1e-12, atol=0)
    np.testing.assert_allclose(o0[..., 3], o1[..., 3], rtol=1e-12, atol=0)


@pytest.mark.parametrize("case", ["random_perm", "horizon", "scores"])
def test_runs_beyond_the_thread_kernel_take_a_warp_plan(case):
    """Random colour orders, fixed-time visits and scores run on a warp plan
    the library installs itself; the results stay the oracle's."""
    import paper_1403_4674_gb300 as kmc
    lat = kmc.Lattice([64], 8, 4, [3])
    assert lat.launch()[0] == THREADS
    lat.set_rates([0.4], [0.0])
    ref = orc.Replica(L=64, Ld=8, k=4, seed=3, beta=0.4)
    if case == "random_perm":
        lat.run(3, schedule=kmc.KMC_SCHEDULE_RANDOM_PERM)
        ref.run(3, schedule=orc.SCHED_RANDOM_PERM)
    elif case == "horizon":
        lat.set_horizon(0.05)
        ref.dtau = 0.05
        lat.run(3, time_mode=kmc.KMC_TIME_HORIZON)
        ref.run(3, time_mode=orc.TIME_HORIZON)
    else:
        lat.enable_grad(True)
        ref.enable_score()
        lat.run(3)
        ref.run(3)
        np.testing.assert_allclose(lat.score().cpu().numpy()[0], ref.score.sum(axis=0), rtol=1e-12, atol=1e-12)
    assert lat.launch()[0] != THREADS
    assert np.array_equal(lat.replica_spins(0).cpu().numpy(), ref.spins)
    lat.close()


def test_bounded_waits_give_up_and_context_survives():
    """Waits for neighbour visits that never come end in KMC_ETIMEOUT."""
    import paper_1403_4674_gb300 as kmc
    lat = kmc.Lattice([128], 8, 2, [5])
    lat.set_launch(THREADS, 8, 2)
    kmc.kmc_debug_barrier(lat.ctx, 1, 20_000_000)  # 20 ms
    lat.run(3)
    with pytest.raises(kmc.KmcError) as ei:
        lat.sync()
    assert ei.value.status == -5
    kmc.kmc_debug_barrier(lat.ctx, 0, 0)
    lat.reset(kmc.KMC_INIT_RANDOM)
    lat.set_rates([0.4], [0.0])
    lat.run(3)
    lat.sync()
    ref = orc.Replica(L=128, Ld=8, k=2, seed=5, beta=0.4)
    ref.run(3)
    assert np.array_equal(lat.replica_spins(0).cpu().numpy(), ref.spins)
    lat.close()


def test_batched_workload_sample():
    """The 512 uneven replicas of the batched workload at L_d = 8, k = 16 in
    one context on the default (thread) plan: a seeded sample of replicas
    against the oracle, largest and smallest included."""
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    w = wl.batched_replicas(512, master=512)
    lat = kmc.Lattice(w.L, 8, 16, w.seeds)
    assert lat.launch()[0] == THREADS
    lat.set_rates(w.beta, w.h)
    obs = lat.run(3, obs_every=1).cpu().numpy()
    idx = sorted({int(np.argmax(w.L)), int(np.argmin(w.L)), 0, 101, 255, 511})
    for r in idx:
        ref = orc.Replica(L=w.L[r], Ld=8, k=16, seed=w.seeds[r], beta=w.beta[r], h=w.h[r])
        robs = ref.run(3, obs_every=1)
        assert np.array_equal(lat.replica_spins(r).cpu().numpy(), ref.spins), r
        assert np.array_equal(obs[:, r, :3], robs[:, :3]), r
        np.testing.assert_allclose(obs[:, r, 3], robs[:, 3], rtol=1e-12, atol=0)
    lat.close()
