"""The thread-per-domain plan at L_d = 16 and 32 (KMC_LAUNCH_THREADS): one
thread runs a whole domain process (Sec. 2.2) with the domain's rows and
class counts in shared memory.  Checked against the oracle element by
element, as the warp plans are: spins, per-domain real-event counts and event
hashes bit-exact, e, m, e*m bit-exact, clocks to 1e-12; and against a warp
plan on the same seeds."""
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


@pytest.mark.parametrize("Ld", [16, 32])
def test_plan_one_domain_per_thread(Ld):
    import paper_1403_4674_gb300 as kmc
    lat = kmc.Lattice([4 * Ld, 8 * Ld], Ld, 4, [1, 2])
    for wpb in (1, 2, 4):
        lat.set_launch(THREADS, 0, wpb)
        mode, _, ctas, w, smem = lat.launch()
        assert mode == THREADS and w == wpb
        # 16 + 64 domains: 4 + 16 per colour, one warp per colour for each replica's part
        assert ctas * wpb >= 4 and smem > 0
    with pytest.raises(kmc.KmcError):
        lat.set_launch(THREADS, 0, 5)
    lat.close()


@pytest.mark.parametrize("Ld", [16, 32])
@pytest.mark.parametrize("k", [1, 5, 16, 40])
@pytest.mark.parametrize("time_mode", [0, 1])
def test_parity_steps_and_clocks(Ld, k, time_mode):
    """k past 32 and fused same-colour phases; exponential and expected
    clocks; partly filled warps (the smaller replicas have fewer than 32
    domains of a colour)."""
    L = [2 * Ld, 4 * Ld, 6 * Ld]
    gpu, ref = run_both(L, Ld, k, [11, 12, 13], [0.45, 0.3, 0.6], [0.0, 0.05, -0.1], 4,
                        time_mode=time_mode, obs_every=1, launch=(THREADS, 0, 4))
    assert_parity(gpu, ref, 3)


@pytest.mark.parametrize("Ld", [16, 32])
@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
@pytest.mark.parametrize("schedule", [0, 1])
def test_laws_and_schedules(Ld, law, schedule):
    gpu, ref = run_both([4 * Ld], Ld, 3, [7], [0.44], [0.02], 5, law=law, schedule=schedule, obs_every=2,
                        launch=(THREADS, 0, 2))
    assert_parity(gpu, ref, 1)


@pytest.mark.parametrize("Ld", [16, 32])
@pytest.mark.parametrize("every", [1, 3])
def test_colour_pass_records(Ld, every):
    gpu, ref = run_both([4 * Ld, 2 * Ld], Ld, 4, [5, 6], [0.4, 0.5], [0.0, 0.03], 3, obs_every=every,
                        obs_per_pass=True, launch=(THREADS, 0, 1))
    assert_parity(gpu, ref, 2)


@pytest.mark.parametrize("Ld", [16, 32])
def test_extreme_temperatures(Ld):
    """beta = 0 (every step a real event for Metropolis) and a cold all-up
    start at beta = 4.5 (almost every step null; the rows hold one class)."""
    gpu, ref = run_both([4 * Ld, 4 * Ld], Ld, 16, [21, 22], [0.0, 4.5], [0.0, 0.0], 3, init=[0, 1],
                        obs_every=1, launch=(THREADS, 0, 4))
    assert_parity(gpu, ref, 2)


def test_uneven_batch_per_replica_k_and_start():
    """Replicas of several sizes in one context, per-replica k and start,
    resumed across calls (a warp may hold domains of two replicas)."""
    L = [32, 64, 96, 128, 160, 192, 256, 64]
    seeds = [int(s) for s in np.random.default_rng(9).integers(1, 2**62, size=len(L))]
    beta = list(np.linspace(1 / 3.5, 1 / 1.5, len(L)))
    h = list(np.linspace(-0.1, 0.1, len(L)))
    ks = [1, 4, 16, 2, 8, 3, 16, 5]
    inits = [0, 1, 0, 1, 0, 1, 0, 1]
    gpu, ref = run_both(L, 16, ks, seeds, beta, h, 6, init=inits, obs_every=2, chunks=[2, 3, 1],
                        launch=(THREADS, 0, 3))
    assert_parity(gpu, ref, len(L))


@pytest.mark.parametrize("Ld", [16, 32])
def test_thread_and_warp_plans_agree(Ld):
    """Same seeds under the thread plan and a warp grid plan: identical
    trajectories and records, clocks to 1e-12 (they multiply the clock
    variates in a different order)."""
    import paper_1403_4674_gb300 as kmc
    L, seeds = [4 * Ld, 8 * Ld, 16 * Ld], [31, 32, 33]
    out = []
    for plan in ((THREADS, 0, 4), (2, 152, 8)):
        lat = kmc.Lattice(L, Ld, 16, seeds)
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


def test_runs_beyond_the_thread_kernel_take_a_warp_plan():
    import paper_1403_4674_gb300 as kmc
    lat = kmc.Lattice([64], 32, 4, [3])
    lat.set_launch(THREADS, 0, 4)
    lat.set_rates([0.4], [0.0])
    lat.enable_grad(True)
    ref = orc.Replica(L=64, Ld=32, k=4, seed=3, beta=0.4)
    ref.enable_score()
    lat.run(3)
    ref.run(3)
    assert lat.launch()[0] != THREADS
    np.testing.assert_allclose(lat.score().cpu().numpy()[0], ref.score.sum(axis=0), rtol=1e-12, atol=1e-12)
    assert np.array_equal(lat.replica_spins(0).cpu().numpy(), ref.spins)
    lat.close()


def test_bounded_waits_give_up_and_context_survives():
    """Waits for neighbour visits that never come end in KMC_ETIMEOUT."""
    import paper_1403_4674_gb300 as kmc
    lat = kmc.Lattice([128], 32, 2, [5])
    lat.set_launch(THREADS, 0, 4)
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
    ref = orc.Replica(L=128, Ld=32, k=2, seed=5, beta=0.4)
    ref.run(3)
    assert np.array_equal(lat.replica_spins(0).cpu().numpy(), ref.spins)
    lat.close()
