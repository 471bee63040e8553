"""C-ABI behaviour on the GPU: argument errors, device-side errors, the bounded
grid barrier, the detailed-balance check of user rate tables, launch plans."""
import math

import numpy as np
import pytest

from gpu_helpers import assert_parity, run_both
from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _kmc():
    import paper_1403_4674_gb300 as kmc
    return kmc


@pytest.mark.parametrize("L,Ld,k", [([48], 16, 1), ([64], 12, 1), ([64], 16, 0), ([64], 16, 70000),
                                    ([8], 8, 1), ([64, 80], 16, 1)])
def test_invalid_geometry_rejected(L, Ld, k):
    kmc = _kmc()
    with pytest.raises(kmc.KmcError) as ei:
        kmc.Lattice(L, Ld, k, [1] * len(L))
    assert ei.value.status == -1


def test_invalid_run_arguments_rejected():
    kmc = _kmc()
    lat = kmc.Lattice([64], 16, 1, [1])
    for args in [(-1, 0, 0, 0), (1, 7, 0, 0), (1, 0, 5, 0), (1, 0, 0, -3)]:
        with pytest.raises(kmc.KmcError) as ei:
            kmc.kmc_run_schedule(lat.ctx, *args, None)
        assert ei.value.status == -1
    with pytest.raises(kmc.KmcError):
        lat.set_rates([-0.5])
    with pytest.raises(kmc.KmcError):
        lat.set_rates([0.4], nu=0.0)
    with pytest.raises(kmc.KmcError):
        lat.set_launch(kmc.KMC_LAUNCH_CLUSTER, 3, 16)
    lat.close()


def test_spins_that_are_not_pm1_raise_device_error():
    import torch
    kmc = _kmc()
    spins = torch.ones(64 * 64, dtype=torch.int8, device="cuda")
    spins[100] = 0
    lat = kmc.Lattice([64], 16, 1, [1], init=kmc.KMC_INIT_KEEP, spins=spins)
    lat.run(1)
    with pytest.raises(kmc.KmcError) as ei:
        lat.sync()
    assert ei.value.status == -6
    lat.spins.fill_(1)
    lat.run(1)
    lat.sync()  # error word was cleared; the context stays usable
    lat.close()


@pytest.mark.parametrize("plan", [(2, 4, 4), (1, 2, 4), (1, 1, 16)])
def test_bounded_waits_give_up_and_context_survives(plan):
    """Neighbour waits that wait for visits that never come return KMC_ETIMEOUT."""
    kmc = _kmc()
    lat = kmc.Lattice([128], 16, 2, [5])
    lat.set_launch(*plan)
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
    ref = orc.Replica(L=128, Ld=16, k=2, seed=5, beta=0.4)
    ref.run(3)
    assert np.array_equal(lat.replica_spins(0).cpu().numpy(), ref.spins)
    lat.close()


def test_rate_table_detailed_balance_check():
    kmc = _kmc()
    lat = kmc.Lattice([64], 16, 4, [9])
    beta, h = 0.45, 0.1
    a, _ = orc.rate_table(1.0, beta, h, orc.RATE_BARKER, 8)
    bad = a.copy()
    bad[3] *= 1.01
    with pytest.raises(kmc.KmcError) as ei:
        kmc.kmc_set_rate_table(lat.ctx, 1.0, [beta], [h], 1.0, bad)
    assert ei.value.status == -4
    # a balanced user table drives exactly the same chain as the built-in law
    kmc.kmc_set_rate_table(lat.ctx, 1.0, [beta], [h], 1.0, a)
    lat.run(5)
    lat.sync()
    ref = orc.Replica(L=64, Ld=16, k=4, seed=9, beta=beta, h=h, law=orc.RATE_BARKER)
    ref.run(5)
    assert np.array_equal(lat.replica_spins(0).cpu().numpy(), ref.spins)
    lat.close()


def test_rate_table_matches_oracle_fixed_point():
    kmc = _kmc()
    for Ld, log2nd in ((8, 6), (16, 8), (32, 10), (64, 12)):
        lat = kmc.Lattice([2 * Ld], Ld, 1, [1])
        for law in (0, 1):
            lat.set_rates([1 / 2.269], [0.01], law=law)
            a, A = lat.rate_table(0)
            ra, rA = orc.rate_table(1.0, 1 / 2.269, 0.01, law, log2nd)
            assert np.array_equal(A, rA)
            assert np.array_equal(a, ra)
        lat.close()


def test_observables_and_counters():
    kmc = _kmc()
    L, Ld, k, n = 128, 32, 4, 6
    lat = kmc.Lattice([L], Ld, k, [77])
    lat.set_rates([0.5], [0.05])
    lat.run(n)
    ob = lat.observables()
    ref = orc.Replica(L=L, Ld=Ld, k=k, seed=77, beta=0.5, h=0.05)
    ref.run(n)
    e, m, _, T = ref.observables()
    assert ob["e"][0] == e and ob["m"][0] == m
    assert math.isclose(ob["t"][0], T, rel_tol=1e-12)
    assert ob["steps"][0] == 2 * (L // Ld) ** 2 * k * n
    assert ob["flips"][0] == int(ref.flips.sum())
    assert lat.kernel_launches() > 0
    lat.close()


def test_profile_counts_run_kernel_launches():
    kmc = _kmc()
    lat = kmc.Lattice([64], 16, 2, [3])
    lat.profile(True)
    lat.run(4)
    lat.run(4)
    ms, n = lat.profile_read()
    assert n == 2 and ms > 0
    lat.close()


@pytest.mark.parametrize("launch", [(1, 4, 16), (2, 152, 16)])
def test_cuda_graph_replay_matches_eager(launch):
    """reset + run captured in one CUDA graph (cluster launch or cooperative
    launch inside) replays the eager trajectory bit for bit; calls that copy
    from pageable memory or synchronise refuse to run while capturing."""
    import torch
    kmc = _kmc()
    L, seeds = [128, 64], [7, 8]
    lat = kmc.Lattice(L, 16, 4, seeds)
    lat.set_launch(*launch)
    lat.set_rates([0.44, 0.5], [0.0, 0.02])
    obs_eager = lat.run(6, obs_every=2).clone()
    lat.sync()
    spins_eager = lat.spins.clone()
    hash_eager = lat.domain_state()[0]

    out = torch.empty_like(obs_eager)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            lat.reset(kmc.KMC_INIT_RANDOM)
            lat.run(6, obs_every=2, out=out)
            with pytest.raises(kmc.KmcError):
                lat.set_rates([0.1, 0.1], [0.0, 0.0])
    for _ in range(2):
        lat.spins.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(lat.spins, spins_eager)
        # e, m, e*m are integer sums; the clock column sums FP64 domain clocks
        # with atomics, whose order may differ between runs
        assert torch.equal(out[..., :3], obs_eager[..., :3])
        torch.testing.assert_close(out[..., 3], obs_eager[..., 3], rtol=1e-12, atol=0)
    # the context's host counters saw one captured run: resync them eagerly
    lat.reset(kmc.KMC_INIT_RANDOM)
    lat.run(6)
    assert np.array_equal(lat.domain_state()[0], hash_eager)
    lat.close()


def test_enable_grad_replans_when_score_kernels_do_not_fit():
    """Three 8-warp CTAs per SM fit the plain kernels (80 registers) but not
    the score-carrying ones; turning scores on re-plans, results stay exact."""
    import torch
    kmc = _kmc()
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    lat = kmc.Lattice([256, 128], 16, 4, [1, 2])
    lat.set_launch(2, 3 * sm, 8)
    assert lat.launch()[2] == 3 * sm
    lat.enable_grad(True)
    mode, size, ctas, wpb, _ = lat.launch()
    assert ctas * wpb <= 2 * sm * 16
    lat.set_rates([0.4, 0.5], [0.0, 0.01])
    lat.run(3)
    lat.sync()
    for r, (L, seed, beta, h) in enumerate([(256, 1, 0.4, 0.0), (128, 2, 0.5, 0.01)]):
        ref = orc.Replica(L=L, Ld=16, k=4, seed=seed, beta=beta, h=h)
        ref.run(3)
        assert np.array_equal(lat.replica_spins(r).cpu().numpy(), ref.spins)
    lat.close()


def test_automatic_domain_side():
    """L_d = 0: the largest side that divides every lattice into an even
    number of domains per side and gives each colour phase 20 visits per SM,
    else the smallest valid side; the run matches the oracle at that side."""
    import torch
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import workloads as wl
    sm = torch.cuda.get_device_properties(0).multi_processor_count

    def chosen(L):
        lat = kmc.Lattice(L, 0, 1, list(range(1, len(L) + 1)))
        side = lat.L_d
        assert side == kmc.kmc_domain_side(lat.ctx)
        lat.close()
        return side

    def expect(L):
        valid = [c for c in (64, 32, 16, 8) if all(x >= 2 * c and x % (2 * c) == 0 for x in L)]
        for c in valid:
            if sum((x // c) ** 2 for x in L) // 4 >= 20 * sm:
                return c
        return valid[-1]

    for L in ([1024] * 18, [8192], wl.batched_replicas(512, master=512).L, [64], [96, 160]):
        assert chosen(L) == expect(L), L
    # a run at the chosen side is the oracle's run at that side
    L, seeds, beta, h = [96, 160], [5, 6], [0.45, 0.5], [0.0, 0.1]
    lat = kmc.Lattice(L, 0, 3, seeds)
    lat.set_rates(beta, h)
    obs = lat.run(4, obs_every=2).cpu().numpy()
    side = lat.L_d
    assert side == expect(L)
    for r in range(2):
        ref = orc.Replica(L=L[r], Ld=side, k=3, seed=seeds[r], beta=beta[r], h=h[r])
        robs = ref.run(4, obs_every=2)
        assert np.array_equal(lat.replica_spins(r).cpu().numpy(), ref.spins)
        assert np.array_equal(obs[:, r, :3], robs[:, :3])
    lat.close()


def test_lattice_beyond_on_chip_capacity_is_refused():
    """16384^2 (268M sites) at L_d = 64: the bit state plus per-domain slots
    exceed what one GPU's shared memory holds in one launch, and one replica
    cannot be split over cluster waves, so planning refuses it with
    KMC_EINVAL (no partial run); the context is still destroyed cleanly and a
    lattice that fits runs afterwards."""
    import torch
    kmc = _kmc()
    with pytest.raises(kmc.KmcError) as ei:
        lat = kmc.Lattice([16384], 64, 8, [1])
        try:
            lat.set_rates([0.44], [0.0])
            lat.run(1)
        finally:
            lat.close()
    assert ei.value.status == -1
    torch.cuda.empty_cache()
    ok = kmc.Lattice([8192], 64, 8, [1])
    ok.set_rates([0.44], [0.0])
    ok.run(1)
    ok.close()


def test_profile_counts_halo_polls():
    """kmc_profile_polls: zero without profiling; with profiling it counts
    the re-reads of neighbours' edge words, many when every wait runs out;
    reading clears the count."""
    kmc = _kmc()
    lat = kmc.Lattice([256], 16, 4, [5])
    lat.set_rates([0.4], [0.0])
    assert lat.profile_polls() == 0
    lat.profile(True)
    lat.run(4)
    normal = lat.profile_polls()
    assert normal >= 0 and lat.profile_polls() == 0
    kmc.kmc_debug_barrier(lat.ctx, 1, 5_000_000)  # 5 ms
    lat.run(1)
    with pytest.raises(kmc.KmcError):
        lat.sync()
    assert lat.profile_polls() > 1000
    kmc.kmc_debug_barrier(lat.ctx, 0, 0)
    lat.close()
