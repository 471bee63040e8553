"""Small lattices under block and vertical-stripe partitions (Sec. 3.2) on the
GPU, through the C ABI, against the oracle: final spins, event hashes,
real-flip and step counts and the records bit for bit (the clock to 1e-12
relative), for domain sizes that are and are not powers of two."""
import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run_both(L, kind, ND, k, n_traj, chunks, schedule, time_mode, law, obs_every, J=1.0, nu=1.0, seed=3):
    import torch
    import paper_1403_4674_gb300 as kmc
    rng = np.random.default_rng(seed)
    seeds = [int(x) for x in rng.integers(1, 2 ** 63 - 1, size=n_traj, dtype=np.int64)]
    s0 = np.where(rng.random((n_traj, L, L)) < 0.5, 1, -1).astype(np.int8)
    beta = list(rng.uniform(0.2, 0.9, size=n_traj))
    h = list(rng.uniform(-0.3, 0.3, size=n_traj))
    spins = torch.from_numpy(s0.copy()).cuda()
    g = kmc.Partitioned(L, kind, ND, k, seeds, spins)
    g.set_rates(beta, h, J=J, nu=nu, law=law)
    obs = []
    for c in chunks:
        o = g.run(c, schedule=schedule, time_mode=time_mode, obs_every=obs_every)
        if o is not None:
            obs.append(o.cpu().numpy())
    torch.cuda.synchronize()
    hashes, flips, steps, T = g.state()
    gs = spins.cpu().numpy()
    g.close()
    gobs = np.concatenate(obs) if obs else None
    for i in range(n_traj):
        r = orc.Partitioned(L=L, kind=kind, ND=ND, k=k, seed=seeds[i], beta=beta[i], h=h[i], J=J, nu=nu, law=law,
                            spins=s0[i])
        ro = [r.run(c, schedule=schedule, time_mode=time_mode, obs_every=obs_every) for c in chunks]
        assert np.array_equal(gs[i], r.spins), "trajectory %d: spins differ" % i
        assert int(hashes[i]) == r.hash, "trajectory %d: event hash differs" % i
        assert int(flips[i]) == r.flips and int(steps[i]) == int(r.steps.sum()), "trajectory %d: counts" % i
        np.testing.assert_allclose(T[i], r.clock(time_mode), rtol=1e-12, atol=0)
        if gobs is not None:
            ro = np.concatenate(ro)
            assert np.array_equal(gobs[:, i, :3], ro[:, :3]), "trajectory %d: e, m, e*m differ" % i
            np.testing.assert_allclose(gobs[:, i, 3], ro[:, 3], rtol=1e-12, atol=0)


S, B = orc.PART_STRIPES, orc.PART_BLOCKS
PAL, FIX, PERM = orc.SCHED_PALINDROME, orc.SCHED_FIXED, orc.SCHED_RANDOM_PERM
CASES = [
    # L, partition, N_D, k, schedule, n_traj
    (12, S, 2, 5, PAL, 37),
    (12, S, 4, 10, PAL, 37),
    (12, B, 4, 2, PAL, 37),
    (12, S, 3, 3, PERM, 37),     # odd number of stripes: random domain order only
    (12, B, 9, 2, PERM, 37),     # 3 x 3 blocks of 16 sites
    (12, B, 1, 7, PAL, 21),      # unpartitioned, n_d = 144
    (100, S, 2, 10, PAL, 9),     # n_d = 5000
    (100, S, 4, 5, PERM, 9),
    (100, B, 16, 2, PAL, 9),     # 25 x 25 blocks
    (100, B, 4, 10, FIX, 9),
    (128, S, 1, 40, PAL, 5),     # n_d = 16384, full 128-bit rows
    (64, B, 16, 33, PAL, 9),     # k > 32: two chunks per visit
    (2, S, 2, 3, PAL, 13),
    (33, S, 1, 4, PAL, 9),       # odd L
    (96, S, 32, 6, PERM, 9),     # 3-wide stripes, 32 domains
    (128, S, 64, 2, PERM, 3),    # the most domains: 64 stripes of width 2
]


@pytest.mark.parametrize("L,kind,ND,k,schedule,n_traj", CASES)
@pytest.mark.parametrize("time_mode,law", [(orc.TIME_EXPONENTIAL, orc.RATE_BARKER),
                                           (orc.TIME_EXPECTED, orc.RATE_METROPOLIS)])
def test_partition_parity(L, kind, ND, k, schedule, n_traj, time_mode, law):
    _run_both(L, kind, ND, k, n_traj, [2, 3], schedule, time_mode, law, obs_every=1)


def test_partition_parity_sparse_records_J_nu():
    _run_both(24, S, 4, 6, 17, [4, 5], PAL, orc.TIME_EXPONENTIAL, orc.RATE_BARKER, obs_every=3, J=0.8, nu=1.7)


def test_partition_edge_cases():
    import torch
    import paper_1403_4674_gb300 as kmc
    _run_both(12, S, 2, 0, 5, [2], PAL, orc.TIME_EXPECTED, orc.RATE_BARKER, obs_every=1)  # k = 0
    _run_both(12, S, 2, 3, 1, [3], PAL, orc.TIME_EXPONENTIAL, orc.RATE_BARKER, obs_every=0)  # no records
    with pytest.raises(kmc.KmcError):
        kmc.Partitioned(12, kmc.KMC_PART_STRIPES, 5, 1, [1])          # 12 % 5 != 0
    with pytest.raises(kmc.KmcError):
        kmc.Partitioned(130, kmc.KMC_PART_STRIPES, 2, 1, [1])         # L > 128
    with pytest.raises(kmc.KmcError):
        kmc.Partitioned(12, kmc.KMC_PART_STRIPES, 3, 1, [1]).run(1)   # three stripes, colour schedule
    # a byte that is not +-1 is reported, not silently read
    sp = torch.ones((1, 12, 12), dtype=torch.int8, device="cuda")
    sp[0, 3, 4] = 0
    g = kmc.Partitioned(12, kmc.KMC_PART_STRIPES, 2, 1, [1], sp)
    g.run(1)
    with pytest.raises(kmc.KmcError):
        g.state()
    g.close()


def test_gpu_final_distribution_matches_enumeration():
    """3 x 3 lattice in three 1 x 3 stripes (n_d = 3), the paper's random
    domain order, one sweep from a fixed start: the GPU's final states
    against the exact enumerated distribution (no oracle sampling)."""
    from scipy import stats
    import torch
    import paper_1403_4674_gb300 as kmc
    from oracle.enumerate import PartEnumerator
    n, L = 60000, 3
    s0 = np.ones((L, L), dtype=np.int8)
    s0[0, 1] = -1
    spins = torch.from_numpy(np.repeat(s0[None], n, axis=0)).cuda()
    g = kmc.Partitioned(L, kmc.KMC_PART_STRIPES, 3, 2, list(range(7, 7 + n)), spins)
    g.set_rates([0.5] * n, [0.1] * n)
    g.run(1, schedule=kmc.KMC_SCHEDULE_RANDOM_PERM)
    torch.cuda.synchronize()
    fs = spins.cpu().numpy().reshape(n, -1)
    idx = ((fs > 0).astype(np.int64) << np.arange(L * L)).sum(axis=1)
    E = PartEnumerator(L, orc.PART_STRIPES, 3, 2, 0.5, h=0.1)
    p0 = np.zeros(E.S)
    p0[int(((s0.reshape(-1) > 0).astype(np.int64) << np.arange(L * L)).sum())] = 1.0
    pe = E.random_perm_schedule(p0)
    cnt = np.bincount(idx, minlength=E.S)
    keep = pe * n >= 5
    chi2 = (((cnt[keep] - pe[keep] * n) ** 2) / (pe[keep] * n)).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-5
    g.close()


@pytest.mark.parametrize("L,kind,ND,k,steps_per_traj,n_traj", [(100, S, 2, 1, 160000, 3), (12, S, 4, 5, 16000, 20),
                                                               (100, B, 16, 10, 160000, 2)])
def test_partition_full_bench_length(L, kind, ND, k, steps_per_traj, n_traj):
    """Settings of the 2D benchmark at their full per-step length (S steps per
    trajectory, the random domain order, 64 energy records), from the all-up
    start, every trajectory against the oracle."""
    import torch
    import paper_1403_4674_gb300 as kmc
    seeds = [1000 + 7 * i for i in range(n_traj)]
    g = kmc.Partitioned(L, kind, ND, k, seeds)
    g.set_rates([1 / 2.4] * n_traj, law=kmc.KMC_RATE_BARKER)
    n_sched = steps_per_traj // (ND * k)
    obs_every = max(1, n_sched * ND // 64)
    obs = g.run(n_sched, schedule=kmc.KMC_SCHEDULE_RANDOM_PERM, obs_every=obs_every).cpu().numpy()
    torch.cuda.synchronize()
    hashes, flips, steps, T = g.state()
    spins = g.spins.cpu().numpy()
    for i in range(n_traj):
        r = orc.Partitioned(L=L, kind=kind, ND=ND, k=k, seed=seeds[i], beta=1 / 2.4)
        ro = r.run(n_sched, schedule=orc.SCHED_RANDOM_PERM, obs_every=obs_every)
        assert np.array_equal(spins[i], r.spins) and int(hashes[i]) == r.hash and int(flips[i]) == r.flips
        assert np.array_equal(obs[:, i, :3], ro[:, :3])
        np.testing.assert_allclose(obs[:, i, 3], ro[:, 3], rtol=1e-12, atol=0)
    g.close()
