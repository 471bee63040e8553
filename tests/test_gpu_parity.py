"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bit-exact: spins, per-domain real-event counts and event-sequence hashes,
e, m and e*m (integer sums, same FP64 formula and order).  Clocks: 1e-12
relative (the device multiplies 64-bit mantissas where the oracle sums
logarithms, Sec. 2.1; the decision path never reads the clock).
"""
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


def test_init_random_and_all_up_bit_exact():
    import paper_1403_4674_gb300 as kmc
    L = [64, 128, 48 * 2, 256]
    seeds = [1, 2**40 + 3, 77, 2**63 - 5]
    lat = kmc.Lattice(L, 16, 1, seeds, init=kmc.KMC_INIT_RANDOM)
    for r, (Lr, s) in enumerate(zip(L, seeds)):
        assert np.array_equal(lat.replica_spins(r).cpu().numpy(), orc.init_spins(Lr, orc.INIT_RANDOM, s))
    lat.reset(kmc.KMC_INIT_ALL_UP)
    lat.sync()
    assert bool((lat.spins == 1).all())
    lat.close()


def test_config_64_T25_k1_1000_schedules():
    """64^2, T=2.5, h=0, L_d=16, k=1, palindrome, 1000 schedules, FP64 clock."""
    gpu, ref = run_both([64], 16, 1, [1], [1 / 2.5], [0.0], 1000, obs_every=10)
    assert_parity(gpu, ref, 1)
    assert gpu["obs"].shape == (100, 1, 4)


@pytest.mark.parametrize("Ld", [8, 16, 32, 64])
@pytest.mark.parametrize("k", [1, 3, 16, 40])
def test_domain_sizes_and_step_counts(Ld, k):
    L = 4 * Ld
    gpu, ref = run_both([L], Ld, k, [1000 + Ld + k], [1 / 2.269], [0.01], 6, obs_every=2)
    assert_parity(gpu, ref, 1)


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
@pytest.mark.parametrize("time_mode", [orc.TIME_EXPONENTIAL, orc.TIME_EXPECTED])
@pytest.mark.parametrize("schedule", [orc.SCHED_PALINDROME, orc.SCHED_FIXED, orc.SCHED_RANDOM_PERM])
def test_laws_time_modes_schedules(law, time_mode, schedule):
    gpu, ref = run_both([64, 96], 16, 4, [11, 12], [0.5, 0.3], [0.2, -0.1], 9, law=law,
                        time_mode=time_mode, schedule=schedule, obs_every=3, nu=0.75)
    assert_parity(gpu, ref, 2)


def test_uneven_batch_of_replicas():
    L = [32, 48, 64, 80, 96, 128, 160, 256]
    seeds = [int(s) for s in np.random.default_rng(5).integers(1, 2**62, size=len(L))]
    beta = list(np.linspace(1 / 3.5, 1 / 1.5, len(L)))
    h = list(np.linspace(-0.1, 0.1, len(L)))
    gpu, ref = run_both(L, 8, 8, seeds, beta, h, 5, obs_every=1)
    assert_parity(gpu, ref, len(L))


def test_resume_across_calls_is_bit_exact():
    gpu, ref = run_both([128], 32, 4, [99], [0.44], [0.0], 10, obs_every=2, chunks=[3, 5, 2])
    assert_parity(gpu, ref, 1)


def test_degenerate_rates():
    # beta = 0: every step is a real event; beta = 4.5: almost every step is
    # null (a = exp(-36) = 2.3e-16 for the aligned classes, A_c = 8 at
    # L_d = 16, the last beta of that order whose table keeps every A_c >= 1)
    gpu, ref = run_both([64, 64], 16, 8, [3, 4], [0.0, 4.5], [0.0, 0.0], 5, init=orc.INIT_ALL_UP)
    assert_parity(gpu, ref, 2)
    assert gpu["flips"][:16].sum() == 16 * 2 * 8 * 5


def test_tables_rounding_an_acceptance_to_zero_are_refused():
    """Eq. 4: an acceptance that rounds to A_c = 0 would be a one-way rate.
    Every way of setting a table refuses it and keeps the previous one."""
    import math
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300._lib import KMC_ENOTBALANCED
    lat = kmc.Lattice([64], 16, 4, [5])
    lat.set_rates([0.4])
    before = lat.rate_table(0)
    with pytest.raises(kmc.KmcError) as e:
        lat.set_rates([5.0])  # exp(-40) < 2^-56 at P = 55
    assert e.value.status == KMC_ENOTBALANCED and "rounds to 0" in str(e.value)
    with pytest.raises(kmc.KmcError) as e:
        a = np.array([[min(1.0, math.exp(-5.0 * orc.class_dE(c, 1.0, 0.0))) for c in range(10)]])
        kmc.kmc_set_rate_table(lat.ctx, 1.0, [5.0], [0.0], 1.0, a)
    assert e.value.status == KMC_ENOTBALANCED
    after = lat.rate_table(0)
    assert np.array_equal(before[1], after[1])
    lat.set_rates([4.5])
    assert 1e-3 < lat.rate_table_error() < 0.1  # A_c = 8 for a = 2.3e-16 * 2^55 = 8.3
    lat.set_rates([1 / 1.5], [0.1])
    assert lat.rate_table_error() < 1e-12
    lat.close()
    ring = kmc.Ring(8, 2, 5, [1], [3])
    with pytest.raises(kmc.KmcError) as e:
        ring.set_rates([12.0], [0.0])  # ring: largest dE = 4, exp(-48) < 2^-63
    assert e.value.status == KMC_ENOTBALANCED
    ring.close()
    part = kmc.Partitioned(12, kmc.KMC_PART_STRIPES, 4, 5, [1])
    with pytest.raises(kmc.KmcError) as e:
        part.set_rates([6.0])
    assert e.value.status == KMC_ENOTBALANCED
    part.close()


def test_minimum_lattice_two_domains_per_side():
    gpu, ref = run_both([16, 32, 64, 128], 8, 5, [1, 2, 3, 4], [0.4] * 4, [0.05] * 4, 7)
    assert_parity(gpu, ref, 4)
    gpu, ref = run_both([128], 64, 5, [9], [0.4], [0.05], 7)
    assert_parity(gpu, ref, 1)


CLUSTER, GRID = 1, 2


@pytest.mark.parametrize("launch", [(CLUSTER, 1, 16), (CLUSTER, 2, 4), (CLUSTER, 4, 16), (CLUSTER, 16, 1),
                                    (GRID, 1, 1), (GRID, 3, 2), (GRID, 7, 16), (GRID, 152, 16)])
def test_launch_plan_does_not_change_results(launch):
    """CLUSTER (DSMEM halos, cluster barriers) and GRID (L2 halos, grid barrier) plans."""
    gpu, ref = run_both([256], 16, 4, [2024], [0.42], [0.01], 4, obs_every=2, launch=launch)
    assert_parity(gpu, ref, 1)


@pytest.mark.parametrize("launch", [(CLUSTER, 8, 16), (GRID, 152, 16)])
def test_batch_under_both_plans(launch):
    L = [32, 64, 96, 128, 160, 192, 224, 256]
    seeds = list(range(101, 109))
    gpu, ref = run_both(L, 16, 6, seeds, [0.45] * 8, [0.02] * 8, 3, obs_every=1, launch=launch,
                        schedule=orc.SCHED_RANDOM_PERM)
    assert_parity(gpu, ref, len(L))


@pytest.mark.parametrize("k", [1, 4, 16])
def test_config_1024_k(k):
    """1024^2, L_d=32, T=2.269 from random and all-up starts, k in {1,4,16}."""
    for init in (orc.INIT_RANDOM, orc.INIT_ALL_UP):
        gpu, ref = run_both([1024], 32, k, [7 + k], [1 / 2.269], [0.0], 2, init=init, obs_every=1)
        assert_parity(gpu, ref, 1)


def test_config_8192_one_schedule():
    """8192^2 (67M sites), T=2.269, h=0.01, L_d=64, k=8: one full schedule vs the oracle
    (a GRID plan: the bit state is larger than one cluster's shared memory)."""
    gpu, ref = run_both([8192], 64, 8, [8192], [1 / 2.269], [0.01], 1, obs_every=1)
    assert_parity(gpu, ref, 1)


@pytest.mark.parametrize("launch", [None, (CLUSTER, 4, 16), (GRID, 152, 16), (GRID, 5, 4)])
@pytest.mark.parametrize("time_mode", [orc.TIME_EXPONENTIAL, orc.TIME_EXPECTED])
def test_per_replica_steps_and_starts(launch, time_mode):
    """One context, replicas with their own k and start (random, all-up, kept):
    each replica's trajectory is the one the oracle runs for it alone."""
    L = [64, 128, 64, 96, 128, 64]
    ks = [16, 1, 4, 1, 16, 7]
    inits = [orc.INIT_RANDOM, orc.INIT_ALL_UP, orc.INIT_RANDOM, orc.INIT_ALL_UP, orc.INIT_RANDOM, orc.INIT_ALL_UP]
    seeds = [31, 32, 33, 34, 35, 36]
    beta = [1 / 1.5, 1 / 2.269, 1 / 3.0, 1 / 1.5, 1 / 2.269, 1 / 3.0]
    gpu, ref = run_both(L, 16, ks, seeds, beta, [0.0, 0.01, -0.02, 0.0, 0.03, 0.0], 6, init=inits,
                        obs_every=2, launch=launch, time_mode=time_mode)
    assert_parity(gpu, ref, len(L))
    # Eq. 11: steps = visits * k * N_D per replica
    steps = gpu["observables"]["steps"]
    for r in range(len(L)):
        assert steps[r] == 6 * 2 * ks[r] * (L[r] // 16) ** 2


def test_per_replica_keep_leaves_spins():
    import torch
    import paper_1403_4674_gb300 as kmc
    lat = kmc.Lattice([64, 64], 16, 2, [5, 6], init=kmc.KMC_INIT_RANDOM)
    lat.run(3)
    lat.sync()
    before = lat.replica_spins(0).clone()
    lat.set_replica_params(init=[kmc.KMC_INIT_KEEP, kmc.KMC_INIT_ALL_UP])
    lat.reset(kmc.KMC_INIT_PER_REPLICA)
    lat.sync()
    assert torch.equal(lat.replica_spins(0), before)
    assert bool((lat.replica_spins(1) == 1).all())
    # k may change only before the first run after a reset
    lat.set_replica_params(k=[3, 1])
    lat.run(1)
    with pytest.raises(kmc.KmcError):
        lat.set_replica_params(k=[1, 1])
    lat.close()


@pytest.mark.parametrize("launch", [(GRID, 152, 16), (GRID, 5, 4), (GRID, 40, 2), (CLUSTER, 2, 16)])
def test_plans_without_observation_points(launch):
    """No observation point means no replica-wide barrier in the launch: the
    write-back at the end must still wait for every warp's last visit."""
    L = [128, 64, 96]
    gpu, ref = run_both(L, 16, [4, 1, 9], [21, 22, 23], [0.5, 0.4, 0.3], [0.0, 0.02, -0.01], 6, launch=launch)
    assert_parity(gpu, ref, len(L), obs=False)
    gpu, ref = run_both(L, 16, 3, [24, 25, 26], [0.5, 0.4, 0.3], [0.0, 0.02, -0.01], 7,
                        schedule=orc.SCHED_RANDOM_PERM, launch=launch)
    assert_parity(gpu, ref, len(L), obs=False)


@pytest.mark.parametrize("launch", [None, (GRID, 152, 16), (CLUSTER, 4, 8)])
@pytest.mark.parametrize("schedule,time_mode", [(orc.SCHED_PALINDROME, orc.TIME_EXPONENTIAL),
                                                (orc.SCHED_PALINDROME, orc.TIME_EXPECTED),
                                                (orc.SCHED_RANDOM_PERM, orc.TIME_EXPONENTIAL)])
@pytest.mark.parametrize("obs_every", [1, 3])
def test_register_shifted_endpoints(launch, schedule, time_mode, obs_every):
    """Records after colour passes (Sec. 2.3 register-shifted endpoints),
    built on the device from per-visit changes, equal the oracle's full
    recomputation after the same passes."""
    L = [64, 96, 128]
    gpu, ref = run_both(L, 16, [3, 1, 5], [41, 42, 43], [0.5, 0.35, 0.44], [0.03, 0.0, -0.02], 5,
                        obs_every=obs_every, launch=launch, schedule=schedule, time_mode=time_mode,
                        obs_per_pass=True, chunks=[2, 3])
    assert_parity(gpu, ref, len(L))
    passes = 8 if schedule == orc.SCHED_PALINDROME else 4
    assert gpu["obs"].shape[0] == (2 * passes) // obs_every + (3 * passes) // obs_every


@pytest.mark.parametrize("Ld,dtau", [(8, 0.05), (16, 0.02), (32, 0.004), (64, 0.002), (16, 0.3)])
@pytest.mark.parametrize("launch", [None, (GRID, 152, 16)])
def test_fixed_time_visits(Ld, dtau, launch):
    """KMC_TIME_HORIZON: each visit runs its domain for domain time dtau (a
    Poisson number of steps by table inversion); bit-exact against the
    oracle, clock exactly dtau per visit, step counts per replica (Eq. 11)."""
    L = [4 * Ld, 6 * Ld]
    gpu, ref = run_both(L, Ld, 1, [61, 62], [0.45, 0.3], [0.02, -0.03], 5, obs_every=1, launch=launch,
                        time_mode=orc.TIME_HORIZON, dtau=dtau, nu=1.1)
    assert_parity(gpu, ref, len(L))


def test_fixed_time_visits_with_pass_records_and_perm_schedule():
    gpu, ref = run_both([64, 128], 16, 1, [71, 72], [0.5, 0.4], [0.0, 0.01], 4, obs_every=3,
                        time_mode=orc.TIME_HORIZON, dtau=0.05, obs_per_pass=True,
                        schedule=orc.SCHED_RANDOM_PERM, chunks=[1, 3])
    assert_parity(gpu, ref, 2)


def test_fixed_time_steps_and_errors():
    import paper_1403_4674_gb300 as kmc
    lat = kmc.Lattice([64], 16, 1, [5])
    with pytest.raises(kmc.KmcError):
        lat.run(1, time_mode=kmc.KMC_TIME_HORIZON)  # no visit time set
    with pytest.raises(kmc.KmcError):
        lat.set_horizon(10.0)  # n_d nu dtau = 2560 steps per visit: table too long
    lat.set_horizon(0.05)
    lat.run(4, time_mode=kmc.KMC_TIME_HORIZON)
    ob = lat.observables()
    ref = orc.Replica(L=64, Ld=16, k=1, seed=5, beta=0.4, dtau=0.05)
    ref.run(4, time_mode=orc.TIME_HORIZON)
    assert ob["steps"][0] == int(ref.steps.sum())
    assert ob["t"][0] == pytest.approx(8 * 0.05, rel=1e-13)
    lat.close()
