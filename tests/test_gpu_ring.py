"""The 1D ring (Sec. 3.1) on the GPU, through the C ABI, against the oracle.

Bit-exact: configuration words, event hashes, real-flip and step counts,
the record states and the integer observables of every record, and the
ensemble sums over trajectories; the clock to 1e-12 relative (the device sums
-ln v as one product per trajectory, the oracle per step and domain).
"""
import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu

IC8 = [(1 << i) | (1 << ((i + 1) % 8)) for i in (6, 5, 4, 3, 2, 1, 0, 7)]  # the paper's 8 ICs: a pair of up spins (Sec. 3.1)


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _inputs(n_traj, NS, seed=1):
    rng = np.random.default_rng(seed)
    seeds = [int(x) for x in rng.integers(1, 2 ** 63 - 1, size=n_traj, dtype=np.int64)]
    if NS == 8:
        init = [IC8[i % 8] for i in range(n_traj)]
    else:
        mask = (1 << NS) - 1
        init = [int(x) & mask for x in rng.integers(0, 2 ** 63 - 1, size=n_traj, dtype=np.int64)]
        init = [(x | (x << 31)) & mask for x in init]
    beta = list(rng.uniform(0.2, 1.2, size=n_traj))
    h = list(rng.uniform(-0.3, 0.3, size=n_traj))
    return seeds, init, beta, h


def _run_both(NS, Ld, k, n_traj, chunks, schedule, time_mode, law, obs_every, J=1.0, nu=1.0, seed=1,
              common=False):
    import torch
    import paper_1403_4674_gb300 as kmc
    seeds, init, beta, h = _inputs(n_traj, NS, seed)
    if common:
        beta, h = [0.5] * n_traj, [0.0] * n_traj
    ring = kmc.Ring(NS, Ld, k, seeds, init)
    ring.set_rates(beta, h, J=J, nu=nu, law=law)
    g_obs, g_st, g_ens = [], [], []
    for c in chunks:
        o, s, e = ring.run(c, schedule=schedule, time_mode=time_mode, obs_every=obs_every, states=True,
                           ensemble=True)
        if o is not None:
            g_obs.append(o.cpu().numpy())
            g_st.append(s.cpu().numpy().view(np.uint64))
            g_ens.append(e.cpu().numpy())
    torch.cuda.synchronize()
    words, hashes, flips, steps, T = ring.state()
    ring.close()
    refs = []
    for i in range(n_traj):
        r = orc.Ring(NS=NS, Ld=Ld, k=k, seed=seeds[i], beta=beta[i], h=h[i], J=J, nu=nu, law=law, state=init[i])
        ro, rs = [], []
        for c in chunks:
            o, s = r.run(c, schedule=schedule, time_mode=time_mode, obs_every=obs_every)
            ro.append(o)
            rs.append(s)
        refs.append((r, np.concatenate(ro), np.concatenate(rs)))
    gpu = dict(words=words, hashes=hashes, flips=flips, steps=steps, T=T,
               obs=np.concatenate(g_obs, axis=0) if g_obs else None,
               st=np.concatenate(g_st) if g_st else None, ens=np.concatenate(g_ens) if g_ens else None)
    return gpu, refs, time_mode


def _assert_parity(gpu, refs, time_mode, NS):
    n = len(refs)
    for i, (r, ro, rs) in enumerate(refs):
        assert int(gpu["words"][i]) == r.state, "trajectory %d: configuration differs" % i
        assert int(gpu["hashes"][i]) == r.hash, "trajectory %d: event hash differs" % i
        assert int(gpu["flips"][i]) == r.flips, "trajectory %d: real flips differ" % i
        assert int(gpu["steps"][i]) == int(r.steps.sum()), "trajectory %d: steps differ" % i
        np.testing.assert_allclose(gpu["T"][i], r.clock(time_mode), rtol=1e-12, atol=0)
        if gpu["obs"] is not None:
            assert np.array_equal(gpu["st"][:, i], rs), "trajectory %d: record states differ" % i
            assert np.array_equal(gpu["obs"][:, i, :3], ro[:, :3]), "trajectory %d: e, m, e*m differ" % i
            np.testing.assert_allclose(gpu["obs"][:, i, 3], ro[:, 3], rtol=1e-12, atol=0)
    if gpu["obs"] is not None:
        # ensemble sums from the oracle's record states
        st = np.stack([rs for _, _, rs in refs], axis=1)  # [rec, traj]
        bits = ((st[:, :, None] >> np.arange(NS, dtype=np.uint64)) & np.uint64(1)).astype(np.int64)
        sig = 2 * bits - 1
        mag = sig.sum(axis=2)
        bonds = (sig * np.roll(sig, -1, axis=2)).sum(axis=2)
        want = np.concatenate([np.stack([bonds.sum(1), mag.sum(1), (bonds * mag).sum(1), (mag * mag).sum(1)], 1),
                               bits.sum(axis=1)], axis=1)
        assert np.array_equal(gpu["ens"], want), "ensemble sums differ"


CASES = [
    # N_S, L_d, k, schedule, n_traj
    (8, 8, 5, orc.SCHED_PALINDROME, 300),
    (8, 4, 2, orc.SCHED_PALINDROME, 300),
    (8, 2, 10, orc.SCHED_PALINDROME, 300),
    (8, 1, 1, orc.SCHED_PALINDROME, 300),
    (8, 2, 5, orc.SCHED_RANDOM_PERM, 300),
    (8, 1, 2, orc.SCHED_RANDOM_PERM, 300),
    (8, 2, 3, orc.SCHED_FIXED, 300),
    (2, 1, 4, orc.SCHED_PALINDROME, 130),
    (12, 4, 3, orc.SCHED_RANDOM_PERM, 200),   # N_D = 3
    (40, 8, 6, orc.SCHED_RANDOM_PERM, 200),   # N_D = 5
    (33, 1, 2, orc.SCHED_RANDOM_PERM, 129),   # N_D = 33, odd N_S
    (64, 8, 7, orc.SCHED_PALINDROME, 257),
    (64, 64, 20, orc.SCHED_PALINDROME, 129),
    (64, 4, 3, orc.SCHED_RANDOM_PERM, 129),
    (48, 8, 9, orc.SCHED_PALINDROME, 200),    # N_D = 6
]


@pytest.mark.parametrize("NS,Ld,k,schedule,n_traj", CASES)
@pytest.mark.parametrize("time_mode,law", [(orc.TIME_EXPONENTIAL, orc.RATE_BARKER),
                                           (orc.TIME_EXPECTED, orc.RATE_METROPOLIS)])
def test_ring_parity(NS, Ld, k, schedule, n_traj, time_mode, law):
    gpu, refs, tm = _run_both(NS, Ld, k, n_traj, [3, 4], schedule, time_mode, law, obs_every=1)
    _assert_parity(gpu, refs, tm, NS)


def test_ring_parity_sparse_records_and_nu():
    gpu, refs, tm = _run_both(16, 4, 4, 500, [5, 7], orc.SCHED_PALINDROME, orc.TIME_EXPONENTIAL, orc.RATE_BARKER,
                              obs_every=3, J=0.7, nu=2.5)
    _assert_parity(gpu, refs, tm, 16)


def test_ring_edge_cases():
    import torch
    import paper_1403_4674_gb300 as kmc
    # k = 0: no steps, records of the untouched start
    gpu, refs, tm = _run_both(8, 2, 0, 40, [2], orc.SCHED_PALINDROME, orc.TIME_EXPECTED, orc.RATE_BARKER, 1)
    _assert_parity(gpu, refs, tm, 8)
    assert np.all(gpu["flips"] == 0) and np.all(gpu["steps"] == 0)
    # one trajectory
    gpu, refs, tm = _run_both(8, 4, 3, 1, [4], orc.SCHED_PALINDROME, orc.TIME_EXPONENTIAL, orc.RATE_BARKER, 2)
    _assert_parity(gpu, refs, tm, 8)
    # no schedules, and fewer passes than obs_every: no records, state unchanged
    ring = kmc.Ring(8, 2, 3, [5], [IC8[0]])
    o, s, e = ring.run(0, obs_every=1, states=True, ensemble=True)
    assert o is None and s is None and e is None
    o, s, e = ring.run(1, obs_every=5, states=True, ensemble=True)
    assert o is None
    words, _, _, steps, _ = ring.state()
    r = orc.Ring(NS=8, Ld=2, k=3, seed=5, beta=0.5, state=IC8[0])
    r.run(0)
    r.run(1, obs_every=5)
    assert int(words[0]) == r.state and int(steps[0]) == int(r.steps.sum())
    # invalid configurations fail loudly
    with pytest.raises(kmc.KmcError):
        kmc.Ring(12, 4, 1, [1], [0]).run(1)              # N_D = 3 with a colour schedule
    with pytest.raises(kmc.KmcError):
        kmc.Ring(8, 3, 1, [1], [0])                      # L_d not a power of two
    with pytest.raises(kmc.KmcError):
        kmc.Ring(8, 2, 1, [1], [1 << 8])                 # bits beyond N_S
    with pytest.raises(kmc.KmcError):
        kmc.Ring(8, 2, 1, [1], [0]).run(1, time_mode=kmc.KMC_TIME_HORIZON)
    with pytest.raises(kmc.KmcError):
        rr = kmc.Ring(8, 2, 1, [1], [0])
        rr.set_rates([0.5], [0.0], law=7)
    ring.close()
    torch.cuda.synchronize()


def test_ring_paper_setting_bit_exact():
    """Sec. 3.1 setting: 8 ICs x 750 trajectories, beta J = 0.5, h = 0,
    Barker, N_D = 4, N_I = 5, the random domain order per sweep, S = 800
    steps (40 sweeps of 4 processes), a record after every domain process;
    every trajectory checked."""
    import torch
    import paper_1403_4674_gb300 as kmc
    n_traj, NS, Ld, k = 6000, 8, 2, 5
    seeds = [1000003 * i + 17 for i in range(n_traj)]
    init = [IC8[i % 8] for i in range(n_traj)]
    ring = kmc.Ring(NS, Ld, k, seeds, init)
    ring.set_rates([0.5] * n_traj, [0.0] * n_traj, law=kmc.KMC_RATE_BARKER)
    o, s, e = ring.run(40, schedule=kmc.KMC_SCHEDULE_RANDOM_PERM, obs_every=1, states=True, ensemble=True)
    torch.cuda.synchronize()
    S, obs, st, H, F = orc.ring_run_many(init, seeds, NS, Ld, k, 0.5, 40, schedule=orc.SCHED_RANDOM_PERM,
                                         obs_every=1)
    words, hashes, flips, _, _ = ring.state()
    assert np.array_equal(words, S) and np.array_equal(hashes, H) and np.array_equal(flips, F)
    assert np.array_equal(s.cpu().numpy().view(np.uint64), st.T)
    assert np.array_equal(o.cpu().numpy()[:, :, :3], obs.transpose(1, 0, 2)[:, :, :3])
    bits = ((st[:, :, None] >> np.arange(NS, dtype=np.uint64)) & np.uint64(1)).astype(np.int64)
    assert np.array_equal(e.cpu().numpy()[:, 4:], bits.sum(axis=0))
    ring.close()


def test_ring_ensemble_matches_exact_time_dependent_averages():
    """The device's ensemble sums against the exact evolution of p(s) of the
    enumerated ring (no oracle sampling): N_D = 4, N_I = 5, palindrome, from
    the paper's first IC; every (record, spin) mean within a Bonferroni bound."""
    from scipy import stats
    import torch
    import paper_1403_4674_gb300 as kmc
    from oracle.enumerate import RingEnumerator
    NS, Ld, k, n_traj, n_sched = 8, 2, 5, 200000, 5
    ring = kmc.Ring(NS, Ld, k, list(range(1, n_traj + 1)), [IC8[0]] * n_traj)
    ring.set_rates([0.5] * n_traj, [0.0] * n_traj)
    _, _, e = ring.run(n_sched, obs_every=1, records=False, ensemble=True)
    torch.cuda.synchronize()
    ens = e.cpu().numpy()
    E = RingEnumerator(NS, Ld, k, 0.5)
    p = np.zeros(E.S)
    p[IC8[0]] = 1.0
    exact = []
    for _ in range(n_sched):
        for c in [0, 1, 1, 0]:
            p = E.phase(c, p, False)
            exact.append(E.spin_means(p))
    exact = np.array(exact)
    mean = 2.0 * ens[:, 4:] / n_traj - 1.0
    se = np.sqrt(np.maximum(1 - exact ** 2, 1e-12) / n_traj)
    z = np.abs(mean - exact) / se
    assert z.max() < stats.norm.isf(1e-6 / (2 * z.size)), z.max()
    # <H>/N_S from the bond sums against the exact one
    H_exact = []
    p = np.zeros(E.S)
    p[IC8[0]] = 1.0
    for _ in range(n_sched):
        for c in [0, 1, 1, 0]:
            p = E.phase(c, p, False)
            H_exact.append(float(p @ E.bonds))
    b_mean = ens[:, 0] / n_traj
    assert np.all(np.abs(b_mean - np.array(H_exact)) < 6 * 8 / np.sqrt(n_traj))
    ring.close()


def test_ring_million_trajectories_sample():
    """A million trajectories of the paper's ring in one launch; 64 sampled
    trajectories against the oracle and the ensemble sums' totals checked
    against the per-trajectory record states."""
    import torch
    import paper_1403_4674_gb300 as kmc
    n = 1 << 20
    seeds = [(0x9E3779B97F4A7C15 * (i + 1)) & ((1 << 63) - 1) for i in range(n)]
    init = [IC8[i % 8] for i in range(n)]
    ring = kmc.Ring(8, 2, 5, seeds, init)
    ring.set_rates([0.5] * n, [0.0] * n)
    o, s, e = ring.run(10, schedule=kmc.KMC_SCHEDULE_RANDOM_PERM, obs_every=4, states=True, ensemble=True)
    torch.cuda.synchronize()
    st = s.cpu().numpy().view(np.uint64)  # [rec, traj]
    bits = ((st[:, :, None] >> np.arange(8, dtype=np.uint64)) & np.uint64(1)).astype(np.int64)
    assert np.array_equal(e.cpu().numpy()[:, 4:], bits.sum(axis=1))
    words, hashes, _, _, _ = ring.state()
    for i in np.random.default_rng(1).choice(n, 64, replace=False):
        r = orc.Ring(NS=8, Ld=2, k=5, seed=seeds[i], beta=0.5, state=init[i])
        _, rs = r.run(10, schedule=orc.SCHED_RANDOM_PERM, obs_every=4)
        assert int(words[i]) == r.state and int(hashes[i]) == r.hash
        assert np.array_equal(st[:, i], rs)
    ring.close()
