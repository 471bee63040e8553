"""Statistical and structural pins of the oracle's sampler.

The sampler (class counts, cumulative fixed-point rates, member selection,
frozen halo) is checked against the exactly enumerated chain of the same
parameters, against the beta = 0 closed form, and against the clock's
Erlang law (Sec. 2.1, Eq. 2).
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as orc
from oracle.enumerate import Enumerator
from oracle.exact_ising import lattice_energy_all_states

PAL = [0, 1, 2, 3, 3, 2, 1, 0]


def _state_index(states):
    flat = (states.reshape(len(states), -1) > 0).astype(np.int64)
    return (flat << np.arange(flat.shape[1])).sum(axis=1)


def _chi2_pvalue(counts, probs, min_expected=5.0):
    n = counts.sum()
    exp = probs * n
    keep = exp >= min_expected
    obs_k = np.append(counts[keep], counts[~keep].sum())
    exp_k = np.append(exp[keep], exp[~keep].sum())
    if exp_k[-1] < min_expected:
        obs_k[-2] += obs_k[-1]
        exp_k[-2] += exp_k[-1]
        obs_k, exp_k = obs_k[:-1], exp_k[:-1]
    chi2 = ((obs_k - exp_k) ** 2 / exp_k).sum()
    return stats.chi2.sf(chi2, len(obs_k) - 1)


@pytest.mark.parametrize("schedule,colours", [(orc.SCHED_PALINDROME, PAL),
                                              (orc.SCHED_FIXED, [0, 1, 2, 3])])
@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
def test_2x2_final_state_distribution(schedule, colours, law):
    beta, h, k = 0.5, 0.3, 2
    E = Enumerator(2, 1, k, beta=beta, h=h, law=law)
    s0 = np.ones((2, 2), dtype=np.int8)
    s0[0, 1] = -1
    _, A = orc.rate_table(1.0, beta, h, law, 0)
    fs = orc.sample_final_states(s0, 1, k, A, 77, 100000, 1, schedule)
    p0 = np.zeros(E.S)
    p0[_state_index(s0[None])[0]] = 1.0
    pe = E.schedule(colours, p0)
    cnt = np.bincount(_state_index(fs), minlength=E.S)
    assert _chi2_pvalue(cnt, pe) > 1e-5


def test_2x2_random_permutation_schedule_distribution():
    beta, h, k = 0.5, 0.3, 2
    E = Enumerator(2, 1, k, beta=beta, h=h)
    s0 = np.ones((2, 2), dtype=np.int8)
    _, A = orc.rate_table(1.0, beta, h, orc.RATE_METROPOLIS, 0)
    fs = orc.sample_final_states(s0, 1, k, A, 1234, 100000, 1, orc.SCHED_RANDOM_PERM)
    p0 = np.zeros(E.S)
    p0[-1] = 1.0
    perms = list(itertools.permutations(range(4)))
    pe = sum(E.schedule(list(pp), p0) for pp in perms) / 24
    cnt = np.bincount(_state_index(fs), minlength=E.S)
    assert _chi2_pvalue(cnt, pe) > 1e-5


def test_4x4_energy_magnetisation_distribution():
    beta, h, k, L, Ld = 0.4, 0.1, 3, 4, 2
    E = Enumerator(L, Ld, k, beta=beta, h=h, law=orc.RATE_BARKER)
    s0 = orc.init_spins(L, orc.INIT_RANDOM, 99)
    _, A = orc.rate_table(1.0, beta, h, orc.RATE_BARKER, 2)
    fs = orc.sample_final_states(s0, Ld, k, A, 5000, 60000, 2)
    p0 = np.zeros(E.S)
    p0[_state_index(s0[None])[0]] = 1.0
    pe = E.schedule(PAL, E.schedule(PAL, p0))
    H, mag = lattice_energy_all_states(L, 1.0, 0.0)
    key_all = (H.astype(np.int64) + 64) * 64 + (mag + 32)
    uniq, inv = np.unique(key_all, return_inverse=True)
    probs = np.bincount(inv, weights=pe, minlength=len(uniq))
    idx = _state_index(fs)
    cnt = np.bincount(inv[idx], minlength=len(uniq))
    assert _chi2_pvalue(cnt, probs) > 1e-5


def test_beta_zero_closed_form():
    """beta = 0: every step flips a uniform site; <m> = (1 - 2/n_d)^(2 k n) from all-up."""
    L, Ld, k, n = 8, 4, 2, 3
    _, A = orc.rate_table(1.0, 0.0, 0.0, orc.RATE_METROPOLIS, 4)
    s0 = np.ones((L, L), dtype=np.int8)
    fs = orc.sample_final_states(s0, Ld, k, A, 42, 6000, n)
    m = fs.reshape(len(fs), -1).mean(axis=1)
    expect = (1 - 2 / (Ld * Ld)) ** (2 * k * n)
    se = m.std(ddof=1) / math.sqrt(len(m))
    assert abs(m.mean() - expect) < 5 * se
    # every step is a real event at beta = 0
    r = orc.Replica(L=L, Ld=Ld, k=k, seed=1, beta=0.0, init=orc.INIT_ALL_UP)
    r.run(n)
    assert int(r.flips.sum()) == int(r.steps.sum()) == (L // Ld) ** 2 * 2 * k * n


def test_exponential_clock_is_erlang():
    r = orc.Replica(L=32, Ld=8, k=8, seed=11, beta=0.5)
    r.run(20, time_mode=orc.TIME_EXPONENTIAL)
    steps = r.steps
    assert np.all(steps == 2 * 8 * 20)
    # esum_d ~ Gamma(steps, 1): standardised mean over the 16 domains ~ N(0, 1)
    z = (r.esum - steps).sum() / math.sqrt(steps.sum())
    assert abs(z) < 5
    assert stats.kstest(r.esum / steps[0], stats.gamma(a=steps[0], scale=1 / steps[0]).cdf).pvalue > 1e-4


def test_expected_clock_is_exact():
    r = orc.Replica(L=16, Ld=4, k=3, seed=5, beta=0.5, nu=1.0)
    r.run(7, time_mode=orc.TIME_EXPECTED)
    t = r.domain_times(orc.TIME_EXPECTED)
    assert np.all(t == 2 * 3 * 7 / 16.0)


def test_schedule_colour_sequences():
    assert orc.schedule_colours(orc.SCHED_PALINDROME, 5, 1) == PAL
    assert orc.schedule_colours(orc.SCHED_FIXED, 5, 1) == [0, 1, 2, 3]
    perms = list(itertools.permutations(range(4)))
    counts = np.zeros(24)
    for n in range(24000):
        p = tuple(orc.schedule_colours(orc.SCHED_RANDOM_PERM, n, 987654321))
        counts[perms.index(p)] += 1
    assert stats.chisquare(counts).pvalue > 1e-5


def test_init_spins():
    up = orc.init_spins(16, orc.INIT_ALL_UP, 3)
    assert np.all(up == 1)
    s = orc.init_spins(256, orc.INIT_RANDOM, 3)
    assert set(np.unique(s)) == {-1, 1}
    frac = (s > 0).mean()
    assert abs(frac - 0.5) < 5 * 0.5 / 256
    assert np.array_equal(s, orc.init_spins(256, orc.INIT_RANDOM, 3))
    assert not np.array_equal(s, orc.init_spins(256, orc.INIT_RANDOM, 4))


def test_energy_function_matches_independent_formula():
    H, mag = lattice_energy_all_states(4, 1.0, 0.0)
    rng = np.random.default_rng(8)
    for idx in rng.integers(0, 1 << 16, size=50):
        s = np.array([1 if (idx >> i) & 1 else -1 for i in range(16)], dtype=np.int8)
        b, m = orc.energy_mag(s.reshape(4, 4))
        assert -b == H[idx] and m == mag[idx]


def test_resume_is_bit_exact():
    a = orc.Replica(L=32, Ld=8, k=4, seed=2024, beta=1 / 2.269, h=0.01)
    b = orc.Replica(L=32, Ld=8, k=4, seed=2024, beta=1 / 2.269, h=0.01)
    a.run(10)
    b.run(4)
    b.run(6)
    assert np.array_equal(a.spins, b.spins)
    assert np.array_equal(a.hash, b.hash)
    assert np.array_equal(a.flips, b.flips)
    assert np.array_equal(a.esum, b.esum)


def test_invalid_domain_counts_rejected():
    with pytest.raises(ValueError):
        orc.Replica(L=24, Ld=8, k=1, seed=1, beta=0.5).run(1)  # 3 domains per side
    with pytest.raises(ValueError):
        orc.Replica(L=12, Ld=6, k=1, seed=1, beta=0.5).run(1)  # n_d = 36 not 2^m


def test_pass_records_contain_schedule_records():
    """Every 8th colour-pass record of a palindromic run is the schedule record."""
    a = orc.Replica(L=16, Ld=4, k=2, seed=3, beta=0.4, h=0.05)
    b = orc.Replica(L=16, Ld=4, k=2, seed=3, beta=0.4, h=0.05)
    per_pass = a.run(5, obs_every=1, obs_per_pass=True)
    per_sched = b.run(5, obs_every=1)
    assert per_pass.shape == (40, 4)
    np.testing.assert_array_equal(per_pass[7::8], per_sched)


def test_register_shifted_endpoints_sample_equilibrium():
    """Sec. 2.3: the end of every colour pass is a valid observation point.
    At equilibrium the mean energy observed after each of the 8 passes of the
    palindrome (also mid-schedule) matches the exact <H>/N of the 4x4 lattice."""
    from oracle.enumerate import Enumerator
    L, Ld, k, beta, h = 4, 2, 3, 0.4, 0.1
    E = Enumerator(L, Ld, k, beta=beta, h=h, quantised=False)
    exact = float(E.pi @ E.H) / (L * L)
    recs = []
    for r in range(32):
        rep = orc.Replica(L=L, Ld=Ld, k=k, seed=5000 + r, beta=beta, h=h)
        rep.run(20)
        recs.append(rep.run(600, obs_every=1, obs_per_pass=True)[:, 0].reshape(600, 8))
    e = np.stack(recs)  # [replica, schedule, pass]
    for p in range(8):
        x = e[:, :, p]
        # batch means over replicas give the error bar
        means = x.mean(axis=1)
        err = means.std(ddof=1) / np.sqrt(len(means))
        assert abs(x.mean() - exact) < 4.5 * err + 1e-3, (p, x.mean(), exact, err)
