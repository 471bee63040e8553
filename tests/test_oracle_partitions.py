"""Pins of the oracle's block and vertical-stripe partitions of small 2D
lattices (Sec. 3.2; Fig. 1 caption), including domain sizes that are not
powers of two (the multiply-high step target).

Exact enumeration on 3 x 3 and 4 x 4 lattices (stationarity, detailed
balance, final-state distributions), the textbook random-site kernel for an
unpartitioned 3 x 3 lattice (n_d = 9), the beta = 0 closed form for 36-site
stripes, and the Kaufman finite-lattice energy of 12 x 12 at T = 2.4.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import exact_ising as ex
from oracle import oracle as orc
from oracle.enumerate import PartEnumerator


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


def _state_index(states):
    flat = (states.reshape(len(states), -1) > 0).astype(np.int64)
    return (flat << np.arange(flat.shape[1])).sum(axis=1)


def test_geometry_and_scale():
    assert orc.part_geometry(12, orc.PART_STRIPES, 4, 1) == (3, 0, 3, 12, 1)
    assert orc.part_geometry(12, orc.PART_BLOCKS, 4, 3) == (6, 6, 6, 6, 3)
    assert orc.part_geometry(100, orc.PART_BLOCKS, 16, 6) == (50, 25, 25, 25, 2)
    assert orc.part_geometry(9, orc.PART_STRIPES, 3, 0)[4] == -1  # three stripes: no 2-colouring
    # P = 63 - ceil(log2 n_d), M = n_d 2^P
    assert orc.part_scale(12, orc.PART_STRIPES, 4) == (57, 36 << 57)
    assert orc.part_scale(100, orc.PART_STRIPES, 2) == (50, 5000 << 50)
    assert orc.part_scale(64, orc.PART_BLOCKS, 16) == (55, 1 << 63)
    assert orc.part_schedule(orc.PART_STRIPES, orc.SCHED_PALINDROME, 0, 1, 4) == ([0, 1, 1, 0], False)
    assert orc.part_schedule(orc.PART_BLOCKS, orc.SCHED_PALINDROME, 0, 1, 4) == ([0, 1, 2, 3, 3, 2, 1, 0], False)
    assert orc.part_schedule(orc.PART_BLOCKS, orc.SCHED_FIXED, 0, 1, 1) == ([0], False)
    with pytest.raises(ValueError):
        orc.part_schedule(orc.PART_STRIPES, orc.SCHED_PALINDROME, 0, 1, 3)
    with pytest.raises(ValueError):
        orc.part_schedule(orc.PART_BLOCKS, orc.SCHED_PALINDROME, 0, 1, 9)
    p, isd = orc.part_schedule(orc.PART_STRIPES, orc.SCHED_RANDOM_PERM, 4, 1, 3)
    assert isd and sorted(p) == [0, 1, 2]


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
def test_unpartitioned_3x3_single_step_is_textbook(law):
    """N_D = 1 on 3 x 3 (n_d = 9, not a power of two): one step is the
    random-site kernel with selection probability 1/9 (App. A)."""
    E = PartEnumerator(3, orc.PART_BLOCKS, 1, 1, 0.6, h=0.1, law=law, quantised=False)
    rng = np.random.default_rng(0)
    p = rng.random(E.S)
    p /= p.sum()
    assert np.max(np.abs(E.step(0, p) - E.reference_step(p, law))) < 1e-15


@pytest.mark.parametrize("L,kind,ND", [(4, orc.PART_STRIPES, 2), (4, orc.PART_STRIPES, 4),
                                       (4, orc.PART_BLOCKS, 4)])
def test_colour_schedules_balance(L, kind, ND):
    E = PartEnumerator(L, kind, ND, 3, 0.5, h=0.1)
    phases, _ = orc.part_schedule(kind, orc.SCHED_PALINDROME, 0, 0, ND)
    pal = lambda p: E.schedule(phases, p)
    assert E.stationarity_error(pal) < 1e-13
    assert E.detailed_balance_error(pal) < 1e-13
    fixed_ph, _ = orc.part_schedule(kind, orc.SCHED_FIXED, 0, 0, ND)
    fixed = lambda p: E.schedule(fixed_ph, p)
    assert E.stationarity_error(fixed) < 1e-13
    assert E.detailed_balance_error(fixed) > 1e-4


@pytest.mark.parametrize("L,kind,ND", [(3, orc.PART_STRIPES, 3), (4, orc.PART_STRIPES, 2),
                                       (4, orc.PART_STRIPES, 4)])
def test_random_domain_order_balance(L, kind, ND):
    """The paper's random schedule per sweep: averaged over all N_D! orders it
    keeps pi and detailed balance, also with 3-site stripes (Sec. 2.2)."""
    E = PartEnumerator(L, kind, ND, 2, 0.5, h=0.2)
    assert E.stationarity_error(E.random_perm_schedule) < 1e-13
    assert E.detailed_balance_error(E.random_perm_schedule) < 1e-13


@pytest.mark.parametrize("L,kind,ND,schedule", [(3, orc.PART_STRIPES, 3, orc.SCHED_RANDOM_PERM),
                                                (3, orc.PART_BLOCKS, 1, orc.SCHED_PALINDROME),
                                                (4, orc.PART_STRIPES, 2, orc.SCHED_PALINDROME),
                                                (4, orc.PART_BLOCKS, 4, orc.SCHED_PALINDROME),
                                                (4, orc.PART_STRIPES, 4, orc.SCHED_FIXED)])
def test_final_state_distribution(L, kind, ND, schedule):
    k, beta, n = 2, 0.5, 60000
    E = PartEnumerator(L, kind, ND, k, beta, h=0.1)
    s0 = np.ones((L, L), dtype=np.int8)
    s0[0, 1] = -1
    s0[L - 1, 0] = -1
    p0 = np.zeros(E.S)
    p0[_state_index(s0[None])[0]] = 1.0
    if schedule == orc.SCHED_RANDOM_PERM:
        pe = E.random_perm_schedule(p0)
    else:
        phases, _ = orc.part_schedule(kind, schedule, 0, 0, ND)
        pe = E.schedule(phases, p0)
    out, _, _, _ = orc.part_run_many(s0, np.arange(500, 500 + n), L, kind, ND, k, beta, 1, h=0.1, schedule=schedule)
    cnt = np.bincount(_state_index(out), minlength=E.S)
    assert _chi2_pvalue(cnt, pe) > 1e-5


def test_beta_zero_closed_form_36_site_stripes():
    """beta = 0, Metropolis, 12 x 12 in four 3 x 12 stripes (n_d = 36): every
    step flips a uniform site of the stripe, so from all up <m> after n
    palindromic schedules is (1 - 2/36)^(2 k n)."""
    L, ND, k, n, n_traj = 12, 4, 3, 2, 20000
    out, obs, _, F = orc.part_run_many(np.ones((L, L), dtype=np.int8), np.arange(1, n_traj + 1), L,
                                       orc.PART_STRIPES, ND, k, 0.0, n, law=orc.RATE_METROPOLIS, obs_every=4)
    m = obs[:, -1, 1]
    expect = (1 - 2 / 36) ** (2 * k * n)
    assert abs(m.mean() - expect) < 5 * m.std(ddof=1) / math.sqrt(n_traj)
    assert np.all(F == ND * 2 * k * n)


def test_stripes_12x12_energy_matches_exact():
    """12 x 12 at T = 2.4 in four stripes, N_I = 5, Barker: the long-run mean
    energy against the Kaufman finite lattice (Sec. 3.2, Table 1: -1.2847)."""
    r = orc.Partitioned(L=12, kind=orc.PART_STRIPES, ND=4, k=5, seed=2024, beta=1 / 2.4)
    r.run(200)
    obs = r.run(12000, obs_every=4)
    x = obs[:, 0]
    b = x[: len(x) // 20 * 20].reshape(20, -1).mean(axis=1)
    se = b.std(ddof=1) / math.sqrt(20)
    assert abs(b.mean() - ex.kaufman_energy(12, 2.4)) < 5 * se, (b.mean(), se)


def test_partitioned_resume_is_bit_exact():
    a = orc.Partitioned(L=12, kind=orc.PART_STRIPES, ND=2, k=4, seed=9, beta=0.4)
    b = orc.Partitioned(L=12, kind=orc.PART_STRIPES, ND=2, k=4, seed=9, beta=0.4)
    oa = a.run(9, obs_every=2)
    ob = np.concatenate([b.run(4, obs_every=2), b.run(5, obs_every=2)])
    assert np.array_equal(a.spins, b.spins) and a.hash == b.hash and a.flips == b.flips
    np.testing.assert_array_equal(oa[:, :3], ob[:, :3])
