"""Pins of the oracle's likelihood-ratio score (path gradient).

The score of a path is d log P(path) / d theta for theta = (beta, h); the
paper's transition matrices (Sec. 2.2, App. A) make P(path) explicit: each
uniformised step has probability a_c/n_d (real flip of a class-c site) or
1 - R/n_d (null step).  Pinned by: finite differences of the rate table,
E[score] = 0, and E[A * score] against the exact forward-mode derivative
d E[A] / d theta of the enumerated distribution.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from oracle.enumerate import Enumerator
from oracle.exact_ising import lattice_energy_all_states

PAL = [0, 1, 2, 3, 3, 2, 1, 0]


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
@pytest.mark.parametrize("beta,h", [(0.4, 0.1), (1 / 2.4, 0.02), (0.8, -0.3)])
def test_score_table_is_derivative_of_log_rate(law, beta, h):
    g = orc.score_table(1.0, beta, h, law)
    a, _ = orc.rate_table(1.0, beta, h, law, 8)
    assert np.array_equal(g[:10], a)
    d = 1e-6
    for c in range(10):
        if law == orc.RATE_METROPOLIS and orc.class_dE(c, 1.0, h) <= 0:
            assert g[10 + c] == 0 and g[20 + c] == 0
            continue
        fb = (math.log(orc.rate_table(1.0, beta + d, h, law, 8)[0][c])
              - math.log(orc.rate_table(1.0, beta - d, h, law, 8)[0][c])) / (2 * d)
        fh = (math.log(orc.rate_table(1.0, beta, h + d, law, 8)[0][c])
              - math.log(orc.rate_table(1.0, beta, h - d, law, 8)[0][c])) / (2 * d)
        assert g[10 + c] == pytest.approx(fb, rel=1e-7, abs=1e-9)
        assert g[20 + c] == pytest.approx(fh, rel=1e-7, abs=1e-9)


def _indices(states):
    flat = (states.reshape(len(states), -1) > 0).astype(np.int64)
    return (flat << np.arange(flat.shape[1])).sum(axis=1)


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
def test_lr_estimator_matches_exact_derivative(law):
    """E[A S] = d E[A] / d theta on a 2x2 lattice after one palindromic schedule."""
    L, Ld, k, beta, h = 2, 1, 2, 0.5, 0.3
    E = Enumerator(L, Ld, k, beta=beta, h=h, law=law, quantised=False)
    g = orc.score_table(1.0, beta, h, law)
    E.set_score_table(g)
    _, A = orc.rate_table(1.0, beta, h, law, 0)
    s0 = np.ones((L, L), dtype=np.int8)
    s0[0, 1] = -1
    p0 = np.zeros(E.S)
    p0[_indices(s0[None])[0]] = 1.0
    p, (dpb, dph) = E.schedule_deriv(PAL, p0, (np.zeros(E.S), np.zeros(E.S)))
    H, mag = lattice_energy_all_states(L, 1.0, h)
    n = 200000
    fs, score = orc.sample_final_states_with_score(s0, Ld, k, A, g, 31337, n, 1)
    idx = _indices(fs)
    for obs in (H.astype(float), mag.astype(float)):
        exact_b = float(obs @ dpb)
        exact_h = float(obs @ dph)
        a = obs[idx]
        c = a - a.mean()
        for j, exact in ((0, exact_b), (1, exact_h)):
            x = c * score[:, j]
            est, se = x.mean(), x.std(ddof=1) / math.sqrt(n)
            assert abs(est - exact) < 5 * se + 1e-3 * abs(exact), (j, est, se, exact)
    # the score of every parameter has mean zero
    for j in range(2):
        assert abs(score[:, j].mean()) < 5 * score[:, j].std(ddof=1) / math.sqrt(n)


def test_lr_estimator_4x4_two_domains_per_side():
    L, Ld, k, beta, h = 4, 2, 3, 0.45, 0.15
    law = orc.RATE_METROPOLIS
    E = Enumerator(L, Ld, k, beta=beta, h=h, law=law, quantised=False)
    g = orc.score_table(1.0, beta, h, law)
    E.set_score_table(g)
    _, A = orc.rate_table(1.0, beta, h, law, 2)
    s0 = orc.init_spins(L, orc.INIT_RANDOM, 5)
    p0 = np.zeros(E.S)
    p0[_indices(s0[None])[0]] = 1.0
    p, (dpb, dph) = E.schedule_deriv(PAL, p0, (np.zeros(E.S), np.zeros(E.S)))
    H, mag = lattice_energy_all_states(L, 1.0, h)
    n = 100000
    fs, score = orc.sample_final_states_with_score(s0, Ld, k, A, g, 777, n, 1)
    a = H.astype(float)[_indices(fs)]
    c = a - a.mean()
    for j, dp in ((0, dpb), (1, dph)):
        exact = float(H.astype(float) @ dp)
        x = c * score[:, j]
        est, se = x.mean(), x.std(ddof=1) / math.sqrt(n)
        assert abs(est - exact) < 5 * se + 1e-3 * abs(exact), (j, est, se, exact)


def test_derivative_enumeration_matches_finite_difference():
    """The forward-mode derivative itself against a central difference in beta and h."""
    L, Ld, k, beta, h = 2, 1, 2, 0.5, 0.3
    s0 = np.ones((L, L), dtype=np.int8)
    p0 = np.zeros(16)
    p0[_indices(s0[None])[0]] = 1.0
    E = Enumerator(L, Ld, k, beta=beta, h=h, quantised=False)
    E.set_score_table(orc.score_table(1.0, beta, h, 0))
    _, (dpb, dph) = E.schedule_deriv(PAL, p0, (np.zeros(16), np.zeros(16)))
    d = 1e-6
    fd_b = (Enumerator(L, Ld, k, beta=beta + d, h=h, quantised=False).schedule(PAL, p0)
            - Enumerator(L, Ld, k, beta=beta - d, h=h, quantised=False).schedule(PAL, p0)) / (2 * d)
    fd_h = (Enumerator(L, Ld, k, beta=beta, h=h + d, quantised=False).schedule(PAL, p0)
            - Enumerator(L, Ld, k, beta=beta, h=h - d, quantised=False).schedule(PAL, p0)) / (2 * d)
    assert np.max(np.abs(dpb - fd_b)) < 1e-7
    assert np.max(np.abs(dph - fd_h)) < 1e-7


def test_nu_score_of_the_exponential_clock():
    """Score of the clock with respect to the rate prefactor nu (Sec. 2.1):
    zero mean, variance steps/nu^2 (each step contributes (1 - E_i)/nu with
    E_i ~ Exp(1)), and E[T S_nu] = dE[T]/dnu = -E[T]/nu, T the replica clock
    (T scales as 1/nu path by path)."""
    import math
    nu, n = 2.5, 600
    S, T = [], []
    steps = None
    for r in range(n):
        rep = orc.Replica(L=16, Ld=4, k=3, seed=9000 + r, beta=0.4, h=0.05, nu=nu)
        obs = rep.run(4, obs_every=4)
        S.append(rep.score_nu())
        T.append(obs[-1, 3])
        steps = int(rep.steps.sum())
    S, T = np.array(S), np.array(T)
    sd = math.sqrt(steps) / nu
    assert abs(S.mean()) < 5 * sd / math.sqrt(n)
    assert S.var(ddof=1) == pytest.approx(steps / nu ** 2, rel=5 * math.sqrt(2 / n))
    lr = np.mean((T - T.mean()) * S)
    exact = -T.mean() / nu
    se = np.std((T - T.mean()) * S, ddof=1) / math.sqrt(n)
    assert abs(lr - exact) < 5 * se, (lr, exact, se)


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
def test_long_time_derivative_is_the_equilibrium_closed_form(law):
    """Iterating the exact forward-mode derivative of the palindromic schedule
    chain converges to the derivative of the Boltzmann distribution: for
    pi ~ exp(-beta H), H = -J sum s s - h M, d<A>/dbeta = -Cov(A, H) and
    d<A>/dh = beta Cov(A, M) (the schedule keeps pi exactly, Sec. 2.2)."""
    L, Ld, k, beta, h = 2, 1, 3, 0.45, 0.2
    E = Enumerator(L, Ld, k, beta=beta, h=h, law=law, quantised=False)
    E.set_score_table(orc.score_table(1.0, beta, h, law))
    H, mag = lattice_energy_all_states(L, 1.0, h)
    H, mag = H.astype(float), mag.astype(float)
    p = np.zeros(E.S)
    p[0] = 1.0
    dps = (np.zeros(E.S), np.zeros(E.S))
    for _ in range(400):
        p, dps = E.schedule_deriv(PAL, p, dps)
    w = np.exp(-beta * (H - H.min()))
    pi = w / w.sum()
    assert np.max(np.abs(p - pi)) < 1e-12
    for A in (H, mag, H * mag):
        cov_H = pi @ (A * H) - (pi @ A) * (pi @ H)
        cov_M = pi @ (A * mag) - (pi @ A) * (pi @ mag)
        assert float(A @ dps[0]) == pytest.approx(-cov_H, rel=1e-9, abs=1e-12)
        assert float(A @ dps[1]) == pytest.approx(beta * cov_M, rel=1e-9, abs=1e-12)


def test_compensated_sum_against_exact_sum():
    """The oracle sums each domain's score with compensated summation.  On
    long zero-mean sequences like a score's per-step terms (1e5 terms, total
    much smaller than the partial sums) it agrees with math.fsum, the
    correctly rounded sum, to a few ulp of the total, while a plain running
    sum is off by far more."""
    import math
    rng = np.random.default_rng(3)
    worst_comp, worst_plain = 0.0, 0.0
    for trial in range(6):
        x = rng.normal(0.0, 3.0, size=100000) * rng.choice([1.0, 1e-3, 7.0], size=100000)
        exact = math.fsum(x)
        comp = orc.sum_compensated(x)
        plain = float(np.cumsum(x)[-1])  # left-to-right running sum
        ulp = np.spacing(abs(exact))
        worst_comp = max(worst_comp, abs(comp - exact) / ulp)
        worst_plain = max(worst_plain, abs(plain - exact) / ulp)
    assert worst_comp <= 2.0
    assert worst_plain > 50.0
