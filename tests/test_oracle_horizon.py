"""Fixed-time domain process (a visit runs its domain for the time dtau):
the step count is Poisson(n_d nu dtau) by table inversion, the visit is the
matrix exponential of the domain's generator, and the schedule stays
stationary and reversible."""
import numpy as np
import pytest
from scipy import linalg, stats

from oracle import oracle as orc
from oracle.enumerate import Enumerator

PAL = [0, 1, 2, 3, 3, 2, 1, 0]


def _table_probs(mu):
    T = orc.horizon_table(mu).astype(np.float64) / 2.0 ** 64
    probs = np.diff(np.concatenate([[0.0], T]))
    return np.append(probs, 1.0 - T[-1])


@pytest.mark.parametrize("mu", [0.05, 0.7, 8.0, 120.0])
def test_table_is_the_poisson_cdf(mu):
    T = orc.horizon_table(mu)
    k = np.arange(len(T))
    # the pmf is summed in FP64 in k order: rounding grows with the number of terms
    np.testing.assert_allclose(T.astype(np.float64) / 2.0 ** 64, stats.poisson.cdf(k, mu), rtol=0,
                               atol=4e-16 * len(T))
    assert np.all(np.diff(T.astype(np.float64)) >= 0)
    assert orc.horizon_kmax(mu) == len(T)
    # the true tail beyond kmax is below 1e-30; what remains at K = kmax is the
    # summation's rounding
    assert 1.0 - T[-1] / 2.0 ** 64 < 4e-16 * len(T)


def test_fixed_time_visit_is_the_matrix_exponential():
    """2x2 lattice, one-site domains: sum_K Poisson(K; mu) P_d^K equals
    expm(dtau Q_d) with Q_d = n_d nu (P_d - I) (uniformisation)."""
    beta, h, nu, dtau = 0.6, 0.2, 1.3, 0.9
    E = Enumerator(2, 1, 1, beta=beta, h=h, quantised=False)
    mu = E.nd * nu * dtau
    kk = np.arange(200)
    pmf = stats.poisson.pmf(kk, mu)
    for d in range(4):
        P = E.dense(lambda v: E.step(d, v))
        Q = E.nd * nu * (P - np.eye(E.S))
        M = E.dense(lambda v: E.horizon_domain(d, v, pmf))
        np.testing.assert_allclose(M, linalg.expm(dtau * Q), rtol=0, atol=1e-14)


def test_fixed_time_palindrome_is_stationary_and_reversible():
    E = Enumerator(4, 2, 1, beta=0.45, h=0.15)
    probs = _table_probs(E.nd * 1.0 * 0.6)
    op = lambda v: E.horizon_schedule(PAL, v, probs)  # noqa: E731
    assert E.stationarity_error(op) < 1e-13
    assert E.detailed_balance_error(op, n_probe=3) < 1e-13


def test_fixed_time_sampler_matches_enumeration():
    """2x2 lattice, L_d = 1, one palindromic schedule of fixed-time visits:
    the oracle's final-state histogram against the enumerated operator."""
    beta, h, dtau = 0.5, 0.3, 0.7
    E = Enumerator(2, 1, 1, beta=beta, h=h)
    probs = _table_probs(E.nd * dtau)
    s0 = np.ones((2, 2), dtype=np.int8)
    s0[0, 1] = -1
    p0 = np.zeros(E.S)
    idx0 = int(((s0.reshape(-1) > 0).astype(np.int64) << np.arange(4)).sum())
    p0[idx0] = 1.0
    pe = E.horizon_schedule(PAL, p0, probs)
    n = 30000
    counts = np.zeros(E.S)
    for r in range(n):
        rep = orc.Replica(L=2, Ld=1, k=1, seed=10000 + r, beta=beta, h=h, dtau=dtau, spins=s0.copy())
        rep.run(1, time_mode=orc.TIME_HORIZON)
        counts[int(((rep.spins.reshape(-1) > 0).astype(np.int64) << np.arange(4)).sum())] += 1
    keep = pe * n >= 5
    chi2 = (((counts - pe * n) ** 2) / (pe * n))[keep].sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-5


def test_steps_per_visit_are_poisson_and_clock_is_exact():
    L, Ld, dtau, nu = 64, 4, 0.4, 1.0
    mu = Ld * Ld * nu * dtau
    rep = orc.Replica(L=L, Ld=Ld, k=1, seed=3, beta=0.4, dtau=dtau, nu=nu)
    n_sched = 100
    rep.run(n_sched, time_mode=orc.TIME_HORIZON)
    visits = 2 * n_sched
    per_domain = rep.steps.astype(np.float64)  # sum of `visits` Poisson(mu) counts
    assert abs(per_domain.mean() / (visits * mu) - 1.0) < 0.02
    # 256 independent domains: the sample variance is within 4 sigma (sqrt(2/255))
    assert abs(per_domain.var(ddof=1) / (visits * mu) - 1.0) < 0.36
    np.testing.assert_allclose(rep.domain_times(orc.TIME_HORIZON), visits * dtau, rtol=1e-13)
