"""Statistics layer (Sec. 2.3, appendix Eq. efficiency) pinned to closed forms
and to the exact autocorrelation of the enumerated schedule chain."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from oracle.enumerate import Enumerator
from paper_1403_4674_gb300 import stats


def test_fit_recovers_exact_exponential():
    d = np.arange(200)
    for tau in (0.7, 3.0, 25.0, 400.0):
        C = 2.5 * np.exp(-d * 4.0 / tau)
        assert math.isclose(stats.fit_tau(C, dt=4.0), tau, rel_tol=1e-6)


def test_autocorrelation_matches_direct_sums():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((5, 37))
    C = stats.autocorrelation(A, max_lag=10)
    dA = A - A.mean()
    for d in range(11):
        direct = np.mean([np.mean(dA[i, :37 - d] * dA[i, d:]) for i in range(5)])
        assert math.isclose(C[d], direct, rel_tol=1e-10, abs_tol=1e-14)


def test_ar1_process_decay_constant():
    """x_{t+1} = phi x_t + sqrt(1-phi^2) e_t has C(d) = phi^d exactly."""
    tau = 12.0
    phi = math.exp(-1.0 / tau)
    rng = np.random.default_rng(11)
    n_traj, n = 200, 4000
    x = np.empty((n_traj, n))
    x[:, 0] = rng.standard_normal(n_traj)
    e = rng.standard_normal((n_traj, n)) * math.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[:, t] = phi * x[:, t - 1] + e[:, t]
    est = stats.tau_par(x, steps_per_record=1.0, max_lag=80)
    assert abs(est / tau - 1.0) < 0.05


def test_efficiency_and_rescaling():
    assert stats.efficiency(100.0, 50.0, 2) == 1.0
    assert stats.efficiency(31.8, 31.8, 1) == 1.0
    np.testing.assert_array_equal(stats.rescale_time([0, 10, 20], 30.0, 60.0), [0.0, 5.0, 10.0])
    assert stats.steps_per_schedule(4, 16) == 2 * 4 * 16
    A = np.arange(12.0).reshape(3, 4)
    np.testing.assert_array_equal(stats.time_dependent_average(A), [4.0, 5.0, 6.0, 7.0])


def test_tau_par_of_oracle_trajectories_matches_exact_chain():
    """tau_PAR estimated from oracle trajectories of A = H m on a 4x4 lattice
    (L_d = 2, k = 1, T = 4, palindrome) agrees with the decay constant of the
    exact autocorrelation <dA, T^n (pi dA)> of the enumerated schedule chain."""
    L, Ld, k, T = 4, 2, 1, 4.0
    E = Enumerator(L, Ld, k, beta=1 / T)
    m = (2 * E.bits.sum(axis=1) - L * L) / float(L * L)
    A = E.H * m
    dA = A - E.pi @ A
    v = E.pi * dA
    C = []
    for _ in range(40):
        C.append(float(dA @ v))
        v = E.schedule([0, 1, 2, 3, 3, 2, 1, 0], v)
    sps = stats.steps_per_schedule(k, (L // Ld) ** 2)
    tau_exact = stats.fit_tau(np.array(C), dt=sps)

    rows = []
    for r in range(48):
        rep = orc.Replica(L=L, Ld=Ld, k=k, seed=9000 + r, beta=1 / T)
        rep.run(100)  # equilibrate (about 20 tau)
        obs = rep.run(2500, obs_every=1)
        rows.append(obs[:, 0] * obs[:, 1] * (L * L) ** 2)  # H m from e and m per site
    est = stats.tau_par(np.array(rows), steps_per_record=sps, max_lag=40)
    assert abs(est / tau_exact - 1.0) < 0.08, (est, tau_exact)


def test_ring_ensemble_averages_match_per_trajectory_records():
    """The averages from the ring's ensemble sums equal the means over the
    oracle's per-trajectory records (e, m, e*m) and record states."""
    from oracle import oracle as orc
    from paper_1403_4674_gb300 import stats as st
    n, NS, J, h = 500, 8, 0.8, 0.15
    _, obs, states, _, _ = orc.ring_run_many([0b11000000] * n, np.arange(3, 3 + n), NS, 2, 5, 0.5, 6, J=J, h=h,
                                             obs_every=1)
    bits = ((states[:, :, None] >> np.arange(NS, dtype=np.uint64)) & np.uint64(1)).astype(np.int64)  # [traj, rec, n]
    sig = 2 * bits - 1
    mag = sig.sum(axis=2)
    bonds = (sig * np.roll(sig, -1, axis=2)).sum(axis=2)
    ens = np.concatenate([np.stack([bonds.sum(0), mag.sum(0), (bonds * mag).sum(0), (mag * mag).sum(0)], 1),
                          bits.sum(axis=0)], axis=1)
    av = st.ring_ensemble_averages(ens, n, NS, J=J, h=h)
    np.testing.assert_allclose(av["energy"], obs[:, :, 0].mean(axis=0), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(av["magnetisation"], obs[:, :, 1].mean(axis=0), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(av["A"], obs[:, :, 2].mean(axis=0), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(av["spin"], sig.mean(axis=0), rtol=0, atol=1e-15)
