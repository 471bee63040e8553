"""Likelihood-ratio gradients on the GPU.

The run kernel's GRAD variant accumulates the path score d log P / d(beta, h)
(App. A: step probabilities a_c/n_d and 1 - R/n_d) per domain.  Checked
against the oracle's score (tests/test_oracle_score.py pins the oracle to the
exact derivative of the enumerated chain), against common-random-number finite
differences, and through the torch.autograd wrapper.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
@pytest.mark.parametrize("Ld,k", [(16, 4), (32, 16), (8, 40)])
@pytest.mark.parametrize("per_pass", [False, True])
def test_score_parity_with_oracle(law, Ld, k, per_pass):
    import paper_1403_4674_gb300 as kmc
    L = [4 * Ld, 6 * Ld]
    seeds, beta, h = [21, 22], [0.45, 0.4], [0.1, -0.05]
    lat = kmc.Lattice(L, Ld, k, seeds)
    lat.enable_grad(True)
    lat.set_rates(beta, h, law=law)
    if per_pass:
        lat.set_observation(kmc.KMC_OBS_PASS)
    obs = lat.run(6, obs_every=2).cpu().numpy()
    score = lat.score().cpu().numpy()
    for r in range(2):
        ref = orc.Replica(L=L[r], Ld=Ld, k=k, seed=seeds[r], beta=beta[r], h=h[r], law=law)
        ref.enable_score()
        robs = ref.run(6, obs_every=2, obs_per_pass=per_pass)
        # the score does not change the trajectory
        assert np.array_equal(lat.replica_spins(r).cpu().numpy(), ref.spins)
        assert np.array_equal(obs[:, r, :3], robs[:, :3])
        scale = 1.0 + np.abs(robs[:, 4:6])
        assert np.all(np.abs(obs[:, r, 4:6] - robs[:, 4:6]) <= 1e-12 * scale), (obs[:, r, 4:6], robs[:, 4:6])
        np.testing.assert_allclose(score[r], ref.score.sum(axis=0), rtol=1e-12, atol=1e-12)
    lat.close()


def test_score_reset_starts_a_new_segment():
    import paper_1403_4674_gb300 as kmc
    lat = kmc.Lattice([64], 16, 4, [5])
    lat.enable_grad(True)
    lat.set_rates([0.44], [0.02])
    lat.run(3)
    first = lat.score(reset=True).cpu().numpy()
    assert np.all(first != 0)
    assert np.all(lat.score().cpu().numpy() == 0)
    lat.run(2)
    ref = orc.Replica(L=64, Ld=16, k=4, seed=5, beta=0.44, h=0.02)
    ref.run(3)
    ref.enable_score()
    ref.run(2)
    np.testing.assert_allclose(lat.score().cpu().numpy()[0], ref.score.sum(axis=0), rtol=1e-12, atol=1e-12)
    lat.close()


def _final_obs(L, Ld, k, seeds, beta, h, n, grad, col):
    import paper_1403_4674_gb300 as kmc
    lat = kmc.Lattice(L, Ld, k, seeds, init=kmc.KMC_INIT_ALL_UP)
    lat.enable_grad(grad)
    nrep = len(L)
    lat.set_rates([beta] * nrep, [h] * nrep)
    obs = lat.run(n, obs_every=n)
    A = obs[-1, :, col].contiguous()
    out = (A.cpu().numpy(), lat.lr_estimate(A).cpu().numpy() if grad else None,
           lat.score().cpu().numpy() if grad else None)
    lat.close()
    return out


@pytest.mark.parametrize("param,col", [("beta", 0), ("beta", 1), ("h", 1)])
def test_lr_gradient_matches_crn_finite_difference(param, col):
    """d E[A]/d theta: likelihood ratio vs common-random-number central difference, step 1e-4.

    A = e (col 0) or m (col 1); e depends on h explicitly, so the h case uses m,
    whose whole h-dependence goes through the path distribution."""
    R, L, Ld, k, n = 4096, 16, 8, 4, 3
    beta, h, d = 1 / 2.4, 0.02, 1e-4
    seeds = list(range(1000, 1000 + R))
    A, lr, S = _final_obs([L] * R, Ld, k, seeds, beta, h, n, True, col)
    j = 0 if param == "beta" else 1
    x = (A - A.mean()) * S[:, j]
    se_lr = x.std(ddof=1) / math.sqrt(R)
    # unbiased sample covariance (the replica mean as baseline)
    assert lr[j] == pytest.approx(x.sum() / (R - 1), rel=1e-12, abs=1e-12 * np.abs(x).sum() / (R - 1))
    bp, hp = (beta + d, h) if j == 0 else (beta, h + d)
    bm, hm = (beta - d, h) if j == 0 else (beta, h - d)
    Ap, _, _ = _final_obs([L] * R, Ld, k, seeds, bp, hp, n, False, col)
    Am, _, _ = _final_obs([L] * R, Ld, k, seeds, bm, hm, n, False, col)
    diff = (Ap - Am) / (2 * d)
    fd, se_fd = diff.mean(), diff.std(ddof=1) / math.sqrt(R)
    assert abs(lr[j] - fd) < 5 * math.hypot(se_lr, se_fd), (lr[j], se_lr, fd, se_fd)


def _oracle_lr(L, Ld, k, seeds, beta, h, n, col):
    """Oracle replicas on the same seeds: per-replica observable A, magnetisation m and score S."""
    A, m, S = [], [], []
    for sd in seeds:
        ref = orc.Replica(L=L, Ld=Ld, k=k, seed=sd, beta=beta, h=h, init=orc.INIT_RANDOM)
        ref.enable_score()
        rec = ref.run(n, obs_every=n)[-1]
        A.append(rec[col])
        m.append(rec[1])
        S.append(ref.score.sum(axis=0))
    return np.array(A), np.array(m), np.array(S)


@pytest.mark.parametrize("name,col", [("e", 0), ("m", 1), ("em", 2)])
def test_autograd_value_matches_oracle_covariance(name, col):
    """expectation(...).backward() against the same estimator built from the
    oracle's records and scores on the same seeds: the unbiased covariance of
    A with the path score plus the explicit h-dependence of A (de/dh = -m,
    d(em)/dh = -m^2, computed here), to 1e-12 of the sum of the terms'
    magnitudes; the forward value is the oracle's replica mean."""
    import torch
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300.autograd import expectation
    R, L, Ld, k, n, b0, h0 = 256, 32, 8, 4, 4, 0.42, 0.05
    seeds = list(range(7, 7 + R))
    lat = kmc.Lattice([L] * R, Ld, k, seeds)
    beta = torch.tensor(b0, dtype=torch.float64, requires_grad=True)
    h = torch.tensor(h0, dtype=torch.float64, requires_grad=True)
    val = expectation(lat, beta, h, n_schedules=n, observable=name)
    val.backward()
    lat.close()
    A, m, S = _oracle_lr(L, Ld, k, seeds, b0, h0, n, col)
    assert val.item() == pytest.approx(A.mean(), rel=1e-14, abs=1e-15)
    xs = {"e": -m, "m": np.zeros(R), "em": -m * m}[name]
    for j, got in ((0, beta.grad.item()), (1, h.grad.item())):
        terms = (A - A.mean()) * S[:, j] / (R - 1)
        want = terms.sum() + (xs.mean() if j == 1 else 0.0)
        mag = np.abs(terms).sum() + (np.abs(xs).mean() if j == 1 else 0.0)
        assert abs(got - want) <= 1e-12 * mag, (name, j, got, want, mag)


def test_autograd_field_gradient_of_energy_matches_crn_finite_difference():
    """d<e>/dh through torch.autograd, where the explicit term -<m> matters,
    against a common-random-number central difference of the forward value
    (step 1e-4) within 5 standard errors."""
    import torch
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300.autograd import expectation
    R, L, Ld, k, n = 4096, 16, 8, 4, 3
    b0, h0, d = 1 / 2.4, 0.02, 1e-4
    seeds = list(range(3000, 3000 + R))
    lat = kmc.Lattice([L] * R, Ld, k, seeds)
    beta = torch.tensor(b0, dtype=torch.float64, requires_grad=True)
    h = torch.tensor(h0, dtype=torch.float64, requires_grad=True)
    up = kmc.KMC_INIT_ALL_UP  # the start of _final_obs
    expectation(lat, beta, h, n_schedules=n, observable="e", init=up).backward()
    lr = h.grad.item()
    # per-replica terms of the same estimate for its standard error
    A, _, S = _final_obs([L] * R, Ld, k, seeds, b0, h0, n, True, 0)
    m, _, _ = _final_obs([L] * R, Ld, k, seeds, b0, h0, n, False, 1)
    x = (A - A.mean()) * S[:, 1] * R / (R - 1) - m
    se_lr = x.std(ddof=1) / math.sqrt(R)
    assert lr == pytest.approx(x.mean(), rel=1e-12, abs=1e-12 * np.abs(x).mean())
    with torch.no_grad():
        ep = expectation(lat, torch.tensor(b0, dtype=torch.float64), torch.tensor(h0 + d, dtype=torch.float64), n,
                         init=up)
        em = expectation(lat, torch.tensor(b0, dtype=torch.float64), torch.tensor(h0 - d, dtype=torch.float64), n,
                         init=up)
    Ap, _, _ = _final_obs([L] * R, Ld, k, seeds, b0, h0 + d, n, False, 0)
    Am, _, _ = _final_obs([L] * R, Ld, k, seeds, b0, h0 - d, n, False, 0)
    assert ep.item() == pytest.approx(Ap.mean(), rel=1e-14) and em.item() == pytest.approx(Am.mean(), rel=1e-14)
    diff = (Ap - Am) / (2 * d)
    fd, se_fd = diff.mean(), diff.std(ddof=1) / math.sqrt(R)
    assert abs(lr - fd) < 5 * math.hypot(se_lr, se_fd), (lr, se_lr, fd, se_fd)
    # without the explicit term the estimate would miss by <m>, many standard errors here
    assert abs(lr + m.mean() - fd) > 5 * math.hypot(se_lr, se_fd)
    lat.close()


def test_nu_score_parity_and_lr():
    """The rate-prefactor clock score per replica against the oracle's, and
    refused after a run with the expected clock."""
    import paper_1403_4674_gb300 as kmc
    L, seeds, beta, h, nu = [64, 96], [31, 32], [0.45, 0.3], [0.0, 0.1], 1.7
    lat = kmc.Lattice(L, 16, 5, seeds)
    lat.set_rates(beta, h, nu=nu)
    lat.run(7)
    s = lat.score_nu().cpu().numpy()
    for r in range(2):
        ref = orc.Replica(L=L[r], Ld=16, k=5, seed=seeds[r], beta=beta[r], h=h[r], nu=nu)
        ref.run(7)
        steps = float(ref.steps.sum())
        assert abs(s[r] - ref.score_nu()) <= 1e-12 * steps / nu, (s[r], ref.score_nu())
    lat.run(1, time_mode=kmc.KMC_TIME_EXPECTED)
    with pytest.raises(kmc.KmcError):
        lat.score_nu()
    lat.reset(kmc.KMC_INIT_RANDOM)
    lat.run(1)
    lat.score_nu()  # a reset starts a new exponential-only segment
    lat.close()
