"""Properties that hold at any size, checked on the GPU path at the
benchmark's sizes: long-run equilibrium energies and magnetisations against
exact results (Onsager, Yang, Kaufman's finite lattice, the ring's transfer
matrix).  The method keeps the Boltzmann distribution exactly (Sec. 2.2), so
its equilibrium averages must agree with them within the statistical error."""
import math

import numpy as np
import pytest

from oracle import exact_ising as ex

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _batch_mean(x, nb=16):
    x = np.asarray(x, dtype=np.float64)
    b = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nb)


@pytest.mark.parametrize("T,k,init,burn", [(3.0, 4, 0, 50), (1.5, 16, 1, 20), (2.5, 1, 0, 100)])
def test_1024_equilibrium_energy_onsager(T, k, init, burn):
    """1024^2, L_d = 32 (the benchmark's lattice): 8 replicas, `burn` sweeps
    (Monte Carlo steps per site; one schedule is 2k/1024 of a sweep), then
    100 sweeps with a record per sweep; the mean energy per site against
    Onsager (finite-size corrections are far below the error at L = 1024
    away from T_c); at T = 1.5 also |m| against Yang's spontaneous
    magnetisation."""
    import paper_1403_4674_gb300 as kmc
    n = 8
    per_sweep = 1024 // (2 * k)
    lat = kmc.Lattice([1024] * n, 32, k, list(range(100 + 17 * k, 100 + 17 * k + n)), init=init)
    lat.set_rates([1 / T] * n, [0.0] * n)
    lat.run(burn * per_sweep)
    obs = lat.run(100 * per_sweep, obs_every=per_sweep).cpu().numpy()
    e = obs[:, :, 0].mean(axis=1)
    mean, se = _batch_mean(e, nb=10)
    assert abs(mean - ex.onsager_energy(T)) < 5 * se + 2e-4, (mean, se, ex.onsager_energy(T))
    if T < 2.0:
        m = np.abs(obs[:, :, 1]).mean(axis=1)
        mm, mse = _batch_mean(m, nb=10)
        assert abs(mm - ex.yang_magnetisation(T)) < 5 * mse + 2e-4, (mm, mse)
    lat.close()


def test_stripes_12x12_equilibrium_energy_kaufman():
    """12^2 in four vertical stripes, N_I = 5, Barker (Sec. 3.2, Table 1's
    lattice at T = 2.4): 500 trajectories' mean energy after burn-in against
    Kaufman's exact finite lattice, -1.28468."""
    import torch
    import paper_1403_4674_gb300 as kmc
    n = 500
    g = kmc.Partitioned(12, kmc.KMC_PART_STRIPES, 4, 5, list(range(1, n + 1)))
    g.set_rates([1 / 2.4] * n)
    g.run(400)
    obs = g.run(2000, obs_every=40).cpu().numpy()  # a record every 10 sweeps
    torch.cuda.synchronize()
    per_traj = obs[:, :, 0].mean(axis=0)
    mean, se = per_traj.mean(), per_traj.std(ddof=1) / math.sqrt(n)
    assert abs(mean - ex.kaufman_energy(12, 2.4)) < 5 * se, (mean, se)
    g.close()


def test_ring_equilibrium_energy_transfer_matrix():
    """8-spin ring, beta J = 0.5, N_D = 8 (one spin per domain), N_I = 10,
    random domain orders: the device ensemble sums at late records against
    the transfer matrix, <H>/N_S = -0.465649."""
    import torch
    import paper_1403_4674_gb300 as kmc
    n = 100000
    ring = kmc.Ring(8, 1, 10, list(range(1, n + 1)), [0b11000000] * n)
    ring.set_rates([0.5] * n, [0.0] * n)
    ring.run(50, schedule=kmc.KMC_SCHEDULE_RANDOM_PERM)
    _, _, ens = ring.run(20, schedule=kmc.KMC_SCHEDULE_RANDOM_PERM, obs_every=8, records=False, ensemble=True)
    torch.cuda.synchronize()
    e = -ens.cpu().numpy()[:, 0] / (n * 8.0)  # -J sum(bonds) / (n N_S) per record
    t = math.tanh(0.5)
    exact = -(t + t ** 7) / (1 + t ** 8)
    # per record the trajectories are independent: sd(e) = 0.32116
    assert np.all(np.abs(e - exact) < 5 * 0.32116 / math.sqrt(n)), (e, exact)
    ring.close()
