"""Autotuner and batched runs on the GPU: the tuned plan, domain side and k
leave every replica's trajectory equal to the oracle's for that (L_d, k), and
a captured batch step replays the eager one bit for bit."""
import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle_spins(L, Ld, k, seed, beta, h, n, init=orc.INIT_RANDOM):
    rep = orc.Replica(L=L, Ld=Ld, k=k, seed=seed, beta=beta, h=h, init=init)
    rep.run(n)
    return rep.spins


def test_tune_plan_keeps_parity():
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import autotune
    L, ks, seeds = [64, 128, 96], [1, 16, 4], [5, 6, 7]
    beta, h = [0.5, 0.44, 0.3], [0.0, 0.01, -0.02]
    lat = kmc.Lattice(L, 16, 1, seeds)
    lat.set_replica_params(k=ks)
    lat.reset(kmc.KMC_INIT_RANDOM)
    lat.set_rates(beta, h)
    plan, trials = autotune.tune_plan(lat, beta, h, trial_schedules=5)
    assert any(t.error is None for t in trials)
    assert lat.launch()[0] == plan[0] or plan[0] == kmc.KMC_LAUNCH_AUTO
    lat.run(4)
    lat.sync()
    for r in range(3):
        assert np.array_equal(lat.replica_spins(r).cpu().numpy(),
                              _oracle_spins(L[r], 16, ks[r], seeds[r], beta[r], h[r], 4))
    lat.close()


def test_tune_batch_groups_and_parity():
    import torch
    from paper_1403_4674_gb300 import autotune
    L = [32, 48, 64, 96, 128, 80, 160]
    seeds = [11 + i for i in range(len(L))]
    beta = list(np.linspace(1 / 3.5, 1 / 1.5, len(L)))
    h = list(np.linspace(-0.1, 0.1, len(L)))
    choices = autotune.tune_batch(L, beta, h, seeds, k_candidates=(2, 4), Ld_candidates=(8, 16),
                                  plans=[(0, 0, 16), (2, 8, 4)], trial_schedules=3)
    covered = sorted(i for ch in choices for i in ch.replicas)
    assert covered == list(range(len(L)))
    for ch in choices:
        assert ch.k in (2, 4) and ch.L_d in (8, 16)
        assert all(L[i] % (2 * ch.L_d) == 0 for i in ch.replicas)
    batch = autotune.Batch(L, beta, h, seeds, choices)
    batch.run(3, obs_every=1)
    torch.cuda.synchronize()
    for ch, lat in zip(choices, batch.lattices):
        for j, i in enumerate(ch.replicas):
            assert np.array_equal(lat.replica_spins(j).cpu().numpy(),
                                  _oracle_spins(L[i], ch.L_d, ch.k, seeds[i], beta[i], h[i], 3))
    # one CUDA graph for the whole batch step replays the eager step
    g = batch.capture(3, obs_every=1, reset=0)
    eager = [lat.spins.clone() for lat in batch.lattices]
    eager_obs = [o.clone() for o in batch.outs]
    for lat in batch.lattices:
        lat.spins.zero_()
    g.replay()
    torch.cuda.synchronize()
    for lat, s, o, eo in zip(batch.lattices, eager, batch.outs, eager_obs):
        assert torch.equal(lat.spins, s)
        assert torch.equal(o[..., :3], eo[..., :3])
        torch.testing.assert_close(o[..., 3], eo[..., 3], rtol=1e-12, atol=0)
    batch.close()
