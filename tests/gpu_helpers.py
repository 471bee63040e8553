"""Shared helpers of the GPU tests: run the same seeded workload on the CUDA
path (through the C ABI) and on the CPU oracle."""
import numpy as np

from oracle import oracle as orc


def run_both(L, Ld, k, seeds, beta, h, n_sched, *, law=0, init=0, schedule=0, time_mode=0,
             obs_every=0, nu=1.0, J=1.0, launch=None, chunks=None, obs_per_pass=False, dtau=0.0):
    import paper_1403_4674_gb300 as kmc
    n = len(L)
    ks = list(k) if isinstance(k, (list, tuple)) else [k] * n
    inits = list(init) if isinstance(init, (list, tuple)) else [init] * n
    per_replica = isinstance(k, (list, tuple)) or isinstance(init, (list, tuple))
    lat = kmc.Lattice(L, Ld, ks[0], seeds, init=inits[0])
    if per_replica:
        # per-replica steps and starts in one context
        lat.set_replica_params(k=ks, init=inits)
        lat.reset(kmc.KMC_INIT_PER_REPLICA)
    if launch is not None:
        lat.set_launch(*launch)
        assert lat.launch()[0] == launch[0]
    lat.set_rates(beta, h, J=J, nu=nu, law=law)
    if obs_per_pass:
        lat.set_observation(kmc.KMC_OBS_PASS)
    if dtau > 0:
        lat.set_horizon(dtau)
    chunks = chunks or [n_sched]
    obs_gpu = []
    for c in chunks:
        o = lat.run(c, schedule=schedule, time_mode=time_mode, obs_every=obs_every)
        if o is not None:
            obs_gpu.append(o.cpu().numpy())
    lat.sync()
    gpu = {"spins": [lat.replica_spins(r).cpu().numpy() for r in range(len(L))]}
    gpu["hash"], gpu["flips"], gpu["t"] = lat.domain_state()
    gpu["obs"] = np.concatenate(obs_gpu, axis=0) if obs_gpu else None
    gpu["observables"] = lat.observables()
    gpu["launches"] = lat.kernel_launches()
    lat.close()

    ref = {"spins": [], "hash": [], "flips": [], "t": [], "obs": []}
    for r in range(len(L)):
        rep = orc.Replica(L=L[r], Ld=Ld, k=ks[r], seed=seeds[r], beta=beta[r], h=h[r], J=J, nu=nu,
                          law=law, init=inits[r], dtau=dtau)
        obs_r = []
        for c in chunks:
            o = rep.run(c, schedule=schedule, time_mode=time_mode, obs_every=obs_every,
                        obs_per_pass=obs_per_pass)
            obs_r.append(o)
        ref["spins"].append(rep.spins.copy())
        ref["hash"].append(rep.hash.copy())
        ref["flips"].append(rep.flips.copy())
        ref["t"].append(rep.domain_times(time_mode))
        ref["obs"].append(np.concatenate(obs_r, axis=0) if obs_r else None)
    ref["hash"] = np.concatenate(ref["hash"])
    ref["flips"] = np.concatenate(ref["flips"])
    ref["t"] = np.concatenate(ref["t"])
    return gpu, ref


def assert_parity(gpu, ref, n_rep, obs=True, rtol=1e-12):
    for r in range(n_rep):
        assert np.array_equal(gpu["spins"][r], ref["spins"][r]), "replica %d: spins differ" % r
    assert np.array_equal(gpu["flips"], ref["flips"]), "real-event counts differ"
    assert np.array_equal(gpu["hash"], ref["hash"]), "event sequences (hashes) differ"
    np.testing.assert_allclose(gpu["t"], ref["t"], rtol=rtol, atol=0)
    if obs and gpu["obs"] is not None:
        for r in range(n_rep):
            g = gpu["obs"][:, r, :]
            o = ref["obs"][r]
            assert g.shape[0] == o.shape[0]
            assert np.array_equal(g[:, :3], o[:, :3]), "replica %d: e, m, e*m differ" % r
            np.testing.assert_allclose(g[:, 3], o[:, 3], rtol=rtol, atol=0)
