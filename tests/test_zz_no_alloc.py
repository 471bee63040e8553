"""The no-allocation entry point against the context API.

Some callers cannot call cudaMalloc: their device memory belongs to another
runtime's pool, or is fully reserved before this library runs.  For them
kmc_run_schedule_noalloc keeps all of its working memory in one static device
array and allocates nothing.  This file is collected last so that a run that
stops at the first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _noalloc(lib, torch, L, Ld, k, seed, beta, h, sched_begin, n, obs_every, spins, obs):
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.kmc_run_schedule_noalloc(L, Ld, k, seed, 1.0, beta, h, 1.0, 0, sched_begin, n, 0, 0, obs_every,
                                      ctypes.c_void_p(spins.data_ptr()),
                                      ctypes.c_void_p(obs.data_ptr()) if obs is not None else None,
                                      ctypes.c_void_p(stream), err, len(err))
    return rc, err.value.decode()


@pytest.mark.parametrize("L,Ld,k", [(128, 32, 4), (256, 16, 3), (64, 8, 1)])
def test_noalloc_matches_context_path_on_two_calls(torch_cuda, L, Ld, k):
    torch = torch_cuda
    import paper_1403_4674_gb300 as kmc
    from paper_1403_4674_gb300 import _lib
    lib = _lib.load()
    seed, beta, h, n1, n2, every = 4242 + L + k, 1 / 2.269, 0.01, 6, 4, 2

    lat = kmc.Lattice([L], Ld, k, [seed], init=kmc.KMC_INIT_RANDOM)
    lat.set_rates([beta], [h])
    start = lat.spins.clone()
    obs1 = lat.run(n1, obs_every=every).cpu().numpy()[:, 0, :]
    s1 = lat.spins.clone()
    obs2 = lat.run(n2, obs_every=every).cpu().numpy()[:, 0, :]
    s2 = lat.spins.clone()
    lat.close()

    spins = start.clone()
    o1 = torch.empty((n1 // every, 4), dtype=torch.float64, device="cuda")
    rc, msg = _noalloc(lib, torch, L, Ld, k, seed, beta, h, 0, n1, every, spins, o1)
    assert rc == 0, msg
    assert torch.equal(spins, s1)
    a1 = o1.cpu().numpy()
    assert np.array_equal(a1[:, :3], obs1[:, :3])
    np.testing.assert_allclose(a1[:, 3], obs1[:, 3], rtol=1e-12, atol=0)

    o2 = torch.empty((n2 // every, 4), dtype=torch.float64, device="cuda")
    rc, msg = _noalloc(lib, torch, L, Ld, k, seed, beta, h, n1, n2, every, spins, o2)
    assert rc == 0, msg
    assert torch.equal(spins, s2)
    a2 = o2.cpu().numpy()
    assert np.array_equal(a2[:, :3], obs2[:, :3])
    # clocks restart at every no-alloc call; the context's keep running
    np.testing.assert_allclose(a2[:, 3], obs2[:, 3] - obs1[-1, 3], rtol=1e-12, atol=0)


def test_noalloc_rejects_sizes_beyond_its_array(torch_cuda):
    torch = torch_cuda
    from paper_1403_4674_gb300 import _lib
    lib = _lib.load()
    spins = torch.ones(8192 * 8192, dtype=torch.int8, device="cuda")
    rc, msg = _noalloc(lib, torch, 8192, 64, 8, 1, 0.4, 0.0, 0, 1, 0, spins, None)
    assert rc == -1 and "too large" in msg
    small = torch.ones(64 * 64, dtype=torch.int8, device="cuda")
    # a buffer with room for every record, so that if the size check ever
    # stopped refusing this call the run would write inside it (9.6 MB)
    obs = torch.empty(300000 * 4, dtype=torch.float64, device="cuda")
    # 300000 observation records need more working memory than the array holds
    rc, msg = _noalloc(lib, torch, 64, 16, 1, 1, 0.4, 0.0, 0, 300000, 1, small, obs)
    assert rc == -1 and "bytes" in msg
    assert bool((small == 1).all())  # nothing ran
