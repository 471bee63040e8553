"""Seeded random configurations against the oracle, across every launch plan.

Each case draws a domain side, a few replicas of different sizes, steps per
visit, temperatures, fields, starts, rate law, schedule kind, clock mode,
record spacing, a launch plan the library accepts for that domain side, and a
split of the schedules over several calls; the CUDA path must reproduce the
oracle's spins, per-domain real-event counts and event hashes and records
bit for bit (clocks to 1e-12).  The draws are seeded, so a failure names its
case."""
import numpy as np
import pytest

from gpu_helpers import assert_parity, run_both

THREADS, GRID, CLUSTER = 3, 2, 1
N_CASES = 24


@pytest.fixture(scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(seed):
    """Case `seed`: the domain side cycles through 8, 16, 32, 64 and the plan
    through the ones the side allows; the rest is drawn."""
    rng = np.random.default_rng(1000 + seed)
    Ld = (8, 16, 32, 64)[seed % 4]
    n = int(rng.integers(1, 4))
    mult = [1, 2, 3] if Ld < 64 else [1, 2]
    L = [2 * Ld * int(rng.choice(mult)) for _ in range(n)]
    k = [int(rng.integers(1, 21)) for _ in range(n)]
    seeds = [int(s) for s in rng.integers(1, 2**62, size=n)]
    beta = [float(b) for b in rng.uniform(0.0, 1.0, size=n)]
    h = [float(x) for x in rng.uniform(-0.2, 0.2, size=n)]
    init = [int(i) for i in rng.integers(0, 2, size=n)]
    law = int(rng.integers(0, 2))
    schedule = int(rng.integers(0, 2))
    time_mode = int(rng.integers(0, 2))
    obs_every = int(rng.integers(0, 3))
    plans = [(GRID, 152, 8), (CLUSTER, 4, 16)]
    if Ld == 8:
        plans += [(THREADS, 0, 4), (THREADS, 16, 2)]
    else:
        plans += [(THREADS, 1, int(rng.integers(1, 5))), (THREADS, 2, int(rng.integers(1, 5)))]
    plan = plans[(seed // 4) % len(plans)]
    chunks = [int(c) for c in rng.integers(1, 4, size=int(rng.integers(1, 3)))]
    return dict(L=L, Ld=Ld, k=k, seeds=seeds, beta=beta, h=h, init=init, law=law, schedule=schedule,
                time_mode=time_mode, obs_every=obs_every, plan=plan, chunks=chunks)


@pytest.mark.gpu
@pytest.mark.parametrize("seed", range(N_CASES))
def test_random_configuration_matches_oracle(_cuda, seed):
    c = _case(seed)
    gpu, ref = run_both(c["L"], c["Ld"], c["k"], c["seeds"], c["beta"], c["h"], sum(c["chunks"]), law=c["law"],
                        init=c["init"], schedule=c["schedule"], time_mode=c["time_mode"],
                        obs_every=c["obs_every"], launch=c["plan"], chunks=c["chunks"])
    assert_parity(gpu, ref, len(c["L"]))


def test_cases_cover_every_plan_and_side():
    """The seeded draws above exercise each domain side and the thread plans."""
    cases = [_case(s) for s in range(N_CASES)]
    assert {c["Ld"] for c in cases} == {8, 16, 32, 64}
    assert any(c["plan"][0] == THREADS and c["Ld"] in (16, 32, 64) and c["plan"][1] == 2 for c in cases)
    assert any(c["plan"][0] == THREADS and c["Ld"] == 64 for c in cases)
    assert any(c["plan"][0] == GRID for c in cases) and any(c["plan"][0] == CLUSTER for c in cases)
