"""Pin the oracle's Philox4x32-10 to a library implementation.

The oracle writes Philox4x32-10 out from Salmon et al. (SC'11).  PyTorch ships
its own host-callable engine (at::Philox4_32: key = seed, counter =
{offset, subsequence}); running it and comparing outputs pins the oracle's
rounds, multipliers and key schedule to something other than itself.
"""
import numpy as np
import pytest

from oracle import oracle as orc


@pytest.fixture(scope="module")
def torch_philox():
    torch = pytest.importorskip("torch")
    from torch.utils.cpp_extension import load_inline
    src = r'''
#include <ATen/core/PhiloxRNGEngine.h>
#include <torch/extension.h>
std::vector<int64_t> draw4(uint64_t seed, uint64_t subseq, uint64_t offset) {
  at::Philox4_32 eng(seed, subseq, offset);
  std::vector<int64_t> out;
  for (int i = 0; i < 4; ++i) out.push_back((int64_t)eng());
  return out;
}
'''
    try:
        return load_inline("kmc_test_torch_philox", cpp_sources=src, functions=["draw4"],
                           verbose=False)
    except Exception as exc:  # pragma: no cover - toolchain missing
        pytest.skip("cannot compile the torch Philox probe: %s" % exc)


def test_philox_matches_torch_engine(torch_philox):
    rng = np.random.default_rng(20240517)
    for _ in range(200):
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64)
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64)
        seed = int(key[0]) | (int(key[1]) << 32)
        offset = int(ctr[0]) | (int(ctr[1]) << 32)
        subseq = int(ctr[2]) | (int(ctr[3]) << 32)
        ref = [x & 0xFFFFFFFF for x in torch_philox.draw4(seed, subseq, offset)]
        got = orc.philox4x32_10(ctr.astype(np.uint32), key.astype(np.uint32))
        assert [int(v) for v in got] == ref


def test_philox_counter_sensitivity():
    a = orc.philox4x32_10([0, 0, 0, 0], [1, 2])
    for w in range(4):
        c = [0, 0, 0, 0]
        c[w] = 1
        assert not np.array_equal(orc.philox4x32_10(c, [1, 2]), a)
    assert not np.array_equal(orc.philox4x32_10([0, 0, 0, 0], [1, 3]), a)
