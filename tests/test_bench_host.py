"""Host-side logic of bench.py that needs no GPU: the name a launch's ncu
counts are keyed by, and the check of those counts against the kernel
sources they were taken on."""
import bench


class _Lat:
    def __init__(self, L_d, n, mode):
        self.L_d, self.n_replicas, self._mode = L_d, n, mode

    def launch(self):
        return (self._mode, 0, 0, 4, 0)


def test_counts_kernel_names():
    assert bench.counts_kernel(_Lat(32, 18, 3), (3, 2, 4)) == "tpdr_kernel/rr"
    assert bench.counts_kernel(_Lat(32, 18, 3), (3, 1, 4)) == "tpdr_kernel"
    assert bench.counts_kernel(_Lat(64, 1, 3), (3, 2, 4)) == "tpdr64_kernel"  # one replica: no other order
    assert bench.counts_kernel(_Lat(8, 512, 3), (3, 0, 4)) == "tpd_kernel"
    assert bench.counts_kernel(_Lat(32, 18, 2), (2, 760, 4)) == "run_kernel"


def test_counts_follow_their_kernel_sources(monkeypatch):
    # every stored count names a kernel whose sources are listed and hashed
    for (_, kern) in bench.NCU_COUNTS:
        assert kern.split("/")[0] in bench.KERNEL_SOURCES
        assert kern.split("/")[0] in bench.NCU_KERNEL_SHA256
    key = next(iter(bench.NCU_COUNTS))
    base = key[1].split("/")[0]
    monkeypatch.setitem(bench.NCU_KERNEL_SHA256, base, bench.kernel_source_sha256(base))
    assert bench.ncu_counts(*key) == bench.NCU_COUNTS[key]
    # a source change (another hash) drops the counts from the line
    monkeypatch.setitem(bench.NCU_KERNEL_SHA256, base, "0" * 64)
    assert bench.ncu_counts(*key) is None
    assert bench.launch_traffic(*key) is None
