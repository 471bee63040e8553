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


def test_part_launch_groups():
    """The 2D experiments' launch groups: every setting once; the 100^2
    settings first, one stream each, longest expected chain (N_I = 1, blocks
    of 16) first; the 12^2 ones dealt over the requested streams, smallest
    N_I first on each."""
    STRIPES, BLOCKS = 1, 0
    settings = bench.part_settings(STRIPES, BLOCKS)
    assert len(settings) == 28
    for n_streams, n_short_groups in ((0, 12), (1, 1), (2, 2), (3, 3), (40, 12)):
        groups = bench.part_launch_groups(settings, BLOCKS, n_streams)
        flat = [i for g in groups for i in g]
        assert sorted(flat) == list(range(28))
        long_, short = groups[:16], groups[16:]
        assert all(len(g) == 1 and settings[g[0]][0] == 100 for g in long_)
        assert len(short) == n_short_groups
        assert all(settings[i][0] == 12 for g in short for i in g)
        for g in short:
            NI = [settings[i][5] for i in g]
            assert NI == sorted(NI)
        first = settings[long_[0][0]]
        assert (first[3], first[4], first[5]) == (BLOCKS, 16, 1)
        NI_long = [settings[g[0]][5] for g in long_]
        assert NI_long == sorted(NI_long)


def test_algorithmic_bytes_of_the_headline():
    """Per-visit bytes (L_d + 2)^2 - 4 + 32 k + 4 L_d at L_d = 32 and the
    headline's bytes per launch: 18 replicas of 1024^2, k in {1, 4, 16} six
    replicas each, two visits per domain and schedule, 1e4 schedules."""
    assert [bench.visit_bytes(32, k) for k in (1, 4, 16)] == [1312, 1408, 1792]
    L = [1024] * 18
    ks = [1, 4, 16] * 6
    per_schedule = bench.schedule_bytes(L, 32, ks)
    assert per_schedule == 2 * 1024 * 6 * (1312 + 1408 + 1792)
    assert per_schedule * 10000 == 554434560000
