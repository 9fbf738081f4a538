"""The named workload presets: five configurations with the parameters the benchmark and the tests
use, and the benchmark reads its house workload from them."""
import os
import sys

from paper_1801_08361_gb300 import presets

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_five_presets_with_consistent_parameters():
    assert set(presets.ALL) == {"tiny", "house", "fragments", "learned", "serving"}
    for w in presets.ALL.values():
        assert w.world in ("room", "house")
        assert 1 <= w.trees <= 16 and 1 <= w.depth <= 16 and 1 <= w.max_modes <= 64
        assert all(1 <= k <= 4096 for k in w.hypotheses)
        assert all(wd % 8 == 0 and ht % 8 == 0 for wd, ht in w.sizes)
    assert presets.HOUSE.sizes == ((640, 480),) and presets.HOUSE.hypotheses == (1024,)
    assert presets.FRAGMENTS.extra["pairs"] == presets.FRAGMENTS.extra["fragments"] * 7


def test_the_benchmark_reads_the_house_preset():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    h = presets.HOUSE
    assert (bench.W, bench.H) == h.sizes[0]
    assert (bench.T_TREES, bench.DEPTH, bench.MAX_MODES, bench.CAPACITY) == (h.trees, h.depth, h.max_modes,
                                                                              h.reservoir)
    assert (bench.K_HYPS, bench.B_PIX) == (h.hypotheses[0], h.batch_pixels)
