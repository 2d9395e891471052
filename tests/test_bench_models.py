"""Host-side pieces of the benchmark: the flop models and the rule that the
recorded DRAM traffic is reported only for the kernel sources it was
captured with (no GPU needed)."""
import bench


def test_iteration_model_counts():
    """Per candidate 30 + 3 d N^3, per iteration 2(6N^3 + 9N^2 + 12N) + 30N + 60
    (at N = 5, d = 3: 1155 and 2280)."""
    assert bench.iteration_model_flops(1, 0, 5, 3) == 30 + 9 * 125
    assert bench.iteration_model_flops(0, 1, 5, 3) == 2 * (750 + 225 + 60) + 150 + 60 == 2280


def test_boxes_flops_hex():
    """Hexes: 6 faces x 3 coordinates x 2 box kinds x (lower + upper) x N^2 M^2
    FMAs of 2 flops."""
    assert bench.boxes_flops(1, 5, 10, 3, 3) == 6 * 3 * 2 * 2 * 2 * 25 * 100


def test_traffic_tied_to_sources(monkeypatch):
    sha = bench.source_sha("k_find_f64")
    monkeypatch.setitem(bench.TRAFFIC, "k_find_f64", {"sha": sha, "bytes": 123})
    assert bench.traffic_of("k_find_f64")[0] == 123
    monkeypatch.setitem(bench.TRAFFIC, "k_find_f64", {"sha": "0" * 16, "bytes": 123})
    assert bench.traffic_of("k_find_f64")[0] is None
