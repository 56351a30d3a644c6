"""Autotuner host logic (no GPU): the search space, workload signatures, the JSON cache."""
from paper_2003_00575_gb300 import autotune


def test_configs_cover_space_default_first():
    cs = autotune.configs()
    n = 1
    for v in autotune.SPACE.values():
        n *= len(v)
    assert len(cs) == n and cs[0] == autotune.DEFAULT
    assert len({tuple(sorted(c.items())) for c in cs}) == n


def test_signature_depends_on_mix_not_order():
    a = autotune.signature([(16, 1800, 1), (64, 2048, 3), (16, 1800, 1)], "GB300")
    b = autotune.signature([(64, 2048, 3), (16, 1800, 1), (16, 1800, 1)], "GB300")
    c = autotune.signature([(64, 2048, 3), (16, 1800, 1)], "GB300")
    d = autotune.signature([(16, 1800, 1), (64, 2048, 3), (16, 1800, 1)], "other")
    assert a == b and a != c and a != d


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "t.json")
    assert autotune.load("k", p) is None
    autotune.save("k", {"config": {"px_per_cta": 8192}, "ms": 1.0}, p)
    autotune.save("j", {"config": {"px_per_cta": 32768}, "ms": 2.0}, p)
    assert autotune.load("k", p)["config"]["px_per_cta"] == 8192
    assert autotune.load("j", p)["ms"] == 2.0
