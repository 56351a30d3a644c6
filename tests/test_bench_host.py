"""Host logic of bench.py, without a GPU: the clock record parsed from nvidia-smi, the
ncu counters taken from the committed summary only when it was made on the current
kernel sources, and the roofline peak."""
import os
import shutil

import bench

SMI = """0, 2070, 2070, 905.2, 96, Not Active, Not Active, Not Active, Active
0, 2055, 2070, 910.0, 97, Not Active, Not Active, Not Active, Not Active
0, 2070, 2070, 915.0, 99, Not Active, Not Active, Not Active, Not Active
0, 1200, 2070, 120.0, 0, Active, Not Active, Not Active, Not Active
a line that is not a sample
"""


def test_clock_record():
    r = bench.ClockSampler.parse(SMI)
    # the idle sample (utilisation 0) is left out of the median and of the reasons
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    assert bench.ClockSampler.parse("")["sm_mhz"] is None
    idle = bench.ClockSampler.parse("0, 1200, 2070, 120.0, 0, Active, Not Active, Not Active, Not Active")
    assert idle["samples"] == 1 and idle["reasons"] == ["hw_slowdown"]


def test_counters_only_for_the_current_sources(tmp_path, monkeypatch):
    note = tmp_path / "note.md"
    note.write_text(f"source_sha256_16: {bench.source_sha()}\n"
                    "traffic_bytes_per_launch_full_batch: 336855040\n"
                    "warp_instructions_per_launch_full_batch: 229898784 (8.3 per pixel)\n")
    monkeypatch.setattr(bench, "PROFILE_NOTE", str(note))
    assert bench.committed_traffic() == 336855040.0
    assert bench.committed_counter("warp_instructions_per_launch_full_batch") == 229898784.0
    assert bench.committed_counter("no_such_counter") is None
    note.write_text("source_sha256_16: 0123456789abcdef\n"
                    "traffic_bytes_per_launch_full_batch: 336855040\n")
    assert bench.committed_traffic() is None  # taken on other sources
    monkeypatch.setattr(bench, "PROFILE_NOTE", str(tmp_path / "absent.md"))
    assert bench.committed_traffic() is None


def test_source_hash_follows_the_kernel_sources(tmp_path, monkeypatch):
    d = tmp_path / "csrc"
    d.mkdir()
    for fn in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(bench.CSRC, fn), d / fn)
    monkeypatch.setattr(bench, "CSRC", str(d))
    h0 = bench.source_sha()
    assert len(h0) == 16
    f = d / bench.KERNEL_SOURCES[-1]
    f.write_text(f.read_text() + "\n")
    assert bench.source_sha() != h0


def test_peak():
    peak, kind = bench.load_peak()
    assert kind in ("measured", "fallback") and 1000.0 < peak < 20000.0


def test_fp64_flip_count_structure_and_bound():
    """The bench's FP64 flip record: per set the candidate pairs, the flips and the largest
    |D - delta| of a flip, every flip within the 1e-5 m bound."""
    import oracle
    import bench
    from paper_2003_00575_gb300 import synth
    fr = synth.config_c4(3)
    r = bench.fp64_flip_count(oracle, synth, fr)
    assert r["c4"]["frames"] == 3 and r["c4"]["pairs"] > 0
    for name in ("c1", "c2", "c3", "c4"):
        rec = r[name]
        assert 0 <= rec["flips"] <= rec["pairs"]
        assert rec["flips"] == 0 or rec["max_abs_d_minus_delta_m"] < r["bound_m"]
