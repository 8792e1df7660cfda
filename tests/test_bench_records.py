"""The committed ncu records that feed bench.py's JSON line still describe the current kernel
sources.  Each record carries a hash of the sources it was counted on; a record whose sources
changed is dropped by the bench (its figure then reads null), so a kernel edit without a new
capture would silently blank the FP64-pipe fractions or the roofline traffic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_fp64_instruction_record_matches_the_sources():
    rec = bench.fp64_inst_record()
    assert set(rec) == {"geometry", "fft", "vorticity", "br64"}
    counts, kind = rec["fft"]
    assert kind == "by_side"
    # the low-order sizes the bench reports, each with its own count; longer transforms and a
    # radix-19 stage cost more FP64 instructions per point
    assert set(counts) == {1024, 4096, 4864}
    assert counts[1024] < counts[4096] < counts[4864]
    for k in ("geometry", "vorticity", "br64"):
        assert rec[k][1] is None and rec[k][0] > 0


def test_traffic_record_matches_the_headline_kernel():
    t = bench.recorded_traffic((16, 16))
    assert t is not None and t > 0
    assert bench.recorded_traffic((8, 32)) is None  # another tile shape was not captured


def test_double_word_instruction_record_matches_the_sources():
    rec = bench.df64_issue_record()
    assert set(rec) == {"geometry", "fft", "vorticity"}
    for k, by_side in rec.items():
        assert set(by_side) == {1024, 4096, 4864} and all(v > 0 for v in by_side.values())
    # the transforms grow with log2 of the side and the radix-19 stage of 4864 = 19 x 256
    assert rec["fft"][1024] < rec["fft"][4096] < rec["fft"][4864]
