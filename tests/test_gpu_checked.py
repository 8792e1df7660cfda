"""The checked build (libzm_checked.so, ZM_CHECKS=1) in place of compute-sanitizer, which this
project does not rely on: every kernel tests the indices it computes (neighbour wraps, tile and
record numbers, transposed writes, shared-memory positions) and counts violations instead of
making the access.

Each kernel family runs on small cases (FP64 and FP32C high order, cutoff, anisotropic tiles,
low order on power-of-two and R 2^a sides in FP64 and double words, medium order, a ragged
batch, the serving loop, the allocation-free sum) once with the default build and once with the
checked build, each in a process of its own.  The checked build must count no violation and
produce the default build's results bit for bit: the tests add branches, not arithmetic.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run_cases(tmp_path, variant):
    out = str(tmp_path / f"{variant}.npz")
    env = dict(os.environ)
    env.pop("ZM_LIB", None)
    if variant == "checked":
        env["ZM_LIB"] = "checked"
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    print(r.stdout[-2000:], r.stderr[-2000:])
    assert r.returncode == 0
    return dict(np.load(out))


def test_checked_build_counts_no_violation_and_matches(tmp_path):
    from paper_2406_05490_gb300 import build
    assert os.path.exists(build.LIB_CHECKED), "libzm_checked.so is built by __graft_entry__.build()"
    plain = run_cases(tmp_path, "plain")
    chk = run_cases(tmp_path, "checked")
    assert plain["checked"][0] == 0 and chk["checked"][0] == 1
    assert plain["hits"][0] == 0
    hits, first, line = (int(v) for v in chk["hits"])
    assert hits == 0, f"checked build: {hits} index violations, first index {first} at line {line}"
    keys = sorted(k for k in plain if k not in ("checked", "hits"))
    assert keys == sorted(k for k in chk if k not in ("checked", "hits"))
    for k in keys:
        assert np.all(np.isfinite(plain[k])), k
        assert np.array_equal(plain[k], chk[k]), k
