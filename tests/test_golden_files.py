"""The stored stepped states under tests/golden/ are the current oracle's, from the stated
inputs: each file records the SHA-256 of the oracle source that wrote it (re-run
tests/golden/make_stepped.py after any change to oracle/zm_oracle.c or zm_oracle.h), and its
initial heights are the seeded multi-mode interface of its description."""
import importlib.util
import json
import os

import numpy as np
import pytest

from paper_2406_05490_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _maker():
    spec = importlib.util.spec_from_file_location("make_stepped", os.path.join(GOLDEN, "make_stepped.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", ["multimode256_20", "multimode512_1"])
def test_stored_state_is_the_current_oracles(name):
    mk = _maker()
    d = np.load(mk.path_of(name))
    meta = json.loads(str(d["meta"]))
    assert meta["oracle_sha256"] == mk.oracle_source_sha256(), \
        "the oracle changed since this file was written: run tests/golden/make_stepped.py"
    case = mk.CASES[name]
    for k in ("n", "n_modes", "seed", "amp", "atwood", "steps"):
        assert meta[k] == case[k]
    z0, _ = mk.initial_state(case)
    # the seeded recipe reproduces the stored initial heights (up to the last bit of numpy's cos)
    assert np.max(np.abs(d["z3_0"] - z0[2])) <= 1e-15
    n = case["n"]
    assert d["z"].shape == (3, n * n) and d["w"].shape == (2, n * n)
    assert np.all(np.isfinite(d["z"])) and np.all(np.isfinite(d["w"]))
    # the interface moved, and the vorticity grew from zero
    assert 0 < np.max(np.abs(d["z"][2] - d["z3_0"])) < 0.1 and np.max(np.abs(d["w"])) > 0
