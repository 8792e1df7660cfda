"""Full-size stepped parity of the benchmarked configurations against the CPU oracle.

* 256^2 multi-mode interface, high order, 20 SSP-RK3 steps: FP32C in the benchmark's launch
  configuration (tile shape and work-item size autotuned on the same interface first, exactly as
  bench.py does), the same with the far tile pairs on the tensor cores, and FP64.  Reference: the oracle's final state, stored by
  tests/golden/make_stepped.py (which calls only the oracle).
* 512^2 8-mode interface (amplitude 0.02, A = 0.7), high order, FP32C, one step, autotuned as in
  the benchmark; reference stored the same way.
* 1024^2 8-mode interface, low order (FFT Riesz velocity), FP64, 10 steps; the oracle runs here.

Tolerances, relative L2 per field: FP64 1e-12; FP32C 1e-6.  Besides z and w the displacement
z - z0 is compared on its own: z itself is dominated by the mesh coordinates, while z - z0 is the
time integral of the velocity, so it carries the velocity's relative error undiluted.  Its
bound is the larger of the field tolerance and the rounding floor of the state: every stage
update rounds z (|z| ~ 1) to FP64 in each code, in different operation orders, so after s steps
(3 s roundings, a random walk) z - z0 differs by about sqrt(3 s) eps |z| per node whatever the
velocity's accuracy; relative to |z - z0| (about 1e-4 of |z| here) that is ~3e-12 after 20
steps.  The bound takes 2.5 sqrt(3 s) eps ||z|| / ||z - z0||.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def zm():
    import torch
    from paper_2406_05490_gb300 import zm as _zm
    assert torch.cuda.is_available()
    _zm.load()
    return _zm


def load_golden(name):
    d = np.load(os.path.join(GOLDEN, f"stepped_{name}.npz"))
    meta = json.loads(str(d["meta"]))
    n = meta["n"]
    a, b = inputs.mesh_coords(n)
    z0 = np.stack([a, b, d["z3_0"]])
    w0 = np.zeros((2, n * n))
    return meta, z0, w0, d["z"], d["w"]


def step_on_gpu(zm, meta, z0, w0, fp32c, autotune, far_path=None):
    n = meta["n"]
    model = zm.ZModel(n, periodic=True, atwood=meta["atwood"], g=meta["g"], mu=meta["mu"],
                      delta=meta["delta"], fp32c=fp32c)
    if far_path is not None:
        zm.zm_set_far_path(model.h, far_path)
    if autotune:
        # as the benchmark: tune on the interface with vorticity, then reset it
        model.set_state(z0, inputs.random_state(n, seed=1)[1])
        zm.zm_autotune_tiles(model.h)
    model.set_state(z0, w0)
    model.step(meta["dt"], meta["steps"])
    z, w = model.get_state()
    model.close()
    return z, w


def compare(label, z, w, z0, zr, wr, tol, steps):
    ez, ed, ew = rel(z, zr), rel(z - z0, zr - z0), rel(w, wr)
    floor = 2.5 * np.sqrt(3 * steps) * 2.0**-53 * np.linalg.norm(zr) / np.linalg.norm(zr - z0)
    print(f"{label}: rel L2 z={ez:.3e} z-z0={ed:.3e} (bound {max(tol, floor):.1e}) w={ew:.3e}")
    assert ez <= tol and ed <= max(tol, floor) and ew <= tol


@pytest.mark.parametrize("fp32c", [True, False])
def test_multimode_256_twenty_steps(zm, fp32c):
    meta, z0, w0, zr, wr = load_golden("multimode256_20")
    z, w = step_on_gpu(zm, meta, z0, w0, fp32c, autotune=fp32c)
    compare(f"256^2 x 20 steps fp32c={fp32c}", z, w, z0, zr, wr, TOL32 if fp32c else TOL64, meta["steps"])


def test_multimode_256_twenty_steps_tensor_far_path(zm):
    """The same 20 steps with the far tile pairs summed on the tensor cores (opt-in path)."""
    meta, z0, w0, zr, wr = load_golden("multimode256_20")
    z, w = step_on_gpu(zm, meta, z0, w0, True, autotune=True, far_path=zm.ZM_FAR_TENSOR)
    compare("256^2 x 20 steps fp32c, tensor-core far path", z, w, z0, zr, wr, TOL32, meta["steps"])


def test_multimode_512_one_step_fp32c(zm):
    meta, z0, w0, zr, wr = load_golden("multimode512_1")
    z, w = step_on_gpu(zm, meta, z0, w0, True, autotune=True)
    compare("512^2 x 1 step fp32c", z, w, z0, zr, wr, TOL32, meta["steps"])


def test_low_order_1024_ten_steps():
    from paper_2406_05490_gb300 import zm
    n, steps = 1024, 10
    z0, w0 = inputs.multi_mode(n, n_modes=8, seed=7, amp=0.02)
    m = oracle.Mesh(n, periodic=True)
    zr, wr = oracle.run(m, z0, w0, 0.7, 1.0, 0.0, 0.0, 1e-3, steps, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW)
    model.set_state(z0, w0)
    model.step(1e-3, steps)
    z, w = model.get_state()
    model.close()
    compare("low order 1024^2 x 10 steps fp64", z, w, z0, zr, wr, TOL64, steps)
