"""Cutoff Birkhoff-Rott sum (sources within a 3D distance only) against the CPU oracle, which
takes the same in/out decision per pair in FP32.  Tolerances: u 1e-6 relative L2 (the FP32C
velocity bound); dw/dt 1e-5, because it differentiates |u|^2 / 2 and the per-target cut makes
the FP32 rounding of neighbouring targets' velocities uncorrelated, which the fourth-order
stencil amplifies by about 1.5 / dx (~100 here) relative to the smooth exact-sum case.
A cutoff larger than the interface gives the exact sum bit for bit; per-interface cutoffs in
a batch equal the same cutoffs alone, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = 1e-6
TOL32_RATE = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def zm():
    import torch
    from paper_2406_05490_gb300 import zm as _zm
    assert torch.cuda.is_available()
    _zm.load()
    return _zm


@pytest.mark.parametrize("n1,n2,periodic,cutoff", [(96, 80, True, 0.15), (64, 64, False, 0.4),
                                                   (48, 48, True, 0.06)])
def test_cutoff_parity(zm, n1, n2, periodic, cutoff):
    z, w = inputs.random_state(n1, n2, seed=n1 + n2)
    delta = 0.1 / max(n1, n2)
    m = oracle.Mesh(n1, n2, periodic=periodic)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, delta, cutoff=cutoff)
    u_ex, _ = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, delta)
    model = zm.ZModel(n1, n2, periodic=periodic, atwood=0.5, g=1.0, delta=delta, fp32c=True)
    zm.zm_set_cutoff(model.h, cutoff)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"cutoff {cutoff} {n1}x{n2}: rel L2 u={eu:.3e} wdot={ew:.3e}; "
          f"cutoff vs exact sum {rel(u_ref, u_ex):.3e}")
    assert eu <= TOL32 and ew <= TOL32_RATE


def test_large_cutoff_is_exact_and_batch_matches_alone(zm):
    n = 64
    z, w = inputs.random_state(n, seed=9)
    model = zm.ZModel(n, periodic=True, fp32c=True)
    u_exact, _ = model.velocity(z, w)
    zm.zm_set_cutoff(model.h, 10.0)
    u_big, _ = model.velocity(z, w)
    zm.zm_set_cutoff(model.h, 0.2)
    u_cut, _ = model.velocity(z, w)
    model.close()
    assert np.array_equal(u_big, u_exact) and not np.array_equal(u_cut, u_exact)
    # per-interface cutoffs inside a batch
    h = zm.zm_batch_create([(n, n, 1.0, 1.0, True), (48, 40, 1.0, 1.0, True)], [0.5, 0.5])
    zm.zm_batch_set_state(h, 0, z, w)
    z2, w2 = inputs.random_state(48, 40, seed=4)
    zm.zm_batch_set_state(h, 1, z2, w2)
    zm.zm_batch_set_cutoff(h, 0, 0.2)
    zm.zm_batch_velocity(h)
    u0 = np.empty((3, n * n))
    u1 = np.empty((3, 48 * 40))
    zm.zm_batch_get_velocity(h, 0, u0, None)
    zm.zm_batch_get_velocity(h, 1, u1, None)
    zm.zm_batch_destroy(h)
    assert np.array_equal(u0, u_cut)
    alone = zm.ZModel(48, 40, periodic=True, fp32c=True)
    u1a, _ = alone.velocity(z2, w2)
    alone.close()
    assert np.array_equal(u1, u1a)


def test_cutoff_needs_fp32c(zm):
    model = zm.ZModel(32, periodic=True, fp32c=False)
    with pytest.raises(zm.ZMError) as e:
        zm.zm_set_cutoff(model.h, 0.2)
    assert e.value.code == zm.ZM_ERR_UNSUPPORTED
    model.close()
