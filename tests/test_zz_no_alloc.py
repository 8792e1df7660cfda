"""zm_br_velocity_noalloc: the FP64 Birkhoff-Rott sum for callers that cannot allocate GPU
memory (it uses a static workspace inside the library instead of cudaMalloc).  Checked against
the allocating entry point zm_velocity on two calls in a row; the second call is smaller and
ends in a ragged tile, so stale workspace contents from the first call would show up.

This file is collected last on purpose (tests/test_zz_*): if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_matches_zm_velocity_on_two_calls():
    import torch
    from paper_2406_05490_gb300 import zm
    assert torch.cuda.is_available()
    stream = torch.cuda.current_stream()
    for n1, n2, periodic, seed in ((64, 64, True, 1), (37, 53, False, 2)):
        z, w = inputs.random_state(n1, n2, seed=seed)
        delta = 0.1 / max(n1, n2)
        N = n1 * n2
        # the allocating entry point: full derivative, velocity from the geometry pass + BR
        model = zm.ZModel(n1, n2, periodic=periodic, delta=delta)
        u_ref = model.velocity(z, w, want_wdot=False)
        model.close()
        # the caller prepares the scaled sheet strengths (dx1 dx2 / 4 pi)(w1 a2 - w2 a1)
        m = oracle.Mesh(n1, n2, periodic=periodic)
        a1, a2, _, _ = oracle.geometry(m, z)
        gam = oracle.sheet_strength(w, a1, a2) * ((1.0 / n1) * (1.0 / n2) / (4 * np.pi))
        zd = torch.from_numpy(np.ascontiguousarray(z)).cuda()
        gd = torch.from_numpy(np.ascontiguousarray(gam)).cuda()
        ud = torch.full((3, N), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        zm.zm_br_velocity_noalloc(N, zd, gd, delta, ud, st, stream.cuda_stream)
        torch.cuda.synchronize()
        assert int(st.item()) == zm.ZM_OK
        e = rel(ud.cpu().numpy(), u_ref)
        print(f"noalloc {n1}x{n2}: rel L2 vs zm_velocity {e:.3e}")
        assert e <= TOL64


def test_noalloc_rejects_bad_sizes_and_host_pointers():
    import torch
    from paper_2406_05490_gb300 import zm
    d = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(zm.ZMError) as e:
        zm.zm_br_velocity_noalloc(65537, d, d, 0.01, d)
    assert e.value.code == zm.ZM_ERR_INVALID
    with pytest.raises(zm.ZMError) as e:
        zm.zm_br_velocity_noalloc(0, d, d, 0.01, d)
    assert e.value.code == zm.ZM_ERR_INVALID
    h = np.zeros((3, 8))
    with pytest.raises(zm.ZMError) as e:
        zm.zm_br_velocity_noalloc(8, h, d, 0.01, d)
    assert e.value.code == zm.ZM_ERR_INVALID
