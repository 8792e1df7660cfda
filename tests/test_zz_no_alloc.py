"""zm_br_velocity_noalloc: the FP64 Birkhoff-Rott sum for callers that cannot allocate GPU
memory (it uses a static workspace inside the library instead of cudaMalloc).

Checked directly against the oracle's all-pairs sum at 1e-12 relative L2 (the FP64 bound), and
against the allocating entry point zm_velocity, on calls in a row: sizes that end in a ragged
tile, the workspace limit n = 65536 (every record and partial-sum slot in use) and n = 65535,
each followed by a smaller call, so that stale workspace contents from a larger call would show
up in the next one.

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


def scaled_strength(n1, n2, z, w, periodic):
    """The oracle's sheet strength gamma = w1 a2 - w2 a1 and its scaled form
    (dx1 dx2 / 4 pi) gamma that the entry point takes."""
    m = oracle.Mesh(n1, n2, periodic=periodic)
    a1, a2, _, _ = oracle.geometry(m, z)
    gam = oracle.sheet_strength(w, a1, a2)
    weight = (1.0 / n1) * (1.0 / n2)
    return gam, gam * (weight / (4 * np.pi)), weight


def call_noalloc(zm, torch, z, gam_scaled, delta):
    n = z.shape[1]
    zd = torch.from_numpy(np.ascontiguousarray(z)).cuda()
    gd = torch.from_numpy(np.ascontiguousarray(gam_scaled)).cuda()
    ud = torch.full((3, n), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    zm.zm_br_velocity_noalloc(n, zd, gd, delta, ud, st, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(st.item()) == zm.ZM_OK
    return ud.cpu().numpy()


def test_noalloc_matches_oracle_and_zm_velocity_on_two_calls():
    import torch
    from paper_2406_05490_gb300 import zm
    assert torch.cuda.is_available()
    for n1, n2, periodic, seed in ((64, 64, True, 1), (37, 53, False, 2)):
        z, w = inputs.random_state(n1, n2, seed=seed)
        delta = 0.1 / max(n1, n2)
        gam, gam_s, weight = scaled_strength(n1, n2, z, w, periodic)
        u = call_noalloc(zm, torch, z, gam_s, delta)
        u_oracle = oracle.br_velocity(z, z, gam, weight, delta)
        # the allocating entry point: full derivative, velocity from the geometry pass + BR
        model = zm.ZModel(n1, n2, periodic=periodic, delta=delta)
        u_ref = model.velocity(z, w, want_wdot=False)
        model.close()
        e_or, e_zm = rel(u, u_oracle), rel(u, u_ref)
        print(f"noalloc {n1}x{n2} (n = {n1 * n2}): rel L2 vs oracle {e_or:.3e}, vs zm_velocity {e_zm:.3e}")
        assert e_or <= TOL64 and e_zm <= TOL64


def test_noalloc_at_the_workspace_limit_then_smaller():
    """n = 65536 fills every record and partial-sum slot of the workspace, n = 65535 leaves one
    padding slot in the last tile; each is followed by a smaller ragged call.  Full-size results
    are checked against the oracle on 512 seeded targets (all sources) and, for the full mesh,
    against zm_velocity everywhere."""
    import torch
    from paper_2406_05490_gb300 import zm
    n1 = n2 = 256
    z, w = inputs.random_state(n1, n2, seed=5)
    delta = 0.1 / n1
    gam, gam_s, weight = scaled_strength(n1, n2, z, w, True)
    idx_all = np.random.default_rng(0).choice(n1 * n2 - 1, 512, replace=False)
    zs, ws = inputs.random_state(41, 47, seed=6)
    gs, gs_s, wts = scaled_strength(41, 47, zs, ws, False)
    us_oracle = oracle.br_velocity(zs, zs, gs, wts, 0.1 / 47)
    for n in (65536, 65535):
        zc, gc, gsc = z[:, :n], gam[:, :n], gam_s[:, :n]
        u = call_noalloc(zm, torch, zc, gsc, delta)
        u_or = oracle.br_velocity(zc[:, idx_all], zc, gc, weight, delta)
        e_or = rel(u[:, idx_all], u_or)
        msg = f"noalloc n = {n}: rel L2 on 512 targets vs oracle {e_or:.3e}"
        if n == n1 * n2:
            model = zm.ZModel(n1, n2, periodic=True, delta=delta)
            u_ref = model.velocity(z, w, want_wdot=False)
            model.close()
            e_zm = rel(u, u_ref)
            msg += f", everywhere vs zm_velocity {e_zm:.3e}"
            assert e_zm <= TOL64
        assert e_or <= TOL64
        # the next, smaller call on the same workspace
        us = call_noalloc(zm, torch, zs, gs_s, 0.1 / 47)
        e_s = rel(us, us_oracle)
        print(msg + f"; next call n = {41 * 47}: vs oracle {e_s:.3e}")
        assert e_s <= TOL64


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
    # buffers shorter than 3 n, and a status word of the wrong type, are refused by the binding
    with pytest.raises(zm.ZMError) as e:
        zm.zm_br_velocity_noalloc(9, d, d, 0.01, d)
    assert e.value.code == zm.ZM_ERR_INVALID
    with pytest.raises(zm.ZMError) as e:
        zm.zm_br_velocity_noalloc(8, d, d, 0.01, d, torch.zeros(1, dtype=torch.int64, device="cuda"))
    assert e.value.code == zm.ZM_ERR_INVALID
    # the same sizes through raw addresses reach the C ABI, which still rejects a bad n
    with pytest.raises(zm.ZMError) as e:
        zm.zm_br_velocity_noalloc(-1, d.data_ptr(), d.data_ptr(), 0.01, d.data_ptr())
    assert e.value.code == zm.ZM_ERR_INVALID
