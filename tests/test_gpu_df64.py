"""Low order in double-word arithmetic (ZM_PREC_DF64: every stencil, FFT and RK3 operation on
FP32 pairs, ~48-bit significand) against the CPU oracle, through the C ABI.

Tolerances (relative L2 per field), derived from the arithmetic; u^2 = 2^-48 is the unit
roundoff of a double word:
  u: 1e-12.  The FFT's error is normwise, ~u^2 log2(n) (measured <= 6e-14 up to 2048^2).
  dw/dt: max(1e-12, (4 + 2 log2 N) u^2 0.95 n / 2 pi + 4 u^2 4.4 mu n^2 |w| / |dw/dt|),
    n = the larger side, N = n1 n2.  Phi and w are stored and formed with ~4 u^2 relative
    rounding per node, and Phi holds |u|^2 / 2, whose relative error is twice the velocity's:
    the FFT's normwise ~u^2 log2 N (measured 1.2-1.8 u^2 log2 N); these errors vary from node to
    node, and the 4th-order first difference amplifies such noise by its coefficient norm
    0.95 / dx = 0.95 n (relative to |D Phi| >= 2 pi |Phi| for the lowest mode), the Laplacian
    (two axes) by 4.4 / dx^2.  So at 4096^2 the bound is ~1e-10 where the FP64 path stays at
    1e-12: 48 bits are 5 fewer than FP64's 53, and the long stencil axis multiplies them.
  stepped state: 1e-12 on z and w, 1e-10 on the displacement z - z0 (as for the FP64 path).
z1 and z2 are stored relative to the mesh coordinates, so the amplification acts on the
perturbation, not on the coordinate.
"""
import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12
U2 = 2.0 ** -48


def wdot_tol(n, mu, w, wd_ref):
    N = w.shape[-1]
    ratio = np.linalg.norm(w) / max(np.linalg.norm(wd_ref), 1e-300)
    return max(TOL, (4 + 2 * np.log2(N)) * U2 * 0.95 * n / (2 * np.pi) + 4 * U2 * 4.4 * mu * n * n * ratio)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def zm():
    import torch
    from paper_2406_05490_gb300 import zm as _zm
    assert torch.cuda.is_available()
    _zm.load()
    return _zm


@pytest.mark.parametrize("n1,n2,mu", [(8, 8, 0.0), (64, 32, 0.0), (128, 128, 0.01), (16, 256, 0.0),
                                      (256, 64, 0.003), (32, 8, 0.0),
                                      # sides R 2^A: every odd factor R = 3 .. 19 once, A = 3 .. 11
                                      (24, 40, 0.0), (56, 72, 0.01), (88, 104, 0.0), (120, 136, 0.0),
                                      (152, 16, 0.0), (96, 320, 0.003), (608, 152, 0.0), (6144, 8, 0.0),
                                      (8, 6144, 0.0),
                                      # columns of 2048: the Hermitian inverse (pass B_h / C_h)
                                      (2048, 16, 0.0), (2048, 64, 0.01)])
def test_df64_velocity_parity(zm, n1, n2, mu):
    z, w = inputs.random_state(n1, n2, seed=n1 + 2 * n2)
    m = oracle.Mesh(n1, n2, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.7, 1.3, mu, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.7, g=1.3, mu=mu, order=zm.ZM_ORDER_LOW, df64=True)
    u, wd = model.velocity(z, w)
    # the resident-state form of the same call
    model.set_state(z, w)
    u2, wd2 = model.velocity()
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    tw = wdot_tol(max(n1, n2), mu, w, wd_ref)
    print(f"df64 low order {n1}x{n2} mu={mu}: rel L2 u={eu:.3e} wdot={ew:.3e} (bound {tw:.1e})")
    assert eu <= TOL and ew <= tw
    assert np.array_equal(u, u2) and np.array_equal(wd, wd2)


def test_df64_non_unit_domain(zm):
    n1, n2 = 64, 128
    L1, L2 = 2.0, 0.75
    a = np.repeat(np.arange(n1) * (L1 / n1), n2)
    b = np.tile(np.arange(n2) * (L2 / n2), n1)
    z = np.stack([a + 0.02 * np.sin(2 * np.pi * b / L2), b, 0.03 * np.cos(2 * np.pi * (a / L1 + 2 * b / L2))])
    w = np.stack([0.2 * np.sin(2 * np.pi * 3 * a / L1), 0.1 * np.cos(2 * np.pi * b / L2)])
    m = oracle.Mesh(n1, n2, L1=L1, L2=L2, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n1, n2, L1=L1, L2=L2, periodic=True, atwood=0.5, g=1.0, order=zm.ZM_ORDER_LOW,
                      df64=True)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    tw = wdot_tol(max(n1, n2), 0.0, w, wd_ref)
    print(f"df64 L=({L1},{L2}): rel L2 u={eu:.3e} wdot={ew:.3e} (bound {tw:.1e})")
    assert eu <= TOL and ew <= tw


def test_df64_steps(zm):
    n = 64
    z0, w0 = inputs.multi_mode(n, n_modes=8, seed=3, amp=0.02)
    m = oracle.Mesh(n, periodic=True)
    zr, wr = oracle.run(m, z0, w0, 0.7, 1.0, 0.0, 0.0, 1e-3, 5, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW, df64=True)
    model.set_state(z0, w0)
    model.step(1e-3, 5)
    z1, w1 = model.get_state()
    model.close()
    ez, ew, dz = rel(z1, zr), rel(w1, wr), rel(z1 - z0, zr - z0)
    print(f"df64 5 steps 64^2: rel L2 z={ez:.3e} w={ew:.3e} (z - z0)={dz:.3e}")
    assert ez <= TOL and ew <= TOL and dz <= 1e-10


def test_df64_steps_viscous_rectangular(zm):
    n1, n2 = 32, 64
    z0, w0 = inputs.random_state(n1, n2, seed=17)
    m = oracle.Mesh(n1, n2, periodic=True)
    zr, wr = oracle.run(m, z0, w0, 0.4, 2.0, 0.005, 0.0, 5e-4, 4, order=oracle.ORDER_LOW)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.4, g=2.0, mu=0.005, order=zm.ZM_ORDER_LOW, df64=True)
    model.set_state(z0, w0)
    model.step(5e-4, 4)
    z1, w1 = model.get_state()
    model.close()
    ez, ew, dz = rel(z1, zr), rel(w1, wr), rel(z1 - z0, zr - z0)
    print(f"df64 4 viscous steps 32x64: rel L2 z={ez:.3e} w={ew:.3e} (z - z0)={dz:.3e}")
    assert ez <= TOL and ew <= TOL and dz <= 1e-10


def test_df64_1024_full(zm):
    n = 1024
    z, _ = inputs.multi_mode(n, n_modes=8, seed=7, amp=0.02)
    _, w = inputs.random_state(n, seed=13)
    m = oracle.Mesh(n, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.7, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW, df64=True)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    tw = wdot_tol(n, 0.0, w, wd_ref)
    print(f"df64 low order 1024^2: rel L2 u={eu:.3e} wdot={ew:.3e} (bound {tw:.1e})")
    assert eu <= TOL and ew <= tw


def test_df64_2048_full(zm):
    n = 2048
    z, _ = inputs.multi_mode(n, n_modes=8, seed=5, amp=0.02)
    _, w = inputs.random_state(n, seed=14)
    m = oracle.Mesh(n, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.7, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW, df64=True)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    tw = wdot_tol(n, 0.0, w, wd_ref)
    print(f"df64 low order 2048^2: rel L2 u={eu:.3e} wdot={ew:.3e} (bound {tw:.1e})")
    assert eu <= TOL and ew <= tw


def test_df64_state_roundtrip_and_finite_check(zm):
    n = 64
    z, w = inputs.random_state(n, seed=2)
    model = zm.ZModel(n, periodic=True, order=zm.ZM_ORDER_LOW, df64=True)
    model.set_state(z, w)
    z1, w1 = model.get_state()
    # stored as FP32 pairs: relative rounding 2^-48 of the displacement / field value
    a, b = inputs.mesh_coords(n)
    disp = np.abs(z - np.stack([a, b, 0 * a]))
    assert np.all(np.abs(z1 - z) <= 2.0 ** -47 * disp + 2.0 ** -52 * np.abs(z))
    assert np.all(np.abs(w1 - w) <= 2.0 ** -47 * np.abs(w))
    assert zm.zm_check_finite(model.h) == zm.ZM_OK
    w_bad = w.copy()
    w_bad[1, 77] = np.nan
    model.set_state(z, w_bad)
    assert zm.zm_check_finite(model.h) == zm.ZM_ERR_NONFINITE
    model.close()


def test_df64_graph_replay_equals_plain_launches(zm):
    n = 128
    z0, w0 = inputs.multi_mode(n, n_modes=4, seed=8, amp=0.02)
    out = []
    for prof in (False, True):
        model = zm.ZModel(n, periodic=True, atwood=0.6, order=zm.ZM_ORDER_LOW, df64=True)
        zm.zm_set_profiling(model.h, 1 if prof else 0)
        model.set_state(z0, w0)
        model.step(1e-3, 3)
        out.append(model.get_state())
        if prof:
            p = zm.zm_get_profile(model.h)
            assert p["launches"]["fft"] == 27 and p["launches"]["geometry"] == 9
        model.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_df64_4864_full(zm):
    """The paper's single-GPU low-order mesh and domain (Sec. 5.1): 4864^2 nodes over (-19, 19)^2
    (dx = 2^-7), all of u and dw/dt against the oracle within the double-word bounds."""
    n, L = 4864, 38.0
    zu, _ = inputs.multi_mode(n, n_modes=8, seed=9, amp=0.02)
    a, b = inputs.mesh_coords(n, n, L, L)
    z = np.stack([a, b, L * zu[2]])
    del zu
    _, w = inputs.random_state(n, seed=15)
    m = oracle.Mesh(n, n, L1=L, L2=L, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.7, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, L1=L, L2=L, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW, df64=True)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    tw = wdot_tol(n, 0.0, w, wd_ref)
    print(f"df64 low order 4864^2: rel L2 u={eu:.3e} wdot={ew:.3e} (bound {tw:.1e})")
    assert eu <= TOL and ew <= tw


def test_df64_steps_mixed_sides(zm):
    n1, n2 = 96, 152
    z0, w0 = inputs.random_state(n1, n2, seed=33)
    m = oracle.Mesh(n1, n2, periodic=True)
    zr, wr = oracle.run(m, z0, w0, 0.7, 1.0, 0.01, 0.0, 1e-3, 4, order=oracle.ORDER_LOW)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.7, g=1.0, mu=0.01, order=zm.ZM_ORDER_LOW, df64=True)
    model.set_state(z0, w0)
    model.step(1e-3, 4)
    z1, w1 = model.get_state()
    model.close()
    ez, ew, dz = rel(z1, zr), rel(w1, wr), rel(z1 - z0, zr - z0)
    print(f"df64 4 steps 96x152: rel L2 z={ez:.3e} w={ew:.3e} (z - z0)={dz:.3e}")
    assert ez <= TOL and ew <= TOL and dz <= 1e-10


def test_df64_flag_rules(zm):
    for n1, n2 in ((12, 16), (168, 64), (64, 44), (8192, 8)):
        with pytest.raises(zm.ZMError) as e:
            zm.zm_create(n1, n2, periodic=True, order=zm.ZM_ORDER_LOW | zm.ZM_PREC_DF64)
        assert e.value.code == zm.ZM_ERR_UNSUPPORTED
    with pytest.raises(zm.ZMError) as e:
        zm.zm_create(32, 32, periodic=True, delta=0.01, order=zm.ZM_ORDER_HIGH | zm.ZM_PREC_DF64)
    assert e.value.code == zm.ZM_ERR_UNSUPPORTED
    with pytest.raises(zm.ZMError) as e:
        zm.zm_create(32, 32, periodic=True, order=zm.ZM_ORDER_LOW | zm.ZM_PREC_DF64 | zm.ZM_PREC_FP32C)
    assert e.value.code == zm.ZM_ERR_INVALID
    with pytest.raises(zm.ZMError) as e:
        zm.zm_create(32, 32, periodic=False, order=zm.ZM_ORDER_LOW | zm.ZM_PREC_DF64)
    assert e.value.code == zm.ZM_ERR_UNSUPPORTED


@pytest.mark.parametrize("df64", [False, True])
def test_low_order_4096_full(zm, df64):
    """The largest FFT side (2^12), 16.8 M points: all of u and dw/dt against the oracle, for the
    FP64 path (1e-12) and the double-word path (its derived bound)."""
    n = 4096
    z, _ = inputs.multi_mode(n, n_modes=8, seed=11, amp=0.02)
    _, w = inputs.random_state(n, seed=15)
    m = oracle.Mesh(n, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.7, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW, df64=df64)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    tw = wdot_tol(n, 0.0, w, wd_ref) if df64 else TOL
    print(f"low order 4096^2 df64={df64}: rel L2 u={eu:.3e} wdot={ew:.3e} (bound {tw:.1e})")
    assert eu <= TOL and ew <= tw
