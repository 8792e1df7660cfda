"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on seeded inputs.

Tolerances (relative L2 per field, ||x_gpu - x_ref|| / ||x_ref|| over all nodes and components):
  FP64 path: 1e-12 for u, dw/dt and the stepped state.
  FP32C path (FP32 Birkhoff-Rott pair terms): 1e-6 for u; dw/dt and the stepped state are
  reported per field and bounded by the same 1e-6 (they inherit u's error through Phi).
"""
import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def zm():
    import torch
    from paper_2406_05490_gb300 import zm as _zm
    assert torch.cuda.is_available()
    _zm.load()
    return _zm


SHAPES = [(16, 16, False), (32, 32, False), (48, 40, True), (37, 53, False), (64, 64, True),
          (5, 7, False), (96, 80, True)]


@pytest.mark.parametrize("n1,n2,periodic", SHAPES)
@pytest.mark.parametrize("fp32c", [False, True])
def test_velocity_parity(zm, n1, n2, periodic, fp32c):
    z, w = inputs.random_state(n1, n2, seed=n1 * 7 + n2)
    A, g, mu = 0.4, 1.3, (0.01 if periodic else 0.0)
    delta = 0.1 / max(n1, n2)
    m = oracle.Mesh(n1, n2, periodic=periodic)
    u_ref, wd_ref = oracle.derivative(m, z, w, A, g, mu, delta)
    model = zm.ZModel(n1, n2, periodic=periodic, atwood=A, g=g, mu=mu, delta=delta, fp32c=fp32c)
    u, wd = model.velocity(z, w)
    model.close()
    tol = TOL32 if fp32c else TOL64
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"n={n1}x{n2} periodic={periodic} fp32c={fp32c}: rel L2 u={eu:.3e} wdot={ew:.3e}")
    assert eu <= tol and ew <= tol


def test_flat_rest_exact(zm):
    n = 32
    a, b = inputs.mesh_coords(n)
    z = np.stack([a, b, 0 * a])
    w = np.zeros((2, n * n))
    for fp32c in (False, True):
        model = zm.ZModel(n, periodic=False, fp32c=fp32c)
        u, wd = model.velocity(z, w)
        model.close()
        assert np.all(u == 0.0) and np.all(wd == 0.0)


@pytest.mark.parametrize("fp32c", [False, True])
def test_single_mode_steps_config1(zm, fp32c):
    """32 x 32 single-mode interface, free edges, A = 0.5, g = 1, delta = 0.1 dx, dt = 1e-3,
    10 SSP-RK3 steps: final state against the oracle."""
    n = 32
    z0, w0 = inputs.single_mode(n)
    m = oracle.Mesh(n, periodic=False)
    zr, wr = oracle.run(m, z0, w0, 0.5, 1.0, 0.0, 0.1 / n, 1e-3, 10)
    model = zm.ZModel(n, periodic=False, atwood=0.5, g=1.0, delta=0.1 / n, fp32c=fp32c)
    model.set_state(z0, w0)
    model.step(1e-3, 10)
    z1, w1 = model.get_state()
    model.close()
    tol = TOL32 if fp32c else TOL64
    ez, ew = rel(z1, zr), rel(w1, wr)
    dz = rel(z1 - z0, zr - z0)
    print(f"config1 fp32c={fp32c}: rel L2 z={ez:.3e} w={ew:.3e} (z - z0)={dz:.3e}")
    assert ez <= tol and ew <= tol and dz <= (1e-5 if fp32c else 1e-10)


@pytest.mark.parametrize("n1,n2", [(8, 8), (64, 32), (128, 128), (16, 256),
                                   # sides R 2^a: every odd factor R = 3 .. 19 once, a = 3 .. 6
                                   (24, 40), (56, 72), (88, 104), (120, 136), (152, 16), (96, 320),
                                   (608, 152)])
def test_low_order_parity(zm, n1, n2):
    z, w = inputs.random_state(n1, n2, seed=n1 + n2)
    m = oracle.Mesh(n1, n2, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.7, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"low order {n1}x{n2}: rel L2 u={eu:.3e} wdot={ew:.3e}")
    assert eu <= TOL64 and ew <= TOL64


@pytest.mark.parametrize("fp32c", [False, True])
@pytest.mark.parametrize("n1,n2", [(16, 16), (64, 32), (24, 40)])
def test_medium_order_parity(zm, n1, n2, fp32c):
    """Medium order: dz/dt from the Birkhoff-Rott sum, Phi from the FFT velocity."""
    tol = TOL32 if fp32c else TOL64
    z, w = inputs.random_state(n1, n2, seed=n1 * 3 + n2)
    delta = 0.1 / max(n1, n2)
    m = oracle.Mesh(n1, n2, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.6, 1.2, 0.01, delta, order=oracle.ORDER_MEDIUM)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.6, g=1.2, mu=0.01, delta=delta,
                      order=zm.ZM_ORDER_MEDIUM, fp32c=fp32c)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"medium order {n1}x{n2} fp32c={fp32c}: rel L2 u={eu:.3e} wdot={ew:.3e}")
    assert eu <= tol and ew <= tol
    # and stepping
    z0, w0 = inputs.multi_mode(n1, n_modes=4, seed=2, amp=0.02) if n1 == n2 else (z, w)
    zr, wr = oracle.run(m, z0, w0, 0.6, 1.2, 0.0, delta, 2e-3, 3, order=oracle.ORDER_MEDIUM)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.6, g=1.2, delta=delta, order=zm.ZM_ORDER_MEDIUM,
                      fp32c=fp32c)
    model.set_state(z0, w0)
    model.step(2e-3, 3)
    z1, w1 = model.get_state()
    model.close()
    assert rel(z1, zr) <= tol and rel(w1, wr) <= tol


def test_low_order_steps(zm):
    n = 64
    z0, w0 = inputs.multi_mode(n, n_modes=8, seed=3, amp=0.02)
    m = oracle.Mesh(n, periodic=True)
    zr, wr = oracle.run(m, z0, w0, 0.7, 1.0, 0.0, 0.0, 1e-3, 5, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW)
    model.set_state(z0, w0)
    model.step(1e-3, 5)
    z1, w1 = model.get_state()
    model.close()
    assert rel(z1, zr) <= TOL64 and rel(w1, wr) <= TOL64


def test_multi_mode_steps_periodic(zm):
    n = 64
    z0, w0 = inputs.multi_mode(n, n_modes=16, seed=1)
    m = oracle.Mesh(n, periodic=True)
    zr, wr = oracle.run(m, z0, w0, 0.5, 1.0, 0.0, 0.1 / n, 1e-3, 3)
    for fp32c, tol in ((False, TOL64), (True, TOL32)):
        model = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n, fp32c=fp32c)
        model.set_state(z0, w0)
        model.step(1e-3, 3)
        z1, w1 = model.get_state()
        model.close()
        assert rel(z1, zr) <= tol and rel(w1, wr) <= tol


@pytest.mark.parametrize("fp32c", [False, True])
def test_full_size_sampled_256(zm, fp32c):
    """256 x 256 periodic multi-mode interface with vorticity (one derivative evaluation in the
    launch configuration of the 256^2 benchmark): all of u from the GPU, 1024 seeded targets
    summed over all 65,536 sources by the oracle."""
    n = 256
    z, w = inputs.random_state(n, seed=11)
    delta = 0.1 / n
    m = oracle.Mesh(n, periodic=True)
    a1, a2, _, _ = oracle.geometry(m, z)
    gam = oracle.sheet_strength(w, a1, a2)
    idx = np.random.default_rng(5).choice(n * n, 1024, replace=False)
    u_ref = oracle.br_velocity(z[:, idx], z, gam, 1.0 / n**2, delta)
    model = zm.ZModel(n, periodic=True, delta=delta, fp32c=fp32c)
    u = model.velocity(z, w, want_wdot=False)
    model.close()
    e = rel(u[:, idx], u_ref)
    print(f"256^2 sampled fp32c={fp32c}: rel L2 u={e:.3e}")
    assert e <= (TOL32 if fp32c else TOL64)


def test_full_size_sampled_512_fp32c(zm):
    n = 512
    z0, w0 = inputs.multi_mode(n, n_modes=8, seed=7, amp=0.02)
    _, w = inputs.random_state(n, seed=12)
    z = z0
    delta = 0.1 / n
    m = oracle.Mesh(n, periodic=True)
    a1, a2, _, _ = oracle.geometry(m, z)
    gam = oracle.sheet_strength(w, a1, a2)
    idx = np.random.default_rng(6).choice(n * n, 256, replace=False)
    u_ref = oracle.br_velocity(z[:, idx], z, gam, 1.0 / n**2, delta)
    model = zm.ZModel(n, periodic=True, atwood=0.7, delta=delta, fp32c=True)
    u = model.velocity(z, w, want_wdot=False)
    model.close()
    e = rel(u[:, idx], u_ref)
    print(f"512^2 sampled fp32c: rel L2 u={e:.3e}")
    assert e <= TOL32


def test_low_order_1024_full(zm):
    n = 1024
    z, _ = inputs.multi_mode(n, n_modes=8, seed=7, amp=0.02)
    _, w = inputs.random_state(n, seed=13)
    m = oracle.Mesh(n, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.7, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"low order 1024^2: rel L2 u={eu:.3e} wdot={ew:.3e}")
    assert eu <= TOL64 and ew <= TOL64


def test_low_order_2048_full(zm):
    """Low order at 2048^2 (4.2 M points; every field larger than L2 together): all of u and
    dw/dt against the oracle."""
    n = 2048
    z, _ = inputs.multi_mode(n, n_modes=8, seed=5, amp=0.02)
    _, w = inputs.random_state(n, seed=14)
    m = oracle.Mesh(n, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.7, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"low order 2048^2: rel L2 u={eu:.3e} wdot={ew:.3e}")
    assert eu <= TOL64 and ew <= TOL64


def test_low_order_4864_full(zm):
    """The paper's single-GPU low-order mesh and domain (Sec. 5.1): 4864^2 nodes (19 x 256 per
    side, 23.7 M points) over (-19, 19)^2, so dx = 38 / 4864 = 2^-7 and the mesh coordinates are
    exact.  All of u and dw/dt against the oracle.

    (On the unit square dx = 1/4864 is inexact: the coordinates z1 = alpha1 then carry roundings
    of about eps |z1|, and the difference stencil turns the roundings of its own sums into
    tangent errors of about eps |z1| / dx, in the oracle and the kernels alike but in different
    operation orders; there the two agree to 7e-14 on u and 1.2e-12 on dw/dt.)"""
    n, L = 4864, 38.0
    zu, _ = inputs.multi_mode(n, n_modes=8, seed=9, amp=0.02)
    a, b = inputs.mesh_coords(n, n, L, L)
    z = np.stack([a, b, L * zu[2]])
    del zu
    _, w = inputs.random_state(n, seed=15)
    m = oracle.Mesh(n, n, L1=L, L2=L, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.7, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    model = zm.ZModel(n, L1=L, L2=L, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"low order 4864^2: rel L2 u={eu:.3e} wdot={ew:.3e}")
    assert eu <= TOL64 and ew <= TOL64


def test_low_order_steps_mixed_sides(zm):
    n1, n2 = 96, 152
    z0, w0 = inputs.random_state(n1, n2, seed=31)
    m = oracle.Mesh(n1, n2, periodic=True)
    zr, wr = oracle.run(m, z0, w0, 0.7, 1.0, 0.01, 0.0, 1e-3, 4, order=oracle.ORDER_LOW)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.7, g=1.0, mu=0.01, order=zm.ZM_ORDER_LOW)
    model.set_state(z0, w0)
    model.step(1e-3, 4)
    z1, w1 = model.get_state()
    model.close()
    print(f"low order steps 96x152: rel L2 z={rel(z1, zr):.3e} w={rel(w1, wr):.3e}")
    assert rel(z1, zr) <= TOL64 and rel(w1, wr) <= TOL64


def test_deterministic_and_device_pointers(zm):
    import torch
    n = 48
    z, w = inputs.random_state(n, seed=21)
    for fp32c in (False, True):
        model = zm.ZModel(n, periodic=True, fp32c=fp32c)
        u1, wd1 = model.velocity(z, w)
        zd = torch.from_numpy(z).cuda()
        wdv = torch.from_numpy(w).cuda()
        ud = torch.empty((3, n * n), dtype=torch.float64, device="cuda")
        wdd = torch.empty((2, n * n), dtype=torch.float64, device="cuda")
        zm.zm_set_stream(model.h, torch.cuda.current_stream().cuda_stream)
        zm.zm_velocity(model.h, zd, wdv, ud, wdd)
        torch.cuda.synchronize()
        model.close()
        assert np.array_equal(ud.cpu().numpy(), u1) and np.array_equal(wdd.cpu().numpy(), wd1)


def test_invalid_arguments(zm):
    with pytest.raises(zm.ZMError) as e:
        zm.zm_create(4, 4)
    assert e.value.code == zm.ZM_ERR_INVALID
    with pytest.raises(zm.ZMError) as e:
        zm.zm_create(32, 32, delta=0.0)
    assert e.value.code == zm.ZM_ERR_INVALID
    with pytest.raises(zm.ZMError) as e:
        zm.zm_create(32, 32, periodic=False, order=zm.ZM_ORDER_LOW)
    assert e.value.code == zm.ZM_ERR_UNSUPPORTED
    # FFT sides R 2^a need a >= 3 and R <= 19 (double words: powers of two up to 4096 only)
    for n1, n2, prec in ((12, 16, 0), (168, 64, 0), (64, 44, 0), (8192, 8, zm.ZM_PREC_DF64)):
        with pytest.raises(zm.ZMError) as e:
            zm.zm_create(n1, n2, periodic=True, order=zm.ZM_ORDER_LOW | prec)
        assert e.value.code == zm.ZM_ERR_UNSUPPORTED
    with pytest.raises(zm.ZMError) as e:
        zm.zm_create(32, 32, periodic=False, order=zm.ZM_ORDER_MEDIUM)
    assert e.value.code == zm.ZM_ERR_UNSUPPORTED


def test_nonfinite_detection(zm):
    n = 16
    z, w = inputs.random_state(n, seed=2)
    w[0, 5] = np.nan
    model = zm.ZModel(n, periodic=True)
    model.set_state(z, w)
    assert zm.zm_check_finite(model.h) == zm.ZM_ERR_NONFINITE
    w[0, 5] = 0.0
    model.set_state(z, w)
    assert zm.zm_check_finite(model.h) == zm.ZM_OK
    model.close()


@pytest.mark.parametrize("order,fp32c,periodic", [("high", False, False), ("low", False, True),
                                                   ("high", True, True)])
def test_graph_replay_equals_plain_launches(zm, order, fp32c, periodic):
    """zm_step replays one captured CUDA graph per step unless event profiling is on (plain
    launches); both must give the same bits."""
    n = 32
    z0, w0 = inputs.random_state(n, seed=8)
    od = zm.ZM_ORDER_HIGH if order == "high" else zm.ZM_ORDER_LOW
    out = []
    for profiled in (False, True):
        model = zm.ZModel(n, periodic=periodic, atwood=0.5, g=1.0, order=od, fp32c=fp32c)
        if profiled:
            zm.zm_set_profiling(model.h, 1)
        model.set_state(z0, w0)
        model.step(1e-3, 3)
        model.step(2e-3, 2)  # a new dt re-captures the graph
        out.append(model.get_state())
        prof = zm.zm_get_profile(model.h)
        model.close()
        assert prof["launches"]["geometry"] == 15 and prof["launches"]["vorticity"] == 15
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_autotune_keeps_results(zm):
    n = 96
    z, w = inputs.random_state(n, seed=4)
    model = zm.ZModel(n, periodic=True, fp32c=True)
    model.set_state(z, w)
    u0, wd0 = model.velocity()
    chosen = zm.zm_autotune(model.h)
    assert chosen in (1, 2, 4, 8, 16, 32)
    assert zm.zm_autotune(model.h) == chosen  # remembered for the process
    u1, wd1 = model.velocity()
    model.close()
    assert np.array_equal(u0, u1) and np.array_equal(wd0, wd1)
    m64 = zm.ZModel(n, periodic=True, fp32c=False)
    assert zm.zm_autotune(m64.h) == 0  # nothing to tune on the FP64 path
    m64.close()


def test_contexts_on_separate_streams_and_threads(zm):
    """Distinct contexts on distinct streams, driven from distinct host threads at once (state
    upload, graph-captured steps, state download), give the results each gives alone, bit for
    bit (every path is deterministic).  Contexts are created and destroyed on the main thread."""
    import threading

    import torch
    cases = [dict(n=64, order=zm.ZM_ORDER_HIGH, fp32c=True, df64=False),
             dict(n=48, order=zm.ZM_ORDER_HIGH, fp32c=False, df64=False),
             dict(n=128, order=zm.ZM_ORDER_LOW, fp32c=False, df64=True),
             dict(n=64, order=zm.ZM_ORDER_LOW, fp32c=False, df64=False)]

    def make(case, stream=None):
        n = case["n"]
        return zm.ZModel(n, periodic=True, atwood=0.6, g=1.0, delta=0.1 / n, order=case["order"],
                         fp32c=case["fp32c"], df64=case["df64"],
                         stream=None if stream is None else stream.cuda_stream)

    def drive(model, case):
        n = case["n"]
        z0, _ = inputs.multi_mode(n, n_modes=4, seed=n, amp=0.02)
        w0 = inputs.random_state(n, seed=n + 1)[1] * 0.1
        model.set_state(z0, w0)
        model.step(1e-3, 3)
        return model.get_state()

    alone = []
    for c in cases:
        m = make(c)
        alone.append(drive(m, c))
        m.close()
    streams = [torch.cuda.Stream() for _ in cases]
    models = [make(c, s) for c, s in zip(cases, streams)]
    got = [None] * len(cases)
    errors = []

    def worker(k):
        try:
            torch.cuda.set_device(0)
            got[k] = drive(models[k], cases[k])
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    for m in models:
        m.close()
    assert not errors, errors
    for a, b in zip(alone, got):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("order,fp32c,df64,n", [("high", False, False, 48), ("high", True, False, 64),
                                                ("low", False, False, 64), ("low", False, True, 64),
                                                ("medium", True, False, 32)])
def test_checkpoint_resume(zm, order, fp32c, df64, n):
    """Six steps in one go equal three steps, a checkpoint (zm_get_state), a fresh context
    restored from it (zm_set_state) and three more steps: bit for bit where the resident state is
    FP64 (FP64 and FP32C contexts); within two units of the double word's rounding where it is
    held as FP32 pairs (the checkpoint passes through FP64)."""
    od = {"high": zm.ZM_ORDER_HIGH, "low": zm.ZM_ORDER_LOW, "medium": zm.ZM_ORDER_MEDIUM}[order]
    z0, _ = inputs.multi_mode(n, n_modes=4, seed=n + 5, amp=0.02)
    w0 = inputs.random_state(n, seed=n + 6)[1] * 0.1

    def make():
        return zm.ZModel(n, periodic=True, atwood=0.6, g=1.0, delta=0.1 / n, order=od, fp32c=fp32c, df64=df64)

    a = make()
    a.set_state(z0, w0)
    a.step(1e-3, 6)
    z6, w6 = a.get_state()
    a.close()
    b = make()
    b.set_state(z0, w0)
    b.step(1e-3, 3)
    zc, wc = b.get_state()
    b.close()
    c = make()
    c.set_state(zc, wc)
    c.step(1e-3, 3)
    z6r, w6r = c.get_state()
    c.close()
    if df64:
        assert rel(z6r, z6) <= 1e-15 and rel(w6r, w6) <= 1e-13
    else:
        assert np.array_equal(z6r, z6) and np.array_equal(w6r, w6)


def test_bounded_wait_gives_up_and_the_gpu_stays_usable(zm):
    """A device-side wait on a flag that nothing sets gives up after its poll limit and reports
    ZM_ERR_TIMEOUT through the status word (no hang, no fault); the same wait with an arrival
    completes; and a full evaluation afterwards still matches the oracle."""
    rc, ms = zm.zm_wait_selftest(1 << 16, 0)
    assert rc == zm.ZM_ERR_TIMEOUT and ms > 0
    rc, _ = zm.zm_wait_selftest(1 << 16, 1)
    assert rc == zm.ZM_OK
    # the library's own limit: about a second of polling, so a stuck copy is reported quickly
    rc, ms = zm.zm_wait_selftest(zm.zm_wait_poll_limit(), 0)
    print(f"bounded wait: {zm.zm_wait_poll_limit()} polls gave up after {ms:.0f} ms")
    assert rc == zm.ZM_ERR_TIMEOUT and 50.0 < ms < 5000.0
    n = 32
    z, w = inputs.random_state(n, seed=5)
    m = oracle.Mesh(n, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, 0.1 / n)
    model = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n)
    u, wd = model.velocity(z, w)
    model.close()
    assert rel(u, u_ref) <= TOL64 and rel(wd, wd_ref) <= TOL64
