"""Batched form (many interfaces of uneven sizes in one set of launches per RK3 stage).

Checks: every interface against the CPU oracle (FP32C tolerance 1e-6 relative L2), results of
an interface alone and inside a mixed batch (bitwise equal: the cross-tile accumulation is exact
fixed point, so neither the batch composition nor the work-item size changes a bit), and RK3
stepping of the batch against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = 1e-6


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


SPECS = [(37, 53, False, 0.4, 1), (64, 64, True, 0.6, 2), (48, 40, True, 0.3, 3), (16, 16, False, 0.7, 4),
         (5, 9, False, 0.5, 5), (80, 96, True, 0.25, 6)]


@pytest.fixture(scope="module")
def zm():
    import torch
    from paper_2406_05490_gb300 import zm as _zm
    assert torch.cuda.is_available()
    _zm.load()
    return _zm


def make_batch(zm, specs):
    meshes = [(n1, n2, 1.0, 1.0, per) for n1, n2, per, _, _ in specs]
    atw = [a for _, _, _, a, _ in specs]
    delta = [0.1 / max(n1, n2) for n1, n2, _, _, _ in specs]
    return zm.zm_batch_create(meshes, atw, g=1.3, mu=0.0, delta=delta), delta


def test_batch_velocity_parity_and_mix_invariance(zm):
    h, delta = make_batch(zm, SPECS)
    states = [inputs.random_state(n1, n2, seed=s) for n1, n2, _, _, s in SPECS]
    for k, (z, w) in enumerate(states):
        zm.zm_batch_set_state(h, k, z, w)
    zm.zm_batch_velocity(h)
    outs = []
    for k, (n1, n2, per, at, s) in enumerate(SPECS):
        N = n1 * n2
        u = np.empty((3, N))
        wd = np.empty((2, N))
        zm.zm_batch_get_velocity(h, k, u, wd)
        outs.append((u, wd))
        m = oracle.Mesh(n1, n2, periodic=per)
        u_ref, wd_ref = oracle.derivative(m, states[k][0], states[k][1], at, 1.3, 0.0, delta[k])
        eu, ew = rel(u, u_ref), rel(wd, wd_ref)
        print(f"batch[{k}] {n1}x{n2}: rel L2 u={eu:.3e} wdot={ew:.3e}")
        assert eu <= TOL32 and ew <= TOL32
    # a different work-item size reorders all accumulation: results must not change by a bit
    zm.zm_batch_set_chunk(h, 1)
    zm.zm_batch_velocity(h)
    for k, (n1, n2, _, _, _) in enumerate(SPECS):
        u = np.empty((3, n1 * n2))
        zm.zm_batch_get_velocity(h, k, u, None)
        assert np.array_equal(u, outs[k][0])
    zm.zm_batch_destroy(h)
    # each interface alone (a context of its own) gives the same bits as inside the mix
    for k, (n1, n2, per, at, s) in enumerate(SPECS):
        model = zm.ZModel(n1, n2, periodic=per, atwood=at, g=1.3, delta=delta[k], fp32c=True)
        u, wd = model.velocity(*states[k])
        model.close()
        assert np.array_equal(u, outs[k][0]) and np.array_equal(wd, outs[k][1])


def test_batch_steps_match_oracle_and_alone(zm):
    specs = SPECS[:4]
    h, delta = make_batch(zm, specs)
    init = [inputs.multi_mode(n1, n_modes=4, seed=s, amp_std=0.02) if n1 == n2 else
            inputs.random_state(n1, n2, seed=s) for n1, n2, _, _, s in specs]
    for k, (z, w) in enumerate(init):
        zm.zm_batch_set_state(h, k, z, w)
    zm.zm_batch_step(h, 2e-3, 3)
    zm.zm_batch_sync(h)
    for k, (n1, n2, per, at, s) in enumerate(specs):
        z1 = np.empty((3, n1 * n2))
        w1 = np.empty((2, n1 * n2))
        zm.zm_batch_get_state(h, k, z1, w1)
        m = oracle.Mesh(n1, n2, periodic=per)
        zr, wr = oracle.run(m, init[k][0], init[k][1], at, 1.3, 0.0, delta[k], 2e-3, 3)
        ez, ew = rel(z1, zr), rel(w1, wr)
        print(f"batch step[{k}] {n1}x{n2}: rel L2 z={ez:.3e} w={ew:.3e}")
        assert ez <= TOL32 and ew <= TOL32
        model = zm.ZModel(n1, n2, periodic=per, atwood=at, g=1.3, delta=delta[k], fp32c=True)
        model.set_state(*init[k])
        model.step(2e-3, 3)
        za, wa = model.get_state()
        model.close()
        assert np.array_equal(za, z1) and np.array_equal(wa, w1)
    zm.zm_batch_destroy(h)


def test_batch_autotune(zm, tmp_path):
    h, delta = make_batch(zm, SPECS)
    for k, (n1, n2, _, _, s) in enumerate(SPECS):
        zm.zm_batch_set_state(h, k, *inputs.random_state(n1, n2, seed=s))
    zm.zm_batch_velocity(h)
    ref = []
    for k, (n1, n2, _, _, _) in enumerate(SPECS):
        u = np.empty((3, n1 * n2))
        zm.zm_batch_get_velocity(h, k, u, None)
        ref.append(u)
    cache = str(tmp_path / "tune.txt")
    chosen, ms = zm.zm_batch_autotune(h, cache)
    assert chosen >= 1 and (tmp_path / "tune.txt").read_text().strip()
    zm.zm_batch_velocity(h)
    for k, (n1, n2, _, _, _) in enumerate(SPECS):
        u = np.empty((3, n1 * n2))
        zm.zm_batch_get_velocity(h, k, u, None)
        assert np.array_equal(u, ref[k])
    zm.zm_batch_destroy(h)


def test_batch_rejects_bad_arguments(zm):
    with pytest.raises(zm.ZMError) as e:
        zm.zm_batch_create([(4, 4, 1.0, 1.0, True)], [0.5])
    assert e.value.code == zm.ZM_ERR_INVALID
    with pytest.raises(zm.ZMError) as e:
        zm.zm_batch_create([(16, 16, 1.0, 1.0, True)], [0.5], delta=[0.0])
    assert e.value.code == zm.ZM_ERR_INVALID


SHAPES = [(16, 16), (8, 32), (32, 8), (4, 64), (64, 4)]


def test_tile_shapes_parity(zm):
    """Every candidate tile shape gives results within the FP32C bound of the oracle, on a mix of
    square, anisotropic (dx1 = 4 dx2), ragged and free-edge interfaces; within one shape the
    work-item size still changes no bit."""
    specs = [(64, 64, True, 0.6, 2), (32, 128, True, 0.5, 7), (37, 53, False, 0.4, 1), (5, 9, False, 0.5, 5)]
    h, delta = make_batch(zm, specs)
    states = [inputs.random_state(n1, n2, seed=s) for n1, n2, _, _, s in specs]
    refs = []
    for k, (z, w) in enumerate(states):
        zm.zm_batch_set_state(h, k, z, w)
        n1, n2, per, at, _ = specs[k]
        refs.append(oracle.derivative(oracle.Mesh(n1, n2, periodic=per), z, w, at, 1.3, 0.0, delta[k]))
    for tp1, tp2 in SHAPES:
        zm.zm_batch_set_tile_shape(h, tp1, tp2)
        assert zm.zm_batch_get_tile_shape(h) == (tp1, tp2)
        zm.zm_batch_set_chunk(h, 0)
        zm.zm_batch_velocity(h)
        first = []
        for k, (n1, n2, _, _, _) in enumerate(specs):
            u, wd = np.empty((3, n1 * n2)), np.empty((2, n1 * n2))
            zm.zm_batch_get_velocity(h, k, u, wd)
            first.append(u)
            eu, ew = rel(u, refs[k][0]), rel(wd, refs[k][1])
            print(f"tiles {tp1}x{tp2} [{k}] {n1}x{n2}: rel L2 u={eu:.3e} wdot={ew:.3e}")
            assert eu <= TOL32 and ew <= TOL32
        zm.zm_batch_set_chunk(h, 1)
        zm.zm_batch_velocity(h)
        for k, (n1, n2, _, _, _) in enumerate(specs):
            u = np.empty((3, n1 * n2))
            zm.zm_batch_get_velocity(h, k, u, None)
            assert np.array_equal(u, first[k])
    with pytest.raises(zm.ZMError):
        zm.zm_batch_set_tile_shape(h, 16, 8)
    zm.zm_batch_destroy(h)


def test_tile_autotune_on_an_anisotropic_mesh(zm, tmp_path):
    """On a 64 x 256 mesh of the unit square (dx1 = 4 dx2) a 16 x 16 tile spans 0.25 x 0.0625,
    an 8 x 32 tile 0.125 x 0.125: the tile autotuner picks a shape no slower than the square one,
    remembers it, and the tuned batch still matches the oracle."""
    import torch
    n1, n2 = 64, 256
    z, w = inputs.random_state(n1, n2, seed=23)
    h = zm.zm_batch_create([(n1, n2, 1.0, 1.0, True)], [0.5], g=1.3, delta=[0.1 / n2])
    zm.zm_batch_set_state(h, 0, z, w)

    def br_ms(shape):
        zm.zm_batch_set_tile_shape(h, *shape)
        zm.zm_batch_set_chunk(h, 0)
        zm.zm_batch_velocity(h)
        zm.zm_batch_set_profiling(h, 1)
        for _ in range(3):
            zm.zm_batch_velocity(h)
        p = zm.zm_batch_get_profile(h)
        zm.zm_batch_set_profiling(h, 0)
        return p["ms"]["br"] / p["launches"]["br"]

    square = br_ms((16, 16))
    cache = str(tmp_path / "tiles.txt")
    shape, chunk, ms = zm.zm_batch_autotune_tiles(h, cache)
    print(f"anisotropic 64x256: tuned tiles {shape}, chunk {chunk}, {ms:.3f} ms/eval; 16x16 BR {square:.3f} ms")
    assert shape in SHAPES and 1 <= chunk <= 32 and ms > 0
    assert zm.zm_batch_get_tile_shape(h) == shape
    zm.zm_batch_set_chunk(h, 0)
    tuned = br_ms(shape)
    assert tuned <= 1.1 * square
    shape2, chunk2, ms2 = zm.zm_batch_autotune_tiles(h, cache)  # remembered
    assert (shape2, chunk2, ms2) == (shape, chunk, -1.0)
    assert any("|tiles" in line for line in open(cache))
    zm.zm_batch_set_chunk(h, chunk)
    zm.zm_batch_velocity(h)
    u, wd = np.empty((3, n1 * n2)), np.empty((2, n1 * n2))
    zm.zm_batch_get_velocity(h, 0, u, wd)
    zm.zm_batch_destroy(h)
    mesh = oracle.Mesh(n1, n2, periodic=True)
    u_ref, wd_ref = oracle.derivative(mesh, z, w, 0.5, 1.3, 0.0, 0.1 / n2)
    # dw/dt differentiates |u|^2/2 with the 1/dx2 = 256 stencil: on this random state, velocity
    # errors of relative size e that are uncorrelated between nodes reach dw/dt amplified about
    # 13-fold.  The bound is that amplification of the velocity bound, measured on the oracle
    # with seeded noise of relative L2 size TOL32 added to its own velocity.
    a1, a2, hm, _ = oracle.geometry(mesh, z)
    noise = np.random.default_rng(0).standard_normal(u_ref.shape)
    u_pert = u_ref + TOL32 * np.linalg.norm(u_ref) / np.linalg.norm(noise) * noise
    wd_pert = oracle.wdot(mesh, oracle.phi(z, w, hm, u_pert, 1.3), w, 0.5, 0.0)
    tol_wd = max(TOL32, rel(wd_pert, wd_ref))
    print(f"anisotropic 64x256: rel L2 u={rel(u, u_ref):.3e} wdot={rel(wd, wd_ref):.3e} (bound {tol_wd:.2e})")
    assert rel(u, u_ref) <= TOL32 and rel(wd, wd_ref) <= tol_wd
    torch.cuda.synchronize()


def test_bench_batch_of_64_sampled(zm):
    """The batched configuration itself: 64 periodic interfaces, sides log-uniform in [64, 384]
    (seed 0), 4 modes, A ~ U[0.2, 0.8], FP32C, one graph-replayed RK3 step on the whole batch;
    eight seeded interfaces of side <= 100 (so that the serial oracle finishes in seconds)
    against the oracle's step, on the state and on the displacement z - z0 (w starts at 0,
    so the first stage moves nothing and the step is carried by the later stages)."""
    insts = inputs.ragged_batch(count=64, lo=64, hi=384, n_modes=4, seed=0)
    delta = [0.1 / r.n for r in insts]
    h = zm.zm_batch_create([(r.n, r.n, 1.0, 1.0, True) for r in insts], [r.atwood for r in insts], g=1.0,
                           delta=delta)
    for k, r in enumerate(insts):
        zm.zm_batch_set_state(h, k, r.z, r.w)
    zm.zm_batch_step(h, 1e-3, 1)
    zm.zm_batch_sync(h)
    small = [k for k, r in enumerate(insts) if r.n <= 100]
    pick = sorted(np.random.default_rng(1).choice(small, size=min(8, len(small)), replace=False).tolist())
    assert len(pick) == 8
    for k in pick:
        r = insts[k]
        N = r.n * r.n
        z1, w1 = np.empty((3, N)), np.empty((2, N))
        zm.zm_batch_get_state(h, k, z1, w1)
        zr, wr = oracle.run(oracle.Mesh(r.n, periodic=True), r.z, r.w, r.atwood, 1.0, 0.0, delta[k], 1e-3, 1)
        ez, ew, dz = rel(z1, zr), rel(w1, wr), rel(z1 - r.z, zr - r.z)
        print(f"batch of 64, interface {k} ({r.n}^2): rel L2 z={ez:.3e} w={ew:.3e} (z - z0)={dz:.3e}")
        assert ez <= TOL32 and ew <= TOL32 and dz <= 1e-5
    zm.zm_batch_destroy(h)


def test_context_tile_shape(zm):
    """zm_set_tile_shape / zm_get_tile_shape on a single FP32C context (a batch of one): every
    shape stays within the FP32C bound of the oracle; other shapes and FP64 contexts are refused."""
    n1, n2 = 32, 128
    z, w = inputs.random_state(n1, n2, seed=29)
    delta = 0.1 / n2
    u_ref, wd_ref = oracle.derivative(oracle.Mesh(n1, n2, periodic=True), z, w, 0.5, 1.3, 0.0, delta)
    m = zm.ZModel(n1, n2, periodic=True, atwood=0.5, g=1.3, delta=delta, fp32c=True)
    assert zm.zm_get_tile_shape(m.h) == (16, 16)
    for shape in SHAPES:
        zm.zm_set_tile_shape(m.h, *shape)
        assert zm.zm_get_tile_shape(m.h) == shape
        u, wd = m.velocity(z, w)
        print(f"context tiles {shape}: rel L2 u={rel(u, u_ref):.3e} wdot={rel(wd, wd_ref):.3e}")
        assert rel(u, u_ref) <= TOL32 and rel(wd, wd_ref) <= TOL32
    with pytest.raises(zm.ZMError) as e:
        zm.zm_set_tile_shape(m.h, 16, 8)
    assert e.value.code == zm.ZM_ERR_INVALID
    m.close()
    m64 = zm.ZModel(n1, n2, periodic=True, atwood=0.5, g=1.3, delta=delta)
    with pytest.raises(zm.ZMError) as e:
        zm.zm_set_tile_shape(m64.h, 8, 32)
    assert e.value.code == zm.ZM_ERR_UNSUPPORTED
    m64.close()
