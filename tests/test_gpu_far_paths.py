"""The two far paths of the FP32C all-pairs sum (far tile pairs: everything on the CUDA cores,
the default, or the Gram part of |t - s|^2 on the tensor cores and the rest on the CUDA cores;
near pairs always on the CUDA cores), each against the CPU oracle at the FP32C velocity bound (1e-6 relative L2) on meshes
with one tile, ragged tiles, free and periodic edges, and against each other; both bitwise
deterministic."""
import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs

pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("n1,n2,periodic", [(16, 16, True), (37, 53, False), (96, 80, True), (128, 128, True)])
def test_far_paths_against_the_oracle(zm, n1, n2, periodic):
    z, w = inputs.random_state(n1, n2, seed=n1 * 3 + n2)
    delta = 0.1 / max(n1, n2)
    m = oracle.Mesh(n1, n2, periodic=periodic)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, delta)
    out = {}
    for path in (zm.ZM_FAR_TENSOR, zm.ZM_FAR_CUDA):
        model = zm.ZModel(n1, n2, periodic=periodic, atwood=0.5, g=1.0, delta=delta, fp32c=True)
        assert zm.zm_get_far_path(model.h) == zm.ZM_FAR_CUDA  # the default
        zm.zm_set_far_path(model.h, path)
        assert zm.zm_get_far_path(model.h) == path
        u, wd = model.velocity(z, w)
        u2, wd2 = model.velocity(z, w)
        model.close()
        assert np.array_equal(u, u2) and np.array_equal(wd, wd2)  # deterministic
        eu, ew = rel(u, u_ref), rel(wd, wd_ref)
        print(f"far path {path} {n1}x{n2}: rel L2 u={eu:.3e} wdot={ew:.3e}")
        assert eu <= TOL32 and ew <= TOL32
        out[path] = u
    assert rel(out[zm.ZM_FAR_TENSOR], out[zm.ZM_FAR_CUDA]) <= 2 * TOL32


def test_far_paths_on_a_folded_interface(zm):
    """An interface that folds over itself (z1 = a + 0.25 sin 2 pi a overhangs), so that nodes 20 and
    more mesh points apart come within 2 dx of each other in space (128^2: 72 % of the tile pairs
    far): the near / far split is decided by the tiles' bounding spheres in space, not by mesh
    distance, and both far paths stay within the FP32C bound of the oracle."""
    n = 128
    a, b = inputs.mesh_coords(n)
    z = np.stack([a + 0.25 * np.sin(2 * np.pi * a), b + 0.05 * np.sin(2 * np.pi * a),
                  0.03 * np.sin(2 * np.pi * a) + 0.02 * np.cos(2 * np.pi * b)])
    _, w = inputs.random_state(n, seed=17)
    delta = 0.1 / n
    u_ref, wd_ref = oracle.derivative(oracle.Mesh(n, periodic=True), z, w, 0.5, 1.0, 0.0, delta)
    for path in (zm.ZM_FAR_TENSOR, zm.ZM_FAR_CUDA):
        model = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=delta, fp32c=True)
        zm.zm_set_far_path(model.h, path)
        u, wd = model.velocity(z, w)
        model.close()
        eu, ew = rel(u, u_ref), rel(wd, wd_ref)
        print(f"folded 128^2, far path {path}: rel L2 u={eu:.3e} wdot={ew:.3e}")
        assert eu <= TOL32 and ew <= TOL32


def test_far_path_at_full_size_sampled(zm):
    """256^2 with vorticity: all of u from each path, 1024 seeded targets summed by the oracle."""
    n = 256
    z, w = inputs.random_state(n, seed=11)
    delta = 0.1 / n
    m = oracle.Mesh(n, periodic=True)
    a1, a2, _, _ = oracle.geometry(m, z)
    gam = oracle.sheet_strength(w, a1, a2)
    idx = np.random.default_rng(5).choice(n * n, 1024, replace=False)
    u_ref = oracle.br_velocity(z[:, idx], z, gam, 1.0 / n**2, delta)
    for path in (zm.ZM_FAR_TENSOR, zm.ZM_FAR_CUDA):
        model = zm.ZModel(n, periodic=True, delta=delta, fp32c=True)
        zm.zm_set_far_path(model.h, path)
        u = model.velocity(z, w, want_wdot=False)
        model.close()
        e = rel(u[:, idx], u_ref)
        print(f"256^2 sampled, far path {path}: rel L2 u={e:.3e}")
        assert e <= TOL32


def test_far_path_rejects_bad_values(zm):
    model = zm.ZModel(32, periodic=True, fp32c=True)
    with pytest.raises(zm.ZMError) as e:
        zm.zm_set_far_path(model.h, 5)
    assert e.value.code == zm.ZM_ERR_INVALID
    model.close()
    model = zm.ZModel(32, periodic=True, fp32c=False)
    with pytest.raises(zm.ZMError) as e:
        zm.zm_set_far_path(model.h, zm.ZM_FAR_CUDA)
    assert e.value.code == zm.ZM_ERR_UNSUPPORTED
    model.close()
    h = zm.zm_batch_create([(32, 32, 1.0, 1.0, True)], [0.5])
    assert zm.zm_batch_get_far_path(h) == zm.ZM_FAR_CUDA
    zm.zm_batch_set_far_path(h, zm.ZM_FAR_TENSOR)
    assert zm.zm_batch_get_far_path(h) == zm.ZM_FAR_TENSOR
    with pytest.raises(zm.ZMError):
        zm.zm_batch_set_far_path(h, -1)
    zm.zm_batch_destroy(h)


def test_tensor_path_runs_three_ctas_per_sm(zm):
    """The tensor-core kernel's residency comes from its own resource use (the runtime's occupancy
    query answers one CTA per SM for it): its registers, shared memory and 128 tensor-memory
    columns leave room for three CTAs per SM, against one for the query's answer."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    h = zm.zm_batch_create([(256, 256, 1.0, 1.0, True)], [0.5])
    cuda_ctas = zm.zm_batch_info(h)["ctas"]
    zm.zm_batch_set_far_path(h, zm.ZM_FAR_TENSOR)
    tc_ctas = zm.zm_batch_info(h)["ctas"]
    zm.zm_batch_destroy(h)
    print(f"persistent CTAs: CUDA-core kernel {cuda_ctas}, tensor-core kernel {tc_ctas} ({sms} SMs)")
    assert tc_ctas == 3 * sms and cuda_ctas >= sms


def test_tensor_path_with_cutoff_and_in_a_batch(zm):
    """The tensor-core far path under a cutoff (its masked near path and tile skipping), against
    the oracle with the boundary-band treatment of test_gpu_cutoff; and inside a ragged batch,
    each interface bitwise equal to the same interface alone on the same path (fixed-point
    accumulation: neither the batch composition nor the scheduling changes a bit)."""
    from test_gpu_cutoff import band_corrected_reference
    n1, n2, c = 96, 80, 0.15
    z, w = inputs.random_state(n1, n2, seed=n1 + n2)
    delta = 0.1 / max(n1, n2)
    m = oracle.Mesh(n1, n2, periodic=True)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.5, g=1.0, delta=delta, fp32c=True)
    zm.zm_set_far_path(model.h, zm.ZM_FAR_TENSOR)
    zm.zm_set_cutoff(model.h, c)
    u, wd = model.velocity(z, w)
    model.close()
    u_ref, wd_ref, nband, nflip = band_corrected_reference(m, z, w, u, 0.5, 1.0, 0.0, delta, c)
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"tensor path, cutoff {c} {n1}x{n2}: rel L2 u={eu:.3e} wdot={ew:.3e} (band {nband}, flipped {nflip})")
    assert eu <= TOL32 and ew <= 1e-5
    specs = [(64, 64), (48, 40), (37, 53)]
    states = [inputs.random_state(a, b, seed=a + 2 * b) for a, b in specs]
    h = zm.zm_batch_create([(a, b, 1.0, 1.0, True) for a, b in specs], [0.5] * len(specs))
    zm.zm_batch_set_far_path(h, zm.ZM_FAR_TENSOR)
    for k, (zz, ww) in enumerate(states):
        zm.zm_batch_set_state(h, k, zz, ww)
    zm.zm_batch_velocity(h)
    for k, (a, b) in enumerate(specs):
        ub = np.empty((3, a * b))
        zm.zm_batch_get_velocity(h, k, ub, None)
        alone = zm.ZModel(a, b, periodic=True, atwood=0.5, g=1.0, fp32c=True)
        zm.zm_set_far_path(alone.h, zm.ZM_FAR_TENSOR)
        ua = alone.velocity(*states[k], want_wdot=False)
        alone.close()
        assert np.array_equal(ub, ua), k
    zm.zm_batch_destroy(h)


def test_tensor_path_every_tile_shape(zm):
    """The tensor-core far path with every candidate tile shape (its operands are built per
    256-slot tile whatever the patch shape) on square, anisotropic (dx1 = 4 dx2), ragged and
    free-edge interfaces in one batch, against the oracle; within one shape the work-item size
    changes no bit."""
    specs = [(64, 64, True, 0.6, 2), (32, 128, True, 0.5, 7), (37, 53, False, 0.4, 1), (5, 9, False, 0.5, 5)]
    meshes = [(n1, n2, 1.0, 1.0, per) for n1, n2, per, _, _ in specs]
    delta = [0.1 / max(n1, n2) for n1, n2, _, _, _ in specs]
    h = zm.zm_batch_create(meshes, [a for _, _, _, a, _ in specs], g=1.3, mu=0.0, delta=delta)
    zm.zm_batch_set_far_path(h, zm.ZM_FAR_TENSOR)
    refs = []
    for k, (n1, n2, per, at, seed) in enumerate(specs):
        z, w = inputs.random_state(n1, n2, seed=seed)
        zm.zm_batch_set_state(h, k, z, w)
        refs.append(oracle.derivative(oracle.Mesh(n1, n2, periodic=per), z, w, at, 1.3, 0.0, delta[k]))
    for tp1, tp2 in [(16, 16), (8, 32), (32, 8), (4, 64), (64, 4)]:
        zm.zm_batch_set_tile_shape(h, tp1, tp2)
        zm.zm_batch_set_chunk(h, 0)
        zm.zm_batch_velocity(h)
        first = []
        for k, (n1, n2, _, _, _) in enumerate(specs):
            u, wd = np.empty((3, n1 * n2)), np.empty((2, n1 * n2))
            zm.zm_batch_get_velocity(h, k, u, wd)
            first.append(u)
            eu, ew = rel(u, refs[k][0]), rel(wd, refs[k][1])
            print(f"tensor path, tiles {tp1}x{tp2} [{k}] {n1}x{n2}: rel L2 u={eu:.3e} wdot={ew:.3e}")
            assert eu <= TOL32 and ew <= TOL32
        zm.zm_batch_set_chunk(h, 1)
        zm.zm_batch_velocity(h)
        for k, (n1, n2, _, _, _) in enumerate(specs):
            u = np.empty((3, n1 * n2))
            zm.zm_batch_get_velocity(h, k, u, None)
            assert np.array_equal(u, first[k])
    zm.zm_batch_destroy(h)


def test_tensor_path_medium_order(zm):
    """Medium order (dz/dt from the all-pairs sum, Phi from the FFT velocity) with the far pairs
    on the tensor cores: one evaluation and three steps against the oracle."""
    n1, n2 = 64, 64
    z, w = inputs.random_state(n1, n2, seed=n1 * 3 + n2)
    delta = 0.1 / n1
    m = oracle.Mesh(n1, n2, periodic=True)
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.6, 1.2, 0.01, delta, order=oracle.ORDER_MEDIUM)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.6, g=1.2, mu=0.01, delta=delta,
                      order=zm.ZM_ORDER_MEDIUM, fp32c=True)
    zm.zm_set_far_path(model.h, zm.ZM_FAR_TENSOR)
    u, wd = model.velocity(z, w)
    model.close()
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"tensor path, medium order {n1}x{n2}: rel L2 u={eu:.3e} wdot={ew:.3e}")
    assert eu <= TOL32 and ew <= TOL32
    z0, w0 = inputs.multi_mode(n1, n_modes=4, seed=2, amp=0.02)
    zr, wr = oracle.run(m, z0, w0, 0.6, 1.2, 0.0, delta, 2e-3, 3, order=oracle.ORDER_MEDIUM)
    model = zm.ZModel(n1, n2, periodic=True, atwood=0.6, g=1.2, delta=delta, order=zm.ZM_ORDER_MEDIUM,
                      fp32c=True)
    zm.zm_set_far_path(model.h, zm.ZM_FAR_TENSOR)
    model.set_state(z0, w0)
    model.step(2e-3, 3)
    z1, w1 = model.get_state()
    model.close()
    assert rel(z1, zr) <= TOL32 and rel(w1, wr) <= TOL32

