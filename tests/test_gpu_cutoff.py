"""Cutoff Birkhoff-Rott sum (Sec. 3.2.2: sources within a 3D distance only) against the CPU
oracle, which decides each pair in FP64 on |z_i - z_j| <= c.

The GPU decides a pair that it cannot place by its tile's bounding sphere in FP32 (hi/lo
position difference, |r|^2 by an FMA chain, compared with fl32(c^2)); that decision is exact to
a relative error of about 2^-22 in the distance.  A pair whose FP64 distance lies within a
relative band of 2^-20 of c may therefore fall either way, and either answer is correct.  The
test finds every such band pair, and for each target picks the in/out assignment of its band
pairs that best explains the GPU result; the oracle's velocity is corrected by exactly those
pairs' oracle contributions, and dw/dt recomputed from it by the oracle.  The GPU result must
then lie within tolerance: u 1e-6 relative L2 (the FP32C velocity bound); dw/dt 1e-5, because it
differentiates |u|^2 / 2 and the per-target cut makes the FP32 rounding of neighbouring targets'
velocities uncorrelated, which the fourth-order stencil amplifies by about 1.5 / dx (~100 here)
relative to the smooth exact-sum case.
A cutoff larger than the interface gives the exact sum bit for bit; per-interface cutoffs in
a batch equal the same cutoffs alone, bit for bit."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs

TOL32 = 1e-6
TOL32_RATE = 1e-5
BAND = 2.0 ** -20


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def zm():
    import torch
    from paper_2406_05490_gb300 import zm as _zm
    assert torch.cuda.is_available()
    _zm.load()
    return _zm


def band_pairs(z, c):
    """(i, j) pairs with | |z_i - z_j| - c | <= BAND c (FP64 distances)."""
    N = z.shape[1]
    out = []
    for i0 in range(0, N, 256):
        d = np.sqrt(((z[:, i0:i0 + 256, None] - z[:, None, :]) ** 2).sum(axis=0))
        ii, jj = np.nonzero(np.abs(d - c) <= BAND * c)
        out += [(int(i + i0), int(j)) for i, j in zip(ii, jj)]
    return out


def band_corrected_reference(mesh, z, w, u_gpu, atwood, g, mu, delta, c):
    """The oracle's (u, dw/dt) with the band pairs of each target assigned in or out as the GPU
    result suggests.  Returns (u_ref, wd_ref, number of band pairs, number flipped)."""
    u_ref, wd_ref = oracle.derivative(mesh, z, w, atwood, g, mu, delta, cutoff=c)
    pairs = band_pairs(z, c)
    if not pairs:
        return u_ref, wd_ref, 0, 0
    a1, a2, h, _ = oracle.geometry(mesh, z)
    gam = oracle.sheet_strength(w, a1, a2)
    weight = (mesh.L1 / mesh.n1) * (mesh.L2 / mesh.n2)
    by_target = {}
    for i, j in pairs:
        term = oracle.br_velocity(z[:, [i]], z[:, [j]], gam[:, [j]], weight, delta)[:, 0]
        # the change of u_i if this pair's decision is flipped relative to the oracle's
        sign = -1.0 if oracle.within_cutoff(z[:, i], z[:, j], c) else 1.0
        by_target.setdefault(i, []).append(sign * term)
    u_adj = u_ref.copy()
    flipped = 0
    for i, terms in by_target.items():
        assert len(terms) <= 12, "too many boundary pairs at one target to enumerate"
        best, best_k = None, 0
        for mask in itertools.product((0, 1), repeat=len(terms)):
            cand = u_ref[:, i] + sum((t for t, m in zip(terms, mask) if m), np.zeros(3))
            err = np.linalg.norm(u_gpu[:, i] - cand)
            if best is None or err < best[0]:
                best, best_k = (err, cand), sum(mask)
        u_adj[:, i] = best[1]
        flipped += best_k
    if flipped == 0:
        return u_ref, wd_ref, len(pairs), 0
    phi = oracle.phi(z, w, h, u_adj, g)
    wd_adj = oracle.wdot(mesh, phi, w, atwood, mu)
    return u_adj, wd_adj, len(pairs), flipped


def test_band_correction_reproduces_the_oracle_without_flips():
    """The dw/dt recomputation from the oracle's pieces equals oracle.derivative bit for bit, so
    the correction above changes nothing but the flipped pairs."""
    n1, n2, c = 24, 20, 0.15
    z, w = inputs.random_state(n1, n2, seed=3)
    m = oracle.Mesh(n1, n2, periodic=True)
    delta = 0.1 / n1
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, delta, cutoff=c)
    _, _, h, _ = oracle.geometry(m, z)
    wd = oracle.wdot(m, oracle.phi(z, w, h, u_ref, 1.0), w, 0.5, 0.0)
    assert np.array_equal(wd, wd_ref)


def test_band_correction_explains_a_flipped_boundary_pair():
    """A result that takes one boundary pair the other way than the oracle (planted here on the
    CPU) is explained exactly by the correction, and only that pair is flipped; the same result
    with a pair far from the boundary flipped is not explained."""
    n1 = n2 = 48
    c = 0.06
    z, w = inputs.random_state(n1, n2, seed=n1 + n2)
    m = oracle.Mesh(n1, n2, periodic=True)
    delta = 0.1 / n1
    u_ref, wd_ref = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, delta, cutoff=c)
    (i, j) = band_pairs(z, c)[0]
    a1, a2, _, _ = oracle.geometry(m, z)
    gam = oracle.sheet_strength(w, a1, a2)
    term = oracle.br_velocity(z[:, [i]], z[:, [j]], gam[:, [j]], 1.0 / (n1 * n2), delta)[:, 0]
    sign = -1.0 if oracle.within_cutoff(z[:, i], z[:, j], c) else 1.0
    u_fake = u_ref.copy()
    u_fake[:, i] += sign * term
    u_adj, wd_adj, nband, nflip = band_corrected_reference(m, z, w, u_fake, 0.5, 1.0, 0.0, delta, c)
    assert nflip == 1 and rel(u_fake, u_adj) < 1e-15 and not np.array_equal(wd_adj, wd_ref)
    # a pair well inside the cutoff is not a band pair: flipping it stays visible
    d = np.linalg.norm(z - z[:, [i]], axis=0)
    k = int(np.argmin(np.abs(d - 0.5 * c)))
    term_k = oracle.br_velocity(z[:, [i]], z[:, [k]], gam[:, [k]], 1.0 / (n1 * n2), delta)[:, 0]
    u_bad = u_ref.copy()
    u_bad[:, i] -= term_k
    u_adj, _, _, _ = band_corrected_reference(m, z, w, u_bad, 0.5, 1.0, 0.0, delta, c)
    assert np.linalg.norm(u_bad[:, i] - u_adj[:, i]) >= 0.5 * np.linalg.norm(term_k)


@pytest.mark.gpu
@pytest.mark.parametrize("n1,n2,periodic,cutoff", [(96, 80, True, 0.15), (64, 64, False, 0.4),
                                                   (48, 48, True, 0.06), (128, 96, True, 0.2)])
def test_cutoff_parity(zm, n1, n2, periodic, cutoff):
    z, w = inputs.random_state(n1, n2, seed=n1 + n2)
    delta = 0.1 / max(n1, n2)
    m = oracle.Mesh(n1, n2, periodic=periodic)
    model = zm.ZModel(n1, n2, periodic=periodic, atwood=0.5, g=1.0, delta=delta, fp32c=True)
    zm.zm_set_cutoff(model.h, cutoff)
    u, wd = model.velocity(z, w)
    model.close()
    u_ref, wd_ref, nband, nflip = band_corrected_reference(m, z, w, u, 0.5, 1.0, 0.0, delta, cutoff)
    u_ex, _ = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, delta)
    eu, ew = rel(u, u_ref), rel(wd, wd_ref)
    print(f"cutoff {cutoff} {n1}x{n2}: rel L2 u={eu:.3e} wdot={ew:.3e}; band pairs {nband}, "
          f"decided the other way {nflip}; cutoff vs exact sum {rel(u_ref, u_ex):.3e}")
    assert eu <= TOL32 and ew <= TOL32_RATE


@pytest.mark.gpu
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


@pytest.mark.gpu
def test_cutoff_needs_fp32c(zm):
    model = zm.ZModel(32, periodic=True, fp32c=False)
    with pytest.raises(zm.ZMError) as e:
        zm.zm_set_cutoff(model.h, 0.2)
    assert e.value.code == zm.ZM_ERR_UNSUPPORTED
    model.close()

@pytest.mark.gpu
def test_cutoff_on_a_folded_interface(zm):
    """A folded interface (z1 = a + 0.25 sin 2 pi a overhangs): tiles far apart on the mesh come
    within the cutoff in space, so skipping a tile pair must follow the bounding spheres in space,
    never mesh distance.  Both far paths against the band-corrected oracle."""
    n, c = 128, 0.05
    a, b = inputs.mesh_coords(n)
    z = np.stack([a + 0.25 * np.sin(2 * np.pi * a), b + 0.05 * np.sin(2 * np.pi * a),
                  0.03 * np.sin(2 * np.pi * a) + 0.02 * np.cos(2 * np.pi * b)])
    _, w = inputs.random_state(n, seed=17)
    delta = 0.1 / n
    m = oracle.Mesh(n, periodic=True)
    # the fold matters: pairs 20 or more mesh rows apart lie within the cutoff
    i1 = np.arange(n * n) // n
    close = np.linalg.norm(z[:, None, ::97] - z[:, ::89, None], axis=0) <= c
    d = np.abs(i1[::89][:, None] - i1[None, ::97])
    assert np.any(close & (np.minimum(d, n - d) >= 20))
    for path in (zm.ZM_FAR_TENSOR, zm.ZM_FAR_CUDA):
        model = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=delta, fp32c=True)
        zm.zm_set_far_path(model.h, path)
        zm.zm_set_cutoff(model.h, c)
        u, wd = model.velocity(z, w)
        model.close()
        u_ref, wd_ref, nband, nflip = band_corrected_reference(m, z, w, u, 0.5, 1.0, 0.0, delta, c)
        eu, ew = rel(u, u_ref), rel(wd, wd_ref)
        print(f"folded 128^2, cutoff {c}, far path {path}: rel L2 u={eu:.3e} wdot={ew:.3e} "
              f"(band {nband}, flipped {nflip})")
        assert eu <= TOL32 and ew <= TOL32_RATE
