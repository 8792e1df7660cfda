"""Pins for the CPU oracle: each test checks it against something other than its own formulas.

Kinds of pin used (the paper prints no equations or worked values, so every pin is a closed
form, an invariant, a special case that reduces to a library routine, or extended-precision
brute force):
  * stencils: exactness on polynomials, the modified wavenumber of the 4th-order stencil, the
    periodic seam shift and free-edge extrapolation on linear data;
  * geometry: tilted plane (closed-form tangents, metric, normal); Lagrange's identity;
  * Birkhoff-Rott sum: flat rest and flat-sheet in-plane velocity (exact zeros), pairwise
    antisymmetry, momentum balance, translation/rotation covariance, exact power-of-two scaling,
    a Gaussian vortex sheet against its Hankel-transform closed form, first-order convergence
    of the sheet response to the continuous Riesz value, and 50-digit brute force;
  * Riesz / FFT: numpy.fft cross-check, a single gradient mode (closed form), a curl field
    (annihilated);
  * RK3 + low-order model: exact linear Rayleigh-Taylor evolution P(dt M)^n on one mode;
  * high-order model: early growth of a single mode against cosh(sqrt(A k g) t).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_05490_gb300 import inputs


def grid(n):
    a, b = inputs.mesh_coords(n)
    return a, b


def interior(n, depth=2):
    i = np.arange(n * n) // n
    j = np.arange(n * n) % n
    return (i >= depth) & (i < n - depth) & (j >= depth) & (j < n - depth)


# ------------------------------------------------------------------------------------------
# stencils
# ------------------------------------------------------------------------------------------

def test_first_derivative_exact_on_quartics():
    n = 16
    m = oracle.Mesh(n, periodic=False)
    a, b = grid(n)
    f = 0.3 + 1.7 * a - 2.1 * a**2 + 0.9 * a**3 - 1.3 * a**4 + 0.5 * b**4 - b * a**2
    d1 = 1.7 - 4.2 * a + 2.7 * a**2 - 5.2 * a**3 - 2 * b * a
    d2 = 2.0 * b**3 - a**2
    inn = interior(n)
    np.testing.assert_allclose(oracle.diff1(m, f, 0)[inn], d1[inn], rtol=0, atol=1e-11)
    np.testing.assert_allclose(oracle.diff1(m, f, 1)[inn], d2[inn], rtol=0, atol=1e-11)


def test_laplacian_exact_on_quintics():
    n = 16
    m = oracle.Mesh(n, periodic=False)
    a, b = grid(n)
    f = a**5 - 2 * b**5 + 3 * a**2 * b**3 + a * b
    lap = 20 * a**3 - 40 * b**3 + 6 * b**3 + 18 * a**2 * b
    inn = interior(n)
    np.testing.assert_allclose(oracle.laplacian(m, f)[inn], lap[inn], rtol=0, atol=1e-9)


def test_free_edges_exact_on_linear_data():
    # linear extrapolation into the halo keeps linear data linear, so the stencils are exact
    # at every node, edges included
    n = 12
    m = oracle.Mesh(n, periodic=False)
    a, b = grid(n)
    f = 0.25 - 1.5 * a + 2.5 * b
    np.testing.assert_allclose(oracle.diff1(m, f, 0), -1.5, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.diff1(m, f, 1), 2.5, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.laplacian(m, f), 0.0, rtol=0, atol=1e-9)


def test_periodic_modified_wavenumber():
    # D cos(k a) = -kappa sin(k a), kappa = (8 sin(k dx) - sin(2 k dx)) / (6 dx)
    n = 32
    m = oracle.Mesh(n, periodic=True)
    a, b = grid(n)
    dx = 1.0 / n
    for mode in (1, 3, 7):
        k = 2 * np.pi * mode
        kap = (8 * np.sin(k * dx) - np.sin(2 * k * dx)) / (6 * dx)
        f = np.cos(k * a) * np.cos(2 * np.pi * b)
        np.testing.assert_allclose(oracle.diff1(m, f, 0),
                                   -kap * np.sin(k * a) * np.cos(2 * np.pi * b), atol=1e-12 * k)
        # second derivative: -(16 sin^2(k dx/2) - sin^2(k dx)) * 4/(12 dx^2) ... written as
        # the symbol of the five-point stencil: (-2cos(2kdx) + 32cos(kdx) - 30) / (12 dx^2)
        sym = (-2 * np.cos(2 * k * dx) + 32 * np.cos(k * dx) - 30) / (12 * dx * dx)
        g = np.cos(k * a)
        np.testing.assert_allclose(oracle.laplacian(m, g), sym * g, atol=1e-10 * k * k)


def test_periodic_seam_shift():
    # z1 = alpha1 is not periodic but jumps by L1 across the seam: its derivative is 1 everywhere
    n = 8
    for L in (1.0, 2.5):
        m = oracle.Mesh(n, L1=L, L2=L, periodic=True)
        a, b = inputs.mesh_coords(n, L1=L, L2=L)
        np.testing.assert_allclose(oracle.diff1(m, a, 0, shift=L), 1.0, rtol=0, atol=1e-13)
        np.testing.assert_allclose(oracle.diff1(m, b, 1, shift=L), 1.0, rtol=0, atol=1e-13)
        np.testing.assert_allclose(oracle.diff1(m, a, 1, shift=0.0), 0.0, rtol=0, atol=1e-13)


def test_vorticity_derivative_terms():
    # dw/dt = -2 A grad Phi + mu Lap w: with quadratic Phi and quintic w both stencils are exact
    # in the interior, so the result is the analytic expression
    n = 16
    m = oracle.Mesh(n, periodic=False)
    a, b = grid(n)
    phi = 0.5 * a * a - 1.5 * a * b + 0.25 * b * b
    w = np.stack([a**5 + b**3, a * a * b - b**5])
    A, mu = 0.35, 0.02
    lap = np.stack([20 * a**3 + 6 * b, 2 * b - 20 * b**3])
    grad = np.stack([a - 1.5 * b, -1.5 * a + 0.5 * b])
    inn = interior(n)
    out = oracle.wdot(m, phi, w, A, mu)
    np.testing.assert_allclose(out[:, inn], (-2 * A * grad + mu * lap)[:, inn], atol=1e-9)


# ------------------------------------------------------------------------------------------
# geometry
# ------------------------------------------------------------------------------------------

def test_tilted_plane_geometry():
    n = 10
    c1, c2 = 0.7, -0.4
    m = oracle.Mesh(n, periodic=False)
    a, b = grid(n)
    z = np.stack([a, b, c1 * a + c2 * b])
    a1, a2, h, nrm = oracle.geometry(m, z)
    one = np.ones_like(a)
    np.testing.assert_allclose(a1, np.stack([one, 0 * a, c1 * one]), atol=1e-12)
    np.testing.assert_allclose(a2, np.stack([0 * a, one, c2 * one]), atol=1e-12)
    np.testing.assert_allclose(h[0], 1 + c1 * c1, atol=1e-12)
    np.testing.assert_allclose(h[1], c1 * c2, atol=1e-12)
    np.testing.assert_allclose(h[2], 1 + c2 * c2, atol=1e-12)
    np.testing.assert_allclose(h[3], 1 + c1 * c1 + c2 * c2, atol=1e-12)
    ref = np.array([-c1, -c2, 1.0]) / math.sqrt(1 + c1 * c1 + c2 * c2)
    np.testing.assert_allclose(nrm, ref[:, None] * one, atol=1e-12)


def test_jump_term_lagrange_identity():
    # w^T h^{-1} w = |w1 a2 - w2 a1|^2 / |a1 x a2|^2 (Lagrange's identity), so with g = 0 and
    # u = 0, 8 Phi |a1 x a2|^2 must equal |gamma|^2 computed from the tangents directly.
    n = 16
    m = oracle.Mesh(n, periodic=True)
    z, w = inputs.random_state(n, seed=3)
    a1, a2, h, _ = oracle.geometry(m, z)
    gamma = oracle.sheet_strength(w, a1, a2)
    phi = oracle.phi(z, w, h, np.zeros((3, n * n)), 0.0)
    cross = np.cross(a1.T, a2.T).T
    lhs = 8 * phi * np.sum(cross**2, axis=0)
    gam_np = w[0] * a2 - w[1] * a1
    np.testing.assert_allclose(gamma, gam_np, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(lhs, np.sum(gam_np**2, axis=0), rtol=1e-12)
    np.testing.assert_allclose(h[3], np.sum(cross**2, axis=0), rtol=1e-12)
    # the other two Phi terms separately
    u = np.random.default_rng(1).normal(size=(3, n * n))
    phi_u = oracle.phi(z, np.zeros((2, n * n)), h, u, 0.0)
    np.testing.assert_allclose(phi_u, 0.5 * np.einsum("cp,cp->p", u, u), rtol=1e-14)
    phi_g = oracle.phi(z, np.zeros((2, n * n)), h, np.zeros((3, n * n)), 9.81)
    np.testing.assert_allclose(phi_g, 9.81 * z[2], rtol=1e-15)


# ------------------------------------------------------------------------------------------
# Birkhoff-Rott sum
# ------------------------------------------------------------------------------------------

def test_flat_rest_is_exactly_at_rest():
    n = 16
    for periodic in (False, True):
        m = oracle.Mesh(n, periodic=periodic)
        a, b = grid(n)
        z = np.stack([a, b, 0 * a])
        w = np.zeros((2, n * n))
        u, wd = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, 0.1 / n)
        assert np.all(u == 0.0) and np.all(wd == 0.0)
        z2, w2 = oracle.run(m, z, w, 0.5, 1.0, 0.0, 0.1 / n, 1e-3, 2)
        # u = 0 and wdot = 0 exactly at every stage; the RK3 combination 3/4 y + 1/4 y only
        # rounds the in-plane coordinates (z3 and w stay exactly zero)
        assert np.all(z2[2] == 0.0) and np.all(w2 == 0.0)
        np.testing.assert_allclose(z2[:2], z[:2], rtol=4e-16, atol=0)


def test_flat_sheet_has_no_in_plane_velocity():
    n = 16
    m = oracle.Mesh(n, periodic=False)
    a, b = grid(n)
    z = np.stack([a, b, 0 * a])
    _, w = inputs.random_state(n, seed=5)
    u, _ = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, 0.1 / n)
    assert np.all(u[0] == 0.0) and np.all(u[1] == 0.0)
    assert np.max(np.abs(u[2])) > 1e-3


def test_pair_antisymmetry_and_momentum_balance():
    rng = np.random.default_rng(7)
    za, zb = rng.normal(size=3), rng.normal(size=3)
    g = rng.normal(size=3)
    z = np.stack([za, zb], axis=1)
    gam = np.stack([g, g], axis=1)
    u = oracle.br_velocity(z, z, gam, 0.3, 0.05)
    assert np.array_equal(u[:, 0], -u[:, 1])
    # uniform strength: the pair terms cancel in the total
    zs = rng.normal(size=(3, 200))
    gam = np.repeat(rng.normal(size=(3, 1)), 200, axis=1)
    u = oracle.br_velocity(zs, zs, gam, 0.01, 0.02)
    tot = np.abs(u).sum()
    assert np.all(np.abs(u.sum(axis=1)) <= 1e-13 * tot)


def test_translation_rotation_and_scaling():
    rng = np.random.default_rng(11)
    n = 12
    z, w = inputs.random_state(n, seed=2)
    m = oracle.Mesh(n, periodic=True)
    a1, a2, _, _ = oracle.geometry(m, z)
    gam = oracle.sheet_strength(w, a1, a2)
    wt, de = 1.0 / n**2, 0.1 / n
    u = oracle.br_velocity(z, z, gam, wt, de)
    scale = np.abs(u).max()
    # translation
    ut = oracle.br_velocity(z + np.array([[0.3], [-1.2], [0.7]]), z + np.array([[0.3], [-1.2], [0.7]]),
                            gam, wt, de)
    np.testing.assert_allclose(ut, u, atol=1e-12 * scale)
    # rotation: u(Qz, Q gamma) = Q u(z, gamma)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    ur = oracle.br_velocity(q @ z, q @ z, q @ gam, wt, de)
    np.testing.assert_allclose(ur, q @ u, atol=1e-12 * scale)
    # power-of-two scaling of positions and core size is exact: u -> u / 4
    us = oracle.br_velocity(2 * z, 2 * z, gam, wt, 2 * de)
    assert np.array_equal(us, u / 4)


def test_gaussian_sheet_closed_form():
    """Flat sheet carrying mu = exp(-rho^2 / 2s^2): the continuous desingularised sum is
    u3(rho) = -(s^2/2) int_0^inf k^2 exp(-k delta - s^2 k^2 / 2) J0(k rho) dk; with delta = 5 dx
    the trapezoidal sum reproduces it up to aliasing of order exp(-2 pi delta / dx)."""
    integrate = pytest.importorskip("scipy.integrate")
    special = pytest.importorskip("scipy.special")
    n = 128
    dx = 1.0 / n
    s, delta = 6 * dx, 5 * dx
    a, b = grid(n)
    x0 = y0 = (n // 2) * dx
    rho2 = (a - x0) ** 2 + (b - y0) ** 2
    mu = np.exp(-rho2 / (2 * s * s))
    w1, w2 = -(a - x0) / (s * s) * mu, -(b - y0) / (s * s) * mu
    z = np.stack([a, b, 0 * a])
    gam = np.stack([-w2, w1, 0 * a])  # w1 a2 - w2 a1 with a1 = e1, a2 = e2
    tidx = [(n // 2) * n + n // 2, (n // 2) * n + n // 2 + 6, (n // 2 + 9) * n + n // 2 + 3,
            (n // 2 - 13) * n + n // 2 + 1]
    u = oracle.br_velocity(z[:, tidx], z, gam, dx * dx, delta)
    for k, t in enumerate(tidx):
        rho = math.sqrt(rho2[t])
        f = lambda q: q * q * math.exp(-q * delta - s * s * q * q / 2) * special.j0(q * rho)
        val, _ = integrate.quad(f, 0, np.inf, epsabs=0, epsrel=1e-13, limit=500)
        ref = -(s * s / 2) * val
        assert abs(u[2, k] - ref) <= 2e-11 * abs(ref), (rho / dx, u[2, k], ref)
        assert u[0, k] == 0.0 and u[1, k] == 0.0


def test_sheet_response_converges_to_riesz():
    """Flat free-edge sheet with mu = cos(k a) cos(k b): in the interior, u3 -> -|k| mu / 2 as
    dx -> 0 with delta = 0.1 dx.  The lattice sum is first-order accurate, so a Richardson
    extrapolation of two resolutions recovers the continuous value."""
    ratios = []
    for n in (32, 64):
        a, b = grid(n)
        dx = 1.0 / n
        k1 = 2 * np.pi * 2
        mu = np.cos(k1 * a) * np.cos(k1 * b)
        w1 = -k1 * np.sin(k1 * a) * np.cos(k1 * b)
        w2 = -k1 * np.cos(k1 * a) * np.sin(k1 * b)
        z = np.stack([a, b, 0 * a])
        gam = np.stack([-w2, w1, 0 * a])
        i, j = np.arange(n * n) // n, np.arange(n * n) % n
        idx = np.where((i >= n // 4) & (i < 3 * n // 4) & (j >= n // 4) & (j < 3 * n // 4))[0]
        u = oracle.br_velocity(z[:, idx], z, gam, dx * dx, 0.1 * dx)
        kk = k1 * math.sqrt(2)
        ratios.append(np.sum(u[2] * mu[idx]) / np.sum(-0.5 * kk * mu[idx] ** 2))
    assert 0.75 < ratios[0] < ratios[1] < 1.0
    assert abs(2 * ratios[1] - ratios[0] - 1.0) < 0.01


def test_brute_force_50_digits():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(19)
    N = 48
    z = rng.normal(size=(3, N)) * 0.3
    gam = rng.normal(size=(3, N))
    wt, de = 1.0 / 64, 0.02
    u = oracle.br_velocity(z, z, gam, wt, de)
    eps = {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}
    pref = -mpmath.mpf(wt) / (4 * mpmath.pi)
    d2 = mpmath.mpf(de) ** 2
    for i in range(0, N, 5):
        acc = [mpmath.mpf(0)] * 3
        for j in range(N):
            r = [mpmath.mpf(z[c, i]) - mpmath.mpf(z[c, j]) for c in range(3)]
            kern = (r[0] ** 2 + r[1] ** 2 + r[2] ** 2 + d2) ** mpmath.mpf(-1.5)
            for (c, p, q), sgn in eps.items():
                acc[c] += sgn * r[p] * mpmath.mpf(gam[q, j]) * kern
        ref = np.array([float(pref * x) for x in acc])
        np.testing.assert_allclose(u[:, i], ref, rtol=0, atol=1e-14 * np.abs(ref).max())


def test_cutoff_sum_decomposes_the_exact_sum():
    """The cutoff sum plus the exact sum over the excluded sources (chosen here by explicit
    distances) is the exact sum; a cutoff past the cloud's diameter is the exact sum itself and
    one below the smallest distance leaves only the (zero) self term."""
    rng = np.random.default_rng(23)
    N = 300
    z = rng.uniform(0, 1, size=(3, N)) * np.array([[1.0], [1.0], [0.2]])
    gam = rng.normal(size=(3, N))
    wt, de, c = 1e-3, 0.01, 0.3
    ucut = oracle.br_velocity_cutoff(z, z, gam, wt, de, c)
    uex = oracle.br_velocity(z, z, gam, wt, de)
    dist = np.linalg.norm(z[:, :, None] - z[:, None, :], axis=0)
    for i in range(0, N, 7):
        far = np.where(dist[i] > c * (1 + 1e-6))[0]
        border = np.where(np.abs(dist[i] - c) <= c * 1e-6)[0]
        assert len(border) == 0  # no pair sits on the FP32 decision boundary in this cloud
        ufar = oracle.br_velocity(z[:, [i]], z[:, far], gam[:, far], wt, de)[:, 0]
        np.testing.assert_allclose(ucut[:, i] + ufar, uex[:, i], rtol=0, atol=1e-13 * np.abs(uex[:, i]).max())
    assert np.array_equal(oracle.br_velocity_cutoff(z, z, gam, wt, de, 10.0), uex)
    assert np.all(oracle.br_velocity_cutoff(z, z, gam, wt, de, 1e-6) == 0.0)


def test_cutoff_boundary_is_the_fp64_distance():
    """Sec. 3.2.2 counts the sources within the cutoff distance: a source at exactly the cutoff
    is in, and sources 2^-40 (relative) inside and outside the cutoff are in and out.  FP32
    cannot tell the three distances apart (they round to the same float), so an FP32 decision,
    a strict inequality or an unsquared comparison each fail here."""
    c = 0.25
    zt = np.zeros((3, 1))
    eps = 2.0 ** -40
    for x, want_in in ((c, True), (c * (1 - eps), True), (c * (1 + eps), False),
                       (c * 0.5, True), (c * 1.5, False)):
        zs = np.array([[x], [0.0], [0.0]])
        gam = np.array([[0.0], [0.0], [1.0]])
        u = oracle.br_velocity_cutoff(zt, zs, gam, 1.0, 0.01, c)
        ref = oracle.br_velocity(zt, zs, gam, 1.0, 0.01)
        assert ref[1, 0] != 0.0
        assert np.array_equal(u, ref if want_in else np.zeros_like(ref)), (x, want_in)
        assert oracle.within_cutoff(zt[:, 0], zs[:, 0], c) == want_in
    # the decision uses all three components: (0.15, 0.2, 0) lies at 0.25 up to rounding, and
    # (0.15, 0.2, 0.01) clearly outside
    assert not oracle.within_cutoff([0, 0, 0], [0.15, 0.2, 0.01], c)
    assert oracle.within_cutoff([0, 0, 0], [0.15, 0.2, 0.0], c * (1 + 1e-12))
    assert oracle.within_cutoff([1.0, 2.0, 3.0], [1.0, 2.0, 3.0 + c * (1 - 1e-9)], c)


# ------------------------------------------------------------------------------------------
# Riesz transform / FFT
# ------------------------------------------------------------------------------------------

def test_fft_matches_numpy():
    rng = np.random.default_rng(4)
    for n1, n2 in ((8, 16), (32, 32), (4, 64)):
        x = rng.normal(size=(n1, n2)) + 1j * rng.normal(size=(n1, n2))
        re, im = oracle.fft2(x.real, x.imag, -1)
        np.testing.assert_allclose(re + 1j * im, np.fft.fft2(x), atol=1e-12 * n1 * n2)
        re, im = oracle.fft2(x.real, x.imag, +1)
        np.testing.assert_allclose(re + 1j * im, np.fft.ifft2(x) * n1 * n2, atol=1e-12 * n1 * n2)


def test_fft_any_length_matches_numpy():
    # lengths that are not powers of two go through the general Cooley-Tukey path: composite
    # (12, 24, 38 = 2 x 19, 152 = 8 x 19), prime (5, 7, 19) and odd composite (9, 15)
    rng = np.random.default_rng(5)
    for n1, n2 in ((12, 19), (38, 24), (152, 9), (5, 7), (15, 16), (16, 152)):
        x = rng.normal(size=(n1, n2)) + 1j * rng.normal(size=(n1, n2))
        re, im = oracle.fft2(x.real, x.imag, -1)
        np.testing.assert_allclose(re + 1j * im, np.fft.fft2(x), atol=1e-12 * n1 * n2)
        re, im = oracle.fft2(x.real, x.imag, +1)
        np.testing.assert_allclose(re + 1j * im, np.fft.ifft2(x) * n1 * n2, atol=1e-12 * n1 * n2)


@pytest.mark.parametrize("n1,n2,m1,m2", [(38, 24, 5, -7), (19, 15, 9, -7), (152, 40, -60, 11)])
def test_riesz_gradient_mode_any_side(n1, n2, m1, m2):
    # the closed form R . grad cos(phase) = |k| cos(phase) on sides that are not powers of two,
    # including odd sides with the highest frequency they carry ((n - 1) / 2), which a wrong
    # signed-frequency map would send to the wrong |k|
    m = oracle.Mesh(n1, n2, L1=1.0, L2=2.0, periodic=True)
    a, b = inputs.mesh_coords(n1, n2, 1.0, 2.0)
    k1, k2 = 2 * np.pi * m1 / 1.0, 2 * np.pi * m2 / 2.0
    ph = k1 * a + k2 * b + 0.4
    kk = math.hypot(k1, k2)
    w = np.stack([-k1 * np.sin(ph), -k2 * np.sin(ph)])
    np.testing.assert_allclose(oracle.riesz_scalar(m, w), kk * np.cos(ph), atol=1e-11 * kk)
    wc = np.stack([-k2 * np.sin(ph), k1 * np.sin(ph)])
    np.testing.assert_allclose(oracle.riesz_scalar(m, wc), 0.0, atol=1e-11 * kk)


def test_riesz_gradient_mode_and_curl():
    n1, n2 = 32, 16
    m = oracle.Mesh(n1, n2, L1=1.0, L2=2.0, periodic=True)
    a, b = inputs.mesh_coords(n1, n2, 1.0, 2.0)
    k1, k2 = 2 * np.pi * 3 / 1.0, 2 * np.pi * (-2) / 2.0
    ph = k1 * a + k2 * b + 0.4
    kk = math.hypot(k1, k2)
    # w = grad cos(phase): R . w = |k| cos(phase)
    w = np.stack([-k1 * np.sin(ph), -k2 * np.sin(ph)])
    np.testing.assert_allclose(oracle.riesz_scalar(m, w), kk * np.cos(ph), atol=1e-12 * kk)
    # a curl field (w1, w2) = (d2 psi, -d1 psi) is annihilated
    wc = np.stack([-k2 * np.sin(ph), k1 * np.sin(ph)])
    np.testing.assert_allclose(oracle.riesz_scalar(m, wc), 0.0, atol=1e-12 * kk)
    # the constant mode and the Nyquist row carry no velocity (the odd multiplier is not
    # Hermitian there, so it is zeroed)
    wn = np.stack([np.ones_like(a), np.cos(np.pi * n1 * a) * np.cos(2 * np.pi * 3 * b / 2.0)])
    np.testing.assert_allclose(oracle.riesz_scalar(m, wn), 0.0, atol=1e-12)
    # low-order velocity on a flat sheet: u = (0, 0, -s/2)
    z = np.stack([a, b, 0 * a])
    u, _ = oracle.derivative(m, z, w, 0.5, 1.0, 0.0, 0.0, order=oracle.ORDER_LOW)
    np.testing.assert_allclose(u[2], -0.5 * kk * np.cos(ph), atol=1e-12 * kk)
    assert np.all(u[0] == 0.0) and np.all(u[1] == 0.0)


def test_medium_order_composition():
    """Medium order moves the interface with the Birkhoff-Rott velocity and updates the vorticity
    with the FFT velocity, so its u equals the high-order u and its dw/dt the low-order dw/dt."""
    n = 32
    m = oracle.Mesh(n, periodic=True)
    z, w = inputs.random_state(n, seed=17)
    args = (0.6, 1.2, 0.01, 0.1 / n)
    um, wm = oracle.derivative(m, z, w, *args, order=oracle.ORDER_MEDIUM)
    uh, wh = oracle.derivative(m, z, w, *args, order=oracle.ORDER_HIGH)
    ul, wl = oracle.derivative(m, z, w, *args, order=oracle.ORDER_LOW)
    assert np.array_equal(um, uh) and np.array_equal(wm, wl)
    assert not np.array_equal(uh, ul) and not np.array_equal(wh, wl)


# ------------------------------------------------------------------------------------------
# time integration and the linear Rayleigh-Taylor limit
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [(2, 3), (1, 0), (5, -4)])
def test_linear_rt_low_order_exact(mode):
    """One small-amplitude mode z3 = eps cos(k.a), w = 0.  The linearised low-order system on
    (a, b) = (z3 amplitude, s amplitude) is d/dt (a, b) = M (a, b) with
    M = [[0, -1/2], [-2 A g (k.kappa)/|k|, 0]] (kappa: stencil's modified wavenumber), so each
    SSP-RK3 step multiplies it by P(dt M) = I + dtM + (dtM)^2/2 + (dtM)^3/6."""
    n = 32
    eps, A, g, dt, nsteps = 1e-9, 0.5, 10.0, 0.01, 20
    m = oracle.Mesh(n, periodic=True)
    a, b = grid(n)
    m1, m2 = mode
    ph = 2 * np.pi * (m1 * a + m2 * b)
    z = np.stack([a, b, eps * np.cos(ph)])
    w = np.zeros((2, n * n))
    z2, w2 = oracle.run(m, z, w, A, g, 0.0, 0.0, dt, nsteps, order=oracle.ORDER_LOW)
    dx = 1.0 / n
    k = np.array([2 * np.pi * m1, 2 * np.pi * m2])
    kk = np.linalg.norm(k)
    kap = (8 * np.sin(k * dx) - np.sin(2 * k * dx)) / (6 * dx)
    M = np.array([[0.0, -0.5], [-2 * A * g * (k @ kap) / kk, 0.0]])
    Z = dt * M
    P = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6
    y = np.linalg.matrix_power(P, nsteps) @ np.array([eps, 0.0])
    meas = 2.0 / (n * n) * np.sum(z2[2] * np.cos(ph))
    assert abs(meas / y[0] - 1) < 1e-8
    # and close to the continuous growth cosh(sigma t), sigma^2 = A g (k.kappa)/|k|
    sig = math.sqrt(A * g * (k @ kap) / kk)
    assert abs(meas / (eps * math.cosh(sig * dt * nsteps)) - 1) < 1e-3


@pytest.mark.slow
def test_linear_rt_high_order_growth_rate():
    """Single mode on a free-edge sheet, high order (all-pairs BR, delta = 0.1 dx): the interior
    amplitude follows cosh(sigma t) with sigma = sqrt(A |k| g) up to the first-order lattice
    error of the desingularised sum (about 0.3 k dx in the response) and edge effects."""
    n = 64
    eps, A, g = 1e-6, 0.5, 4.0
    m = oracle.Mesh(n, periodic=False)
    a, b = grid(n)
    mm = 2
    shape = np.cos(2 * np.pi * mm * a) * np.cos(2 * np.pi * mm * b)
    z = np.stack([a, b, eps * shape])
    w = np.zeros((2, n * n))
    kk = 2 * np.pi * mm * math.sqrt(2)
    sig = math.sqrt(A * kk * g)
    nst = 10
    dt = 2.0 / sig / nst
    z2, _ = oracle.run(m, z, w, A, g, 0.0, 0.1 / n, dt, nst, order=oracle.ORDER_HIGH)
    i, j = np.arange(n * n) // n, np.arange(n * n) % n
    inn = (i >= n // 4) & (i < 3 * n // 4) & (j >= n // 4) & (j < 3 * n // 4)
    amp = np.sum(z2[2][inn] * shape[inn]) / np.sum(shape[inn] ** 2) / eps
    ref = math.cosh(2.0)
    assert 0.85 * ref < amp < 1.02 * ref, (amp, ref)
