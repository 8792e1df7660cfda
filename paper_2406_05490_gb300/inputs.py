"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only *draws* interfaces and workloads; it contains none of the method's arithmetic
(no stencils, no Birkhoff-Rott sum, no time stepping).  Every generator is deterministic in its
seed (numpy PCG64 via ``default_rng``).  The shapes and value distributions stand in for the
rocket-rig single-mode and multi-mode decks of Beatnik (Sec. 4), which are not published:

* single mode: z = (a, b, amp * cos(2 pi a) cos(2 pi b)) on [0,1)^2, w = 0;
* multi mode: z3 = sum_m a_m cos(2 pi (kx_m a + ky_m b) + phi_m) with integer (kx, ky) drawn
  uniformly from [kmin, kmax]^2, a_m ~ N(0, amp_std) (or a fixed amplitude), phi_m ~ U[0, 2pi);
* ragged batches and Poisson serving traces with log-uniform mesh sides.

Arrays are float64, component-major: z has shape (3, n1*n2), w has shape (2, n1*n2), node
p = i*n2 + j with i along the first parameter direction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def mesh_coords(n1, n2=None, L1=1.0, L2=1.0):
    """Parameter coordinates (alpha1, alpha2) of every node, flattened (p = i*n2 + j)."""
    n2 = n1 if n2 is None else n2
    a1 = (np.arange(n1, dtype=np.float64) * (L1 / n1))[:, None] * np.ones((1, n2))
    a2 = np.ones((n1, 1)) * (np.arange(n2, dtype=np.float64) * (L2 / n2))[None, :]
    return a1.reshape(-1), a2.reshape(-1)


def single_mode(n, amp=0.05):
    """Single-mode rocket-rig interface: z3 = amp cos(2 pi a) cos(2 pi b), w = 0."""
    a, b = mesh_coords(n)
    z = np.stack([a, b, amp * np.cos(2 * np.pi * a) * np.cos(2 * np.pi * b)])
    w = np.zeros((2, n * n))
    return z, w


def draw_modes(rng, n_modes, kmin=2, kmax=8, amp_std=None, amp=None):
    """Integer wave vectors, amplitudes and phases for a multi-mode perturbation."""
    kx = rng.integers(kmin, kmax + 1, size=n_modes)
    ky = rng.integers(kmin, kmax + 1, size=n_modes)
    if amp is not None:
        a = np.full(n_modes, float(amp))
    else:
        a = rng.normal(0.0, amp_std, size=n_modes)
    ph = rng.uniform(0.0, 2 * np.pi, size=n_modes)
    return kx, ky, a, ph


def multi_mode(n, n_modes=16, seed=0, kmin=2, kmax=8, amp_std=0.01, amp=None):
    """Multi-mode periodic interface z3 = sum a cos(2 pi (kx a + ky b) + phi), w = 0."""
    rng = np.random.default_rng(seed)
    kx, ky, a_m, ph = draw_modes(rng, n_modes, kmin, kmax, amp_std=amp_std, amp=amp)
    a, b = mesh_coords(n)
    z3 = np.zeros(n * n)
    for m in range(n_modes):
        z3 += a_m[m] * np.cos(2 * np.pi * (kx[m] * a + ky[m] * b) + ph[m])
    z = np.stack([a, b, z3])
    w = np.zeros((2, n * n))
    return z, w


def random_state(n1, n2=None, seed=0, z_amp=0.05, w_amp=0.5, n_modes=6, periodic=True):
    """A smooth interface with non-zero vorticity, for single-evaluation parity tests.

    Both z3 and w are sums of a few low Fourier modes (so that the free-edge and periodic
    ghost rules both see smooth data); w is not a gradient, which exercises every term.
    """
    n2 = n1 if n2 is None else n2
    rng = np.random.default_rng(seed)
    a, b = mesh_coords(n1, n2)
    z3 = np.zeros(n1 * n2)
    w = np.zeros((2, n1 * n2))
    for _ in range(n_modes):
        kx, ky = rng.integers(1, 4, size=2)
        z3 += z_amp / n_modes * rng.normal() * np.cos(2 * np.pi * (kx * a + ky * b) + rng.uniform(0, 6.3))
        for c in range(2):
            w[c] += w_amp / n_modes * rng.normal() * np.sin(2 * np.pi * (kx * a - ky * b) + rng.uniform(0, 6.3))
    # small in-plane displacements keep the seam shift and the general geometry honest
    z1 = a + 0.01 * np.sin(2 * np.pi * b + rng.uniform(0, 6.3))
    z2 = b + 0.01 * np.sin(2 * np.pi * a + rng.uniform(0, 6.3))
    return np.stack([z1, z2, z3]), w


@dataclass
class Instance:
    """One interface of a ragged batch or serving trace."""
    n: int
    atwood: float
    z: np.ndarray
    w: np.ndarray
    seed: int
    arrival_s: float = 0.0
    nsteps: int = 0
    extra: dict = field(default_factory=dict)


def log_uniform_sides(rng, count, lo, hi):
    """Integer mesh sides drawn log-uniformly in [lo, hi]."""
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return np.clip(np.rint(s).astype(int), lo, hi)


def ragged_batch(count=64, lo=64, hi=384, n_modes=4, seed=0, amp_std=0.01):
    """Batch of independent periodic interfaces with log-uniform sides and A ~ U[0.2, 0.8]."""
    rng = np.random.default_rng(seed)
    sides = log_uniform_sides(rng, count, lo, hi)
    out = []
    for k, n in enumerate(sides):
        at = float(rng.uniform(0.2, 0.8))
        s = int(rng.integers(0, 2**31 - 1))
        z, w = multi_mode(int(n), n_modes=n_modes, seed=s, amp_std=amp_std)
        out.append(Instance(n=int(n), atwood=at, z=z, w=w, seed=s))
    return out


def poisson_trace(count=256, rate_hz=200.0, lo=32, hi=512, nsteps=20, n_modes=4, seed=0,
                  amp_std=0.01):
    """Serving trace: Poisson arrivals at rate_hz, log-uniform sides, multi-mode interfaces."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    sides = log_uniform_sides(rng, count, lo, hi)
    out = []
    for k in range(count):
        s = int(rng.integers(0, 2**31 - 1))
        at = float(rng.uniform(0.2, 0.8))
        z, w = multi_mode(int(sides[k]), n_modes=n_modes, seed=s, amp_std=amp_std)
        out.append(Instance(n=int(sides[k]), atwood=at, z=z, w=w, seed=s, arrival_s=float(t[k]),
                            nsteps=nsteps))
    return out
