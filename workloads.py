"""Seeded synthetic workloads (inputs only; no arithmetic of the scheme lives here).

The paper's workloads are analytic PEC cavity modes (Sec. 5.1, Eq. "eq:data"); these
generators draw the mode indices and amplitudes of each configuration from numpy's PCG64
with a recorded seed.  Both the oracle-side tests and the GPU path take their inputs from
here, so neither imports the other.
"""
from __future__ import annotations

import numpy as np


def config1():
    """2D TM_z, 64 x 64 cells, r = 0.5, mode (2, 3) with unit amplitude, run to t = 1 (128 steps)."""
    return dict(n=64, r=0.5, modes=[(2, 3, 1.0)], steps=128)


def config2(seed: int = 0):
    """2D TM_z, 2048 x 2048 cells, r = 0.5, 4000 steps; 8 modes with (m, n) uniform in [1, 40]
    and N(0, 1) amplitudes."""
    rng = np.random.default_rng(seed)
    mn = rng.integers(1, 41, size=(8, 2))
    amp = rng.standard_normal(8)
    return dict(n=2048, r=0.5, modes=[(int(a), int(b), float(c)) for (a, b), c in zip(mn, amp)], steps=4000)


def random_modes(count: int, kmax: int, seed: int):
    """`count` modes with indices uniform in [1, kmax] and N(0, 1) amplitudes."""
    rng = np.random.default_rng(seed)
    mn = rng.integers(1, kmax + 1, size=(count, 2))
    amp = rng.standard_normal(count)
    return [(int(a), int(b), float(c)) for (a, b), c in zip(mn, amp)]


def random_fields(n: int, seed: int):
    """Random staggered fields (E_z, H_x, H_y) with zero Dirichlet boundary values."""
    rng = np.random.default_rng(seed)
    ez = np.zeros((n + 1, n + 1))
    hx = np.zeros((n, n + 1))
    hy = np.zeros((n + 1, n))
    ez[1:-1, 1:-1] = rng.standard_normal((n - 1, n - 1))
    hx[:, 1:-1] = rng.standard_normal((n, n - 1))
    hy[1:-1, :] = rng.standard_normal((n - 1, n))
    return ez, hx, hy


def config4(seed: int = 0):
    """512 independent 2D TM_z cavities, r = 0.5, 1000 steps; side lengths uniform in
    {64, 96, ..., 768}; each cavity has 4 modes with indices uniform in [1, 30] and N(0, 1)
    amplitudes."""
    rng = np.random.default_rng(seed)
    sizes = [int(64 + 32 * k) for k in rng.integers(0, 23, size=512)]
    modes = []
    for _ in sizes:
        mn = rng.integers(1, 31, size=(4, 2))
        amp = rng.standard_normal(4)
        modes.append([(int(a), int(b), float(c)) for (a, b), c in zip(mn, amp)])
    return dict(sizes=sizes, r=0.5, modes=modes, steps=1000)
