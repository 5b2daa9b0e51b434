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


def sine_series_field(n: int, ell: float, seed: int, mmax: int = 96):
    """Gaussian random field on the (n+1)^2 E_z nodes as a sine series
    sum a_mn sin(m pi x) sin(n pi y), a_mn ~ N(0, 1) exp(-pi^2 (m^2 + n^2) ell^2 / 4), m, n <= mmax
    (zero on the walls), normalised to unit RMS over the interior nodes."""
    rng = np.random.default_rng(seed)
    mc = min(mmax, n - 1)
    k = np.arange(1, mc + 1)
    env = np.exp(-np.pi ** 2 * (k[:, None] ** 2 + k[None, :] ** 2) * ell ** 2 / 4.0)
    a = rng.standard_normal((mc, mc)) * env
    # sin(k pi i / n) with the argument reduced exactly in integers
    q = np.mod(np.outer(np.arange(n + 1), k), 2 * n)
    s = np.sin(np.pi * q / n)
    s[0, :] = 0.0
    s[n, :] = 0.0
    f = s @ a.T @ s.T  # f[j, i] = sum_mn a_mn sin(m pi x_i) sin(n pi y_j)
    rms = np.sqrt(np.mean(f[1:-1, 1:-1] ** 2))
    return f / rms


def config5(seed: int = 0, n: int = 1024, steps: int = 2000):
    """Reverse-pass workload: 2D TM_z, n x n cells, r = 0.5, `steps` steps.  E_z^0 is a Gaussian
    random field of correlation length 0.05 (sine series, unit RMS), H^0 = 0 and H^{1/2} from the
    Taylor series; the target is a 4-mode superposition (indices uniform in [1, 30], N(0, 1)
    amplitudes) at the final time; 16 directions are further fields of the same law."""
    rng = np.random.default_rng(seed)
    seeds = rng.integers(0, 2 ** 31, size=18)
    mn = rng.integers(1, 31, size=(4, 2))
    amp = rng.standard_normal(4)
    return dict(n=n, r=0.5, steps=steps, ell=0.05,
                ez0_seed=int(seeds[0]), direction_seeds=[int(x) for x in seeds[2:18]],
                target_modes=[(int(a), int(b), float(c)) for (a, b), c in zip(mn, amp)])


def mode3(m: int, n: int, p: int, amp: float):
    """3D cavity mode with polarisation amp (-n, m, 0) / max(m, n) (divergence-free; the largest
    component has magnitude |amp|)."""
    s = amp / max(m, n)
    return (int(m), int(n), int(p), -n * s, m * s, 0.0)


def config3(seed: int = 0):
    """3D six-component cavity, 256^3 cells, r = 0.4, 500 steps: mode (2, 3, 1) with unit
    amplitude plus one mode with (m, n, p) uniform in [1, 16] and an N(0, 1) amplitude."""
    rng = np.random.default_rng(seed)
    mnp = rng.integers(1, 17, size=3)
    amp = float(rng.standard_normal())
    return dict(n=256, r=0.4, steps=500, modes=[mode3(2, 3, 1, 1.0), mode3(*[int(v) for v in mnp], amp)])


def random_fields3(n: int, seed: int):
    """Random 3D staggered fields (E_x, E_y, E_z, H_x, H_y, H_z), [z][y][x], with zero values at
    the walls of every component's node axes."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(6):
        node = [(a != c % 3) if c < 3 else (a == c % 3) for a in range(3)]
        nx, ny, nz = (n + 1 if q else n for q in node)
        f = rng.standard_normal((nz, ny, nx))
        if node[0]:
            f[:, :, 0] = f[:, :, -1] = 0.0
        if node[1]:
            f[:, 0, :] = f[:, -1, :] = 0.0
        if node[2]:
            f[0, :, :] = f[-1, :, :] = 0.0
        out.append(f)
    return out
