"""Pins of the tracked-Delta-E variant of the oracle (Sec. 3.4 as printed: Delta E advanced by
the modified Helmholtz equation Eq. "eq:mhe", Step 2 filtered with it as in Eq. "eq:helm2"):
the closed-form per-mode recurrence under the REFLECT closure, and Table "table:cfl"."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from closed_forms import mode_basis, mode_step_matrix_tracked

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("kx,ky,Z", [(2, 3, 1.0), (5, 1, 2.5), (7, 6, 0.6)])
def test_reflect_tracked_step_is_mode_recurrence(kx, ky, Z):
    N, r, K = 16, 0.5, 7
    o = oracle.Oracle2D(N, r, Z=Z, closure=oracle.CLOSURE_REFLECT)
    ez_b, hx_b, hy_b = mode_basis(N, kx, ky)
    coef = np.random.default_rng(kx * 10 + ky).standard_normal(4)
    ez, hx, hy, de = coef[0] * ez_b, coef[1] * hx_b, coef[2] * hy_b, coef[3] * ez_b
    for _ in range(K):
        o.step_tracked(ez, hx, hy, de)
    want = np.linalg.matrix_power(mode_step_matrix_tracked(N, r, kx, ky, Z), K) @ coef
    for got, w, b in ((ez, want[0], ez_b), (hx, want[1], hx_b), (hy, want[2], hy_b)):
        assert np.abs(got - w * b).max() <= 1e-12 * max(1.0, np.abs(w * b).max())
    # the Delta E update cancels terms of size kappa^2 |E|: rounding relative to that scale
    scale = o.kappa2 * max(1.0, np.abs(ez).max())
    assert np.abs(de - want[3] * ez_b).max() <= 1e-14 * scale


def test_table_cfl_c4_column_tracked():
    """With Delta E^0 exact for the mode, the tracked variant reproduces the C4 column of Table
    "table:cfl" within 3% for both wavenumbers and every CFL number."""
    g = json.load(open(os.path.join(GOLDEN, "table_cfl_c4.json")))
    N, T = g["N"], g["T"]
    for k in (2, 21):
        for rn, want in zip(g["r_numerators_over_6sqrt2"], g["mae"][str(k)]):
            o = oracle.Oracle2D(N, rn / (6 * math.sqrt(2)))
            modes = [(k, k, 1.0)]
            K = int(round(T / o.ht))
            ez, hx, hy = o.init_modes(modes)
            de = -(math.pi ** 2) * (2 * k * k) * ez
            acc = 0.0
            for n in range(1, K + 1):
                o.step_tracked(ez, hx, hy, de)
                acc += o.error(modes, n, ez, hx, hy)[3]
            got = acc / (3.0 * K * N * N)
            assert abs(got - want) <= 0.03 * want, (k, rn, got, want)
