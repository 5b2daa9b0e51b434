"""Pins of the NC comparator in the oracle (Sec. 5.2, stencil K4 with a = 0, fourth-order
one-sided differences at the line ends): exactness of the derivative on polynomials, the NC
column of Table "table:cfl" and the NC grid-convergence rates of Table "table:conv_rates"."""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("nin", [6, 11])
def test_derivative_exact_on_cubics(nin):
    h = 0.37
    for start in (0.0, 0.5):  # node lines (x_0 = 0) and half-node lines (x_0 = h/2)
        x = (start + np.arange(nin)) * h
        xo = (start + 0.5 + np.arange(nin - 1)) * h
        for p in range(4):
            d = oracle.nc_line(x ** p, h)
            ref = p * xo ** (p - 1) if p else np.zeros_like(xo)
            assert np.allclose(d, ref, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(ref).max()))
        # degree 4: exact in the interior (central stencil), not at the one-sided ends
        d = oracle.nc_line(x ** 4, h)
        ref = 4 * xo ** 3
        assert np.allclose(d[1:-1], ref[1:-1], rtol=1e-11, atol=1e-11)
        assert abs(d[0] - ref[0]) > 1e-6 and abs(d[-1] - ref[-1]) > 1e-6


def _mae_nc(N, r, k, T):
    o = oracle.Oracle2D(N, r)
    modes = [(k, k, 1.0)]
    K = int(round(T / o.ht))
    f = list(o.init_modes(modes))
    acc = 0.0
    for n in range(1, K + 1):
        o.nc_step(*f)
        acc += o.error(modes, n, *f)[3]
    return acc / (3.0 * K * N * N)


def test_table_cfl_nc_column():
    g = json.load(open(os.path.join(GOLDEN, "table_cfl_nc.json")))
    for rn, want in zip(g["r_num"], g["mae"]):
        got = _mae_nc(g["N"], rn / (6 * math.sqrt(2)), g["k"], g["T"])
        assert abs(got - want) <= 0.05 * want, (rn, got, want)


def test_table_conv_rates_nc():
    g = json.load(open(os.path.join(GOLDEN, "table_conv_rates_nc.json")))
    for case in g["cases"]:
        r = case["r_num"] / (6 * math.sqrt(2))
        errs = {N: _mae_nc(N, r, case["k"], g["T"]) for N in [16] + case["N"][:2]}
        for N, want in zip(case["N"][:2], case["rate"][:2]):
            got = math.log2(errs[N // 2] / errs[N])
            assert abs(got - want) <= 0.1, (case, N, got, want)
