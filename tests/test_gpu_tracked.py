"""Tracked-Delta-E variant on the GB300 (FP64): parity with the oracle's tracked step, and the
C4 column of Table "table:cfl" through the C ABI."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import bench  # noqa: E402
import paper_2306_17263_gb300 as pkg  # noqa: E402


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
@pytest.mark.parametrize("n,steps", [(8, 2), (37, 5)])
def test_tracked_random_fields_match_oracle(closure, n, steps):
    r, Z = 0.5, 1.2
    init = workloads.random_fields(n, seed=1200 + n)
    o = oracle.Oracle2D(n, r, Z=Z, closure=closure)
    ez, hx, hy = (a.copy() for a in init)
    de = o.laplacian(oracle.F_EZ, ez)  # the library's reading for data set through ms_set_fields
    for _ in range(steps):
        o.step_tracked(ez, hx, hy, de)
    with pkg.Grid(n, r, z=Z, closure=closure, scheme=pkg.SCHEME_C4_DE) as g:
        g.set_fields(*init)
        g.run(steps)
        got = g.get_fields()
    cat = lambda fs: np.concatenate([np.ravel(a) for a in fs])
    ref = cat((ez, hx, hy))
    assert np.linalg.norm(cat(got) - ref) <= 1e-12 * np.linalg.norm(ref)


def test_tracked_modes_match_oracle():
    n, r, steps = 48, 0.5, 30
    modes = workloads.random_modes(3, 10, seed=4)
    o = oracle.Oracle2D(n, r)
    ez, hx, hy = o.init_modes(modes)
    de = np.zeros_like(ez)
    for m, q, a in modes:
        de += -(math.pi ** 2) * (m * m + q * q) * o.exact([(m, q, a)], 0.0, 0.0)[0]
    for _ in range(steps):
        o.step_tracked(ez, hx, hy, de)
    with pkg.Grid(n, r, scheme=pkg.SCHEME_C4_DE) as g:
        g.init_modes(modes)
        g.run(steps)
        got = g.get_fields()
    for a, b in zip(got, (ez, hx, hy)):
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())


def test_table_cfl_c4_column_tracked_gpu():
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_cfl_c4.json")))
    for k in (2, 21):
        for rn, want in zip(g["r_numerators_over_6sqrt2"], g["mae"][str(k)]):
            got, _ = bench.wavenumber_mae(pkg, k, pkg.SCHEME_C4_DE, g["N"], rn / (6 * math.sqrt(2)), g["T"])
            assert abs(got - want) <= 0.03 * want, (k, rn, got, want)
