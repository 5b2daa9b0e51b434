"""NC comparator on the GB300 (FP64): parity with the oracle's NC step, and its mean absolute
error on the setting of Table "table:cfl" (the oracle's value, within 1e-9)."""
import math

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


@pytest.mark.parametrize("n,steps", [(4, 3), (37, 9), (64, 40)])
def test_nc_random_fields_match_oracle(n, steps):
    r, Z = 0.5, 1.4
    init = workloads.random_fields(n, seed=900 + n)
    o = oracle.Oracle2D(n, r, Z=Z)
    ref = [a.copy() for a in init]
    for _ in range(steps):
        o.nc_step(*ref)
    with pkg.Grid(n, r, z=Z, scheme=pkg.SCHEME_NC4) as g:
        g.set_fields(*init)
        g.run(steps)
        got = g.get_fields()
    cat = lambda fs: np.concatenate([np.ravel(a) for a in fs])
    assert np.linalg.norm(cat(got) - cat(ref)) <= 1e-12 * np.linalg.norm(cat(ref))


def test_nc_mae_table_cfl_setting():
    T, r = 4.0 / math.sqrt(2.0), 5 / (6 * math.sqrt(2))
    got, K = bench.wavenumber_mae(pkg, 2, pkg.SCHEME_NC4, 64, r, T)
    o = oracle.Oracle2D(64, r)
    modes = [(2, 2, 1.0)]
    f = list(o.init_modes(modes))
    acc = 0.0
    for n in range(1, K + 1):
        o.nc_step(*f)
        acc += o.error(modes, n, *f)[3]
    ref = acc / (3.0 * K * 64 * 64)
    assert abs(got - ref) <= 1e-9 * ref
    assert abs(got - 7.38e-4) <= 0.05 * 7.38e-4  # Table "table:cfl", NC column, r = 5/(6 sqrt 2)
