"""Error against wavenumber (the experiment of Fig. "fig:error(k)", h = 1/64, k_x = k_y = k,
T = 4/sqrt(2)): the mean absolute error of Sec. 5.1 measured on the GPU through the C ABI equals
the oracle's for the compact scheme and for the plain Yee scheme."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import bench  # noqa: E402
import paper_2306_17263_gb300 as pkg  # noqa: E402

N, R, T = 64, 0.5, 4.0 / math.sqrt(2.0)


def _oracle_mae(k, yee):
    o = oracle.Oracle2D(N, R)
    modes = [(k, k, 1.0)]
    K = int(round(T / o.ht))
    f = list(o.init_modes(modes))
    if not yee:
        return o.run(*f, K, modes=modes), K
    acc = 0.0
    for n in range(1, K + 1):
        o.yee_step(*f)
        acc += o.error(modes, n, *f)[3]
    return acc / (3.0 * K * N * N), K


@pytest.mark.parametrize("k", [2, 16, 40])
@pytest.mark.parametrize("yee", [False, True])
def test_mae_matches_oracle(k, yee):
    got, K = bench.wavenumber_mae(pkg, k, pkg.SCHEME_YEE2 if yee else pkg.SCHEME_C4, N, R, T)
    ref, K2 = _oracle_mae(k, yee)
    assert K == K2 == 362
    assert abs(got - ref) <= 1e-9 * ref


def test_compact_scheme_wins_at_high_ppw():
    """At 64 points per wavelength the fourth-order scheme's error is orders of magnitude below
    Yee's; at 2.56 points per wavelength both are of order one (pollution)."""
    c4, _ = bench.wavenumber_mae(pkg, 2, pkg.SCHEME_C4, N, R, T)
    yee, _ = bench.wavenumber_mae(pkg, 2, pkg.SCHEME_YEE2, N, R, T)
    assert c4 < 1e-3 * yee
    c4_50, _ = bench.wavenumber_mae(pkg, 50, pkg.SCHEME_C4, N, R, T)
    assert c4_50 > 1e3 * c4
