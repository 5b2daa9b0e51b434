"""Failure paths of allocation: every device allocation of a grid, a batch and the lazily built
reverse-pass planes is made to fail in turn (host-side injection through ms_debug_fail_alloc; the
device is never actually out of memory).  Each failure must come back as MS_ENOMEM with a message,
release everything the failed call had allocated, and leave the library usable."""
import numpy as np
import pytest

import paper_2306_17263_gb300 as pkg

pytestmark = pytest.mark.gpu

MS_ENOMEM = -3


def _make(kind):
    if kind == "fp64_2d":
        return pkg.Grid(24, 0.5, precision=pkg.FP64)
    if kind == "fp32_2d":
        return pkg.Grid(40, 0.5, precision=pkg.FP32_REFINED)
    if kind == "de_2d":
        return pkg.Grid(24, 0.4, precision=pkg.FP64, scheme=pkg.SCHEME_C4_DE)
    if kind == "de32_2d":
        return pkg.Grid(40, 0.4, precision=pkg.FP32_REFINED, scheme=pkg.SCHEME_C4_DE)
    if kind == "fp64_3d":
        return pkg.Grid(8, 0.4, precision=pkg.FP64, dim=3)
    if kind == "fp32_3d":
        return pkg.Grid(12, 0.4, precision=pkg.FP32_REFINED, dim=3)
    if kind == "batch":
        return pkg.Batch([16, 24, 40], 0.5)
    raise ValueError(kind)


def _allocs_of(fn):
    base = pkg.debug_live_allocs()
    obj = fn()
    n = pkg.debug_live_allocs() - base
    return obj, n, base


@pytest.mark.parametrize("kind", ["fp64_2d", "fp32_2d", "de_2d", "de32_2d", "fp64_3d", "fp32_3d", "batch"])
def test_every_creation_allocation_failure_is_reported_and_released(kind):
    obj, n, base = _allocs_of(lambda: _make(kind))
    obj.close()
    assert n > 0
    assert pkg.debug_live_allocs() == base
    try:
        for k in range(1, n + 1):
            pkg.debug_fail_alloc(k)
            with pytest.raises(pkg.MaxwellError) as e:
                _make(kind)
            assert e.value.status == MS_ENOMEM, (k, str(e.value))
            assert "alloc" in str(e.value).lower() or "memory" in str(e.value).lower(), str(e.value)
            assert pkg.debug_live_allocs() == base, (kind, k)
    finally:
        pkg.debug_fail_alloc(0)
    # the library still works: a fresh object of the same kind is created and steps
    obj = _make(kind)
    obj.run(2)
    obj.close()
    assert pkg.debug_live_allocs() == base


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.FP32_REFINED])
def test_reverse_pass_allocation_failure_leaves_the_grid_usable(precision):
    """The reverse pass allocates its tables and adjoint planes on first use; a failure at any of
    those allocations is MS_ENOMEM and leaks nothing (a part whose set-up completed is kept for
    the next call), and the next call (nothing armed) gives the same gradient as a fresh grid."""
    n = 32
    rng = np.random.default_rng(5)
    lt = rng.standard_normal((n + 1, n + 1))
    lt[0, :] = lt[-1, :] = lt[:, 0] = lt[:, -1] = 0.0
    ref = pkg.Grid(n, 0.5, precision=precision)
    base = pkg.debug_live_allocs()
    want = ref.adjoint_run(4, lt)
    n_alloc = pkg.debug_live_allocs() - base
    ref.close()
    assert n_alloc > 0
    start = pkg.debug_live_allocs()
    for k in range(1, n_alloc + 1):
        g = pkg.Grid(n, 0.5, precision=precision)
        before = pkg.debug_live_allocs()
        try:
            pkg.debug_fail_alloc(k)
            with pytest.raises(pkg.MaxwellError) as e:
                g.adjoint_run(4, lt)
            assert e.value.status == MS_ENOMEM, (k, str(e.value))
            assert pkg.debug_live_allocs() - before < n_alloc, k
        finally:
            pkg.debug_fail_alloc(0)
        got = g.adjoint_run(4, lt)
        assert pkg.debug_live_allocs() - before == n_alloc, k
        g.close()
        assert pkg.debug_live_allocs() == start, k
        assert np.array_equal(np.asarray(got), np.asarray(want)), k
