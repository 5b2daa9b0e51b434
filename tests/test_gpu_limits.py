"""Edge cases of size and content on the GB300: the largest grids the library accepts (2D n = 32768,
about 90 GB on the device, and 3D n = 512), where the 32-bit in-plane offsets of the kernels come
closest to their limits, checked against the exact cavity modes; and the degenerate inputs (no
steps, no modes, a zero state)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_17263_gb300 as pkg  # noqa: E402


def test_largest_2d_grid_fp32_refined_matches_exact_modes():
    """n = 32768 (32769^2 = 1.07e9 points per E_z plane, the largest the C ABI takes): after a few
    steps the state agrees with the exact modes to FP32 rounding (the discretisation error of these
    low modes is far below it at h = 1/32768), so no offset has wrapped anywhere in the grid."""
    n, r = 32768, 0.5
    modes = [(1, 1, 1.0), (3, 2, 0.5), (40, 17, 0.25)]
    with pkg.Grid(n, r, precision=pkg.FP32_REFINED) as g:
        g.init_modes(modes)
        g.run(4)
        l2_abs, l2_rel, max_abs, _ = g.error_vs_exact(modes)
    assert np.isfinite(l2_rel) and l2_rel <= 1e-6, (l2_abs, l2_rel, max_abs)
    assert max_abs <= 1e-5, max_abs


def test_largest_3d_grid_fp32_refined_matches_exact_modes():
    """n = 512 (513^3 = 1.35e8 points per node component, the 3D limit)."""
    n, r = 512, 0.4
    modes = [workloads.mode3(2, 3, 1, 1.0), workloads.mode3(5, 1, 4, 0.5)]
    with pkg.Grid(n, r, precision=pkg.FP32_REFINED, dim=3) as g:
        g.init_modes(modes)
        g.run(3)
        l2_abs, l2_rel, max_abs, _ = g.error_vs_exact(modes)
    assert np.isfinite(l2_rel) and l2_rel <= 1e-6, (l2_abs, l2_rel, max_abs)


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.FP32_REFINED])
def test_degenerate_inputs(precision):
    """No steps leave the state and the step counter as they are; no modes give the zero state;
    the zero state stays zero."""
    n = 33
    init = workloads.random_fields(n, seed=12)
    with pkg.Grid(n, 0.5, precision=precision) as g:
        g.set_fields(*init, step=7)
        before = g.get_fields()
        g.run(0)
        after = g.get_fields()
        assert g.step_count == 7
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        g.init_modes([])
        assert g.step_count == 0
        g.run(5)
        for a in g.get_fields():
            assert not np.any(a)
