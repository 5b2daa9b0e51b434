"""ms_p1_solve_static: the P1 solve for callers that cannot allocate device memory.

Such callers (a latency-critical loop where cudaMalloc may synchronise the device, or a host
application that owns all device memory through its own pool) call this entry point with their
own input and output arrays; its scratch is a fixed __device__ array inside the library.  The
test calls it through the C ABI and checks it against the grid's regular solve (ms_apply_op,
MS_OP_P1SOLVE_*), within the FP64 tolerance of the other parity tests, on two calls in a row
(the second call runs on the scratch array left behind by the first).  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_17263_gb300 as pkg  # noqa: E402

NAMES = ("ez", "hx", "hy")


def _entry():
    L = pkg.load()
    f = L.ms_p1_solve_static
    f.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L, f


@pytest.mark.parametrize("n,r", [(37, 0.5), (512, 5 / (6 * 2 ** 0.5))])
def test_static_solve_matches_grid_solve(n, r):
    L, solve_static = _entry()
    fields = workloads.random_fields(n, seed=100 + n)
    with pkg.Grid(n, r) as g:
        for field, (arr, name) in enumerate(zip(fields, NAMES)):
            for call in range(2):
                b = torch.from_numpy(np.ascontiguousarray(arr * (1.0 + 0.5 * call))).cuda()
                ref = torch.zeros_like(b)
                g.apply_op(f"p1solve_{name}", [b], [ref])
                g.sync()
                out = torch.full_like(b, float("nan"))
                status = solve_static(n, r, field, b.data_ptr(), out.data_ptr(), None)
                assert status == 0, L.ms_last_error().decode()
                torch.cuda.synchronize()
                got, want = out.cpu().numpy(), ref.cpu().numpy()
                assert np.all(np.isfinite(got))
                assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), (name, call)


def test_static_solve_rejects_sizes_beyond_the_maximum():
    L, solve_static = _entry()
    n = 513  # MS_STATIC_MAX_N + 1
    b = torch.zeros((n + 1, n + 1), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    assert solve_static(n, 0.5, 0, b.data_ptr(), x.data_ptr(), None) == -1
    assert "MS_STATIC_MAX_N" in L.ms_last_error().decode()
    assert solve_static(64, 0.5, 3, b.data_ptr(), x.data_ptr(), None) == -1
    assert solve_static(64, 0.5, 0, b.data_ptr(), b.data_ptr(), None) == -1
