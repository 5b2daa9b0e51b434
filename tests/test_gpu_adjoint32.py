"""The FP32 reverse pass of FP32_REFINED grids (GB300): float-float adjoint state, the transpose of
the FP32_REFINED forward operator computed in FP32 with the transposed Pade band accumulated in
float-float before its difference (Sec. 3.4 transposed, App. A.1).

- reverse steps against the oracle's reverse step on random adjoint fields, both closures
  (FP32 noise, relative L2 <= 2e-6 after 20 steps, as for the forward on random fields);
- the misfit gradient (Taylor-initialised run, Sec. 5.1) against the oracle's, relative <= 1e-5;
- <M^K u, v> = <u, (M^T)^K v> with the FP32_REFINED forward and the FP32 reverse pass;
- the FP64 reverse pass stays selectable on FP32_REFINED grids and matches the oracle to 1e-12.
Expected values come only from oracle/ (or from the FP32 forward for the dot-product identity).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_17263_gb300 as pkg  # noqa: E402


def _rel(a, b):
    a = np.concatenate([np.ravel(x) for x in a]) if isinstance(a, (list, tuple)) else np.ravel(a)
    b = np.concatenate([np.ravel(x) for x in b]) if isinstance(b, (list, tuple)) else np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
@pytest.mark.parametrize("n", [37, 64, 129])
def test_fp32_reverse_steps_match_oracle(closure, n):
    steps = 20
    lam = workloads.random_fields(n, seed=500 + n)
    o = oracle.Oracle2D(n, 0.5, closure=closure)
    ref = [a.copy() for a in lam]
    for _ in range(steps):
        o.step_T(*ref)
    with pkg.Grid(n, 0.5, closure=closure, precision=pkg.FP32_REFINED) as g:
        got = g.adjoint_steps(steps, *lam)
    assert _rel(got, ref) <= 2e-6


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
@pytest.mark.parametrize("n", [37, 64])
def test_fp32_misfit_gradient_matches_oracle(closure, n):
    K = 40
    o = oracle.Oracle2D(n, 0.5, closure=closure)
    e0 = workloads.sine_series_field(n, 0.05, seed=3)
    target = o.exact([(1, 2, 0.7), (3, 1, -0.4)], K * o.ht, K * o.ht)[0]
    L, grad = o.misfit_grad(e0, target, K)
    with pkg.Grid(n, 0.5, closure=closure, precision=pkg.FP32_REFINED) as g:
        g.taylor_init(e0)
        g.run(K)
        d = g.get_fields()[0] - target
        d[0, :] = d[-1, :] = d[:, 0] = d[:, -1] = 0
        got = g.adjoint_run(K, g.h ** 2 * d)
    assert _rel(got, grad) <= 1e-5


def test_fp32_forward_and_reverse_are_transposes():
    n, K = 96, 19
    u, v = workloads.random_fields(n, seed=61), workloads.random_fields(n, seed=62)
    with pkg.Grid(n, 0.5, precision=pkg.FP32_REFINED) as g:
        g.set_fields(*u)
        g.run(K)
        mu = g.get_fields()
        mtv = g.adjoint_steps(K, *v)
    lhs = sum(float(np.sum(a * b)) for a, b in zip(mu, v))
    rhs = sum(float(np.sum(a * b)) for a, b in zip(u, mtv))
    scale = np.linalg.norm(np.concatenate([np.ravel(a) for a in mu])) * np.linalg.norm(
        np.concatenate([np.ravel(a) for a in v]))
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_fp64_reverse_selectable_on_fp32_grids():
    n, steps = 37, 3
    lam = workloads.random_fields(n, seed=7)
    o = oracle.Oracle2D(n, 0.5)
    ref = [a.copy() for a in lam]
    for _ in range(steps):
        o.step_T(*ref)
    with pkg.Grid(n, 0.5, precision=pkg.FP32_REFINED) as g:
        g.set_adjoint_precision(pkg.FP64)
        got = g.adjoint_steps(steps, *lam)
    assert _rel(got, ref) <= 1e-12
    with pkg.Grid(n, 0.5) as g:
        with pytest.raises(pkg.MaxwellError) as e:
            g.set_adjoint_precision(pkg.FP32_REFINED)
        assert e.value.status == -7
        with pytest.raises(pkg.MaxwellError) as e:
            g.set_adjoint_precision(4)
        assert e.value.status == -1
