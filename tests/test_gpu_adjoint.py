"""Reverse pass on the GB300 (FP64): parity with the oracle's reverse pass element by element,
dot-product identities between the GPU forward step and the GPU reverse step, the Taylor
initialisation, and the misfit gradient through torch.autograd against central differences
(exact for the quadratic misfit) at the full reverse-pass workload size."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_17263_gb300 as pkg  # noqa: E402
from paper_2306_17263_gb300.autograd import propagate_ez  # noqa: E402


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
@pytest.mark.parametrize("n,steps", [(8, 1), (37, 3), (64, 2)])
def test_adjoint_steps_match_oracle(closure, n, steps):
    lam = workloads.random_fields(n, seed=300 + n)
    o = oracle.Oracle2D(n, 0.5, closure=closure)
    ref = [a.copy() for a in lam]
    for _ in range(steps):
        o.step_T(*ref)
    with pkg.Grid(n, 0.5, closure=closure) as g:
        got = g.adjoint_steps(steps, *lam)
    for a, b in zip(got, ref):
        assert _rel(a, b) <= 1e-12


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.FP32_REFINED])
def test_taylor_init_and_transpose_match_oracle(precision):
    n = 40
    e0 = workloads.sine_series_field(n, 0.05, seed=5)
    o = oracle.Oracle2D(n, 0.5)
    hx, hy = o.taylor_h(e0)
    with pkg.Grid(n, 0.5, precision=precision) as g:
        g.taylor_init(e0)
        ez, gx, gy = g.get_fields()
        assert g.step_count == 0
        lx, ly = workloads.random_fields(n, seed=9)[1:]
        t = g.taylor_init_T(lx, ly)
    tol = 1e-12 if precision == pkg.FP64 else 1e-7  # FP32_REFINED stores ~48-bit state
    e_ref = e0.copy()
    e_ref[0, :] = e_ref[-1, :] = e_ref[:, 0] = e_ref[:, -1] = 0
    assert _rel(ez, e_ref) <= tol and _rel(gx, hx) <= tol and _rel(gy, hy) <= tol
    assert _rel(t, o.taylor_h_T(lx, ly)) <= 1e-12


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
def test_misfit_gradient_matches_oracle(closure):
    n, K = 24, 20
    o = oracle.Oracle2D(n, 0.5, closure=closure)
    e0 = workloads.sine_series_field(n, 0.05, seed=2)
    target = o.exact([(1, 2, 0.7), (3, 1, -0.4)], K * o.ht, K * o.ht)[0]
    L, grad = o.misfit_grad(e0, target, K)
    with pkg.Grid(n, 0.5, closure=closure) as g:
        g.taylor_init(e0)
        g.run(K)
        ez = g.get_fields()[0]
        d = ez - target
        d[0, :] = d[-1, :] = d[:, 0] = d[:, -1] = 0
        got = g.adjoint_run(K, g.h ** 2 * d)
    assert abs(0.5 * g.h ** 2 * np.sum(d * d) - L) <= 1e-12 * L
    assert _rel(got, grad) <= 1e-12


def test_gpu_forward_and_reverse_are_transposes():
    """<M^K u, v> = <u, (M^T)^K v> with the GPU forward step and the GPU reverse step."""
    n, K = 96, 19
    u, v = workloads.random_fields(n, seed=41), workloads.random_fields(n, seed=42)
    with pkg.Grid(n, 0.5) as g:
        g.set_fields(*u)
        g.run(K)
        mu = g.get_fields()
        mtv = g.adjoint_steps(K, *v)
    lhs = sum(float(np.sum(a * b)) for a, b in zip(mu, v))
    rhs = sum(float(np.sum(a * b)) for a, b in zip(u, mtv))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def _loss_and_grad(g, ez0, target, K):
    x = torch.tensor(ez0, device="cuda", requires_grad=True)
    t = torch.tensor(target, device="cuda")
    ez = propagate_ez(g, x, K)
    mask = torch.zeros_like(t)
    mask[1:-1, 1:-1] = 1
    L = 0.5 * g.h ** 2 * torch.sum((mask * (ez - t)) ** 2)
    L.backward()
    return float(L.detach()), x.grad.cpu().numpy()


def _loss(g, ez0, target, K):
    g.taylor_init(ez0)
    g.run(K)
    d = g.get_fields()[0] - target
    d[0, :] = d[-1, :] = d[:, 0] = d[:, -1] = 0
    return 0.5 * g.h ** 2 * float(np.sum(d * d))


def test_autograd_gradient_matches_oracle_small():
    n, K = 20, 12
    o = oracle.Oracle2D(n, 0.5)
    e0 = workloads.sine_series_field(n, 0.05, seed=3)
    target = o.exact([(2, 1, 1.0)], K * o.ht, K * o.ht)[0]
    L_ref, g_ref = o.misfit_grad(e0, target, K)
    with pkg.Grid(n, 0.5) as g:
        L, grad = _loss_and_grad(g, e0, target, K)
    assert abs(L - L_ref) <= 1e-12 * L_ref
    assert _rel(grad, g_ref) <= 1e-12


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.FP32_REFINED])
def test_full_size_gradient_central_differences(precision):
    """The reverse-pass workload at full size (1024^2 cells, 2000 steps): the gradient from
    torch.autograd against central differences of the loss on random directions of the same
    law.  The loss is quadratic, so central differences have no truncation error; with the FP64
    forward they agree to rounding, with the FP32_REFINED forward to its stated accuracy
    (relative state error ~1e-6 at this size)."""
    c = workloads.config5()
    n, K = c["n"], c["steps"]
    ndir = 4 if precision == pkg.FP64 else 16
    with pkg.Grid(n, c["r"], precision=precision) as g:
        ez0 = workloads.sine_series_field(n, c["ell"], c["ez0_seed"])
        # target: the exact mode superposition at the final time
        tE = K * g.ht
        modes_t = [(m, q, a * np.cos(np.pi * np.hypot(m, q) * tE)) for m, q, a in c["target_modes"]]
        g.init_modes(modes_t)
        target = g.get_fields()[0]
        L, grad = _loss_and_grad(g, ez0, target, K)
        assert np.all(grad[0, :] == 0) and np.all(grad[:, 0] == 0)
        tol = 1e-9 if precision == pkg.FP64 else 2e-4
        for s in c["direction_seeds"][:ndir]:
            d = workloads.sine_series_field(n, c["ell"], s)
            gd = float(np.sum(grad * d))
            eps = 0.25 * L / max(abs(gd), 1e-300)
            fd = (_loss(g, ez0 + eps * d, target, K) - _loss(g, ez0 - eps * d, target, K)) / (2 * eps)
            assert abs(fd - gd) <= tol * (abs(gd) + L / eps), (s, fd, gd)
