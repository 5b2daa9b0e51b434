"""Pins of the oracle's reverse pass: the transposes against the forward operators
(dot-product identities, which hold exactly in exact arithmetic), the Taylor initialisation
against the exact cavity mode, and the misfit gradient against central differences, which are
exact for the quadratic misfit whatever the step size."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import CLOSURE_PAPER, CLOSURE_REFLECT, F_EZ, F_HX, F_HY, HALF_TO_NODE, NODE_TO_HALF


@pytest.mark.parametrize("closure", [CLOSURE_PAPER, CLOSURE_REFLECT])
@pytest.mark.parametrize("kind", [HALF_TO_NODE, NODE_TO_HALF])
@pytest.mark.parametrize("M", [5, 9, 30])
def test_pade_transpose_dot_product(closure, kind, M):
    rng = np.random.default_rng(M)
    f, g = rng.standard_normal(M + 1), rng.standard_normal(M)
    h = 0.37
    lhs = np.dot(oracle.pade_line(f, h, closure, kind), g)
    rhs = np.dot(f, oracle.pade_line_T(g, h, closure, kind))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def _interior(o, rng):
    ez, hx, hy = workloads.random_fields(o.N, seed=int(rng.integers(1 << 30)))
    return ez, hx, hy


@pytest.mark.parametrize("closure", [CLOSURE_PAPER, CLOSURE_REFLECT])
@pytest.mark.parametrize("N,r,Z", [(12, 0.5, 1.0), (17, 5 / (6 * math.sqrt(2)), 2.0)])
def test_step_transpose_dot_product(closure, N, r, Z):
    """<M u, v> = <u, M^T v> on the unknowns for one full step."""
    o = oracle.Oracle2D(N, r, Z=Z, closure=closure)
    rng = np.random.default_rng(N)
    u, v = _interior(o, rng), _interior(o, rng)
    mu = [a.copy() for a in u]
    o.step(*mu)
    mtv = [a.copy() for a in v]
    o.step_T(*mtv)
    lhs = sum(float(np.sum(a * b)) for a, b in zip(mu, v))
    rhs = sum(float(np.sum(a * b)) for a, b in zip(u, mtv))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs))


@pytest.mark.parametrize("closure", [CLOSURE_PAPER, CLOSURE_REFLECT])
def test_taylor_transpose_dot_product(closure):
    o = oracle.Oracle2D(14, 0.5, Z=1.3, closure=closure)
    rng = np.random.default_rng(3)
    e = _interior(o, rng)[0]
    _, lx, ly = _interior(o, rng)
    hx, hy = o.taylor_h(e)
    lhs = float(np.sum(hx * lx) + np.sum(hy * ly))
    rhs = float(np.sum(e * o.taylor_h_T(lx, ly)))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs))


def test_taylor_init_matches_exact_mode():
    """Sec. 5.1 Eq. "talorh" with H^0 = 0: H^{1/2} from E^0 of an exact mode is the exact
    H(h_tau/2) up to the Taylor remainder and the fourth-order spatial error."""
    for N in (32, 64):
        o = oracle.Oracle2D(N, 0.5)
        m = [(2, 3, 1.0)]
        ez0, _, _ = o.exact(m, 0.0, 0.0)
        hx, hy = o.taylor_h(ez0)
        _, hx_ex, hy_ex = o.exact(m, 0.0, 0.5 * o.ht)
        err = np.linalg.norm(np.concatenate([(hx - hx_ex).ravel(), (hy - hy_ex).ravel()]))
        ref = np.linalg.norm(np.concatenate([hx_ex.ravel(), hy_ex.ravel()]))
        assert err / ref < 2e-5 * (64 / N) ** 4


@pytest.mark.parametrize("closure", [CLOSURE_PAPER, CLOSURE_REFLECT])
def test_misfit_gradient_matches_central_differences(closure):
    N, r, K = 16, 0.5, 12
    o = oracle.Oracle2D(N, r, closure=closure)
    rng = np.random.default_rng(11)
    e0 = _interior(o, rng)[0]
    target = o.exact([(1, 2, 0.7), (3, 1, -0.4)], K * o.ht, K * o.ht)[0]
    L, g = o.misfit_grad(e0, target, K)
    assert np.all(g[0, :] == 0) and np.all(g[:, 0] == 0)
    for k in range(3):
        d = _interior(o, rng)[0]
        eps = 0.5  # central differences are exact for the quadratic misfit
        lp = o.misfit_grad(e0 + eps * d, target, K, grad=False)
        lm = o.misfit_grad(e0 - eps * d, target, K, grad=False)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - float(np.sum(g * d))) <= 1e-9 * (abs(fd) + L)
