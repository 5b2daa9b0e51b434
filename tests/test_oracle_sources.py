"""Pins of the oracle's step with current sources (2D TM_z, J_z a sum of driven sine modes):
the closed-form affine per-mode recurrence under the REFLECT closure, fourth-order convergence
to the exact driven solution under both closures, and no effect of zero-amplitude sources."""
import math

import numpy as np
import pytest

import oracle
import workloads
from closed_forms import mode_basis, mode_step_forced

SRC = [(2, 3, 1.0, 5.0), (1, 1, -0.5, 11.0)]


@pytest.mark.parametrize("m,n,w,Z", [(2, 3, 5.0, 1.0), (4, 1, 17.0, 1.7)])
def test_reflect_forced_step_is_affine_mode_recurrence(m, n, w, Z):
    N, r, K = 16, 0.5, 9
    o = oracle.Oracle2D(N, r, Z=Z, closure=oracle.CLOSURE_REFLECT)
    eb, xb, yb = mode_basis(N, m, n)
    v = np.random.default_rng(m + n).standard_normal(3)
    f = [v[0] * eb, v[1] * xb, v[2] * yb]
    for s in range(K):
        o.step_src(*f, [(m, n, 0.8, w)], s)
        M, c = mode_step_forced(N, r, m, n, Z, 0.8, w, s)
        v = M @ v + c
    for got, coef, b in zip(f, v, (eb, xb, yb)):
        assert np.abs(got - coef * b).max() <= 1e-12 * max(1.0, np.abs(coef * b).max())


@pytest.mark.parametrize("closure", [oracle.CLOSURE_PAPER, oracle.CLOSURE_REFLECT])
def test_fourth_order_convergence_to_driven_solution(closure):
    T, errs = 0.5, []
    for N in (16, 32, 64):
        o = oracle.Oracle2D(N, 0.5, Z=1.3, closure=closure)
        K = int(round(T / o.ht))
        f = list(o.exact_driven(SRC, 0.0, 0.5 * o.ht))
        for s in range(K):
            o.step_src(*f, SRC, s)
        ex = o.exact_driven(SRC, K * o.ht, (K + 0.5) * o.ht)
        errs.append(math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(f, ex))) / N)
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 3.7, (errs, rates)


def test_zero_sources_equal_plain_step():
    o = oracle.Oracle2D(12, 0.5)
    a = list(workloads.random_fields(12, seed=5))
    b = [x.copy() for x in a]
    for s in range(3):
        o.step(*a)
        o.step_src(*b, [(1, 2, 0.0, 3.0)], s)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
