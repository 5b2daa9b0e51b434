"""Pins of the 3D oracle's current sources (divergence-free driven modes, Sec. 3.1 and Sec. 3.4
with J != 0), each against something other than the 3D source code itself:
  - a source independent of one coordinate on fields independent of it is the 2D TM_z source
    step of the 2D oracle (itself pinned by tests/test_oracle_sources.py), all three orientations,
    both closures;
  - zero amplitudes give the plain step exactly;
  - the step converges at fourth order to the exact driven solution of a genuinely 3D current.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import CLOSURE_PAPER, CLOSURE_REFLECT
from test_oracle3d_pins import _extrude


@pytest.mark.parametrize("closure", [CLOSURE_PAPER, CLOSURE_REFLECT])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sources_reduce_to_2d(closure, axis):
    N, r, Z, K = 9, 0.4, 1.3, 3
    src2 = [(2, 3, 0.7, 5.0), (1, 1, -0.4, 11.0)]
    src3 = []
    for (m, n, a, w) in src2:
        k, amp = [0, 0, 0], [0.0, 0.0, 0.0]
        k[(axis + 1) % 3], k[(axis + 2) % 3] = m, n
        amp[axis] = a
        src3.append((*k, *amp, w))
    o2 = oracle.Oracle2D(N, r, Z=Z, closure=closure)
    o3 = oracle.Oracle3D(N, r, Z=Z, closure=closure)
    s2 = list(workloads.random_fields(N, seed=90 + axis))
    f, _ = _extrude(s2, N, axis)
    for n in range(K):
        o3.step_src(f, src3, n)
        o2.step_src(*s2, src2, n)
    ref, _ = _extrude(s2, N, axis)
    for c in range(6):
        scale = max(1.0, np.abs(ref[c]).max())
        assert np.abs(f[c] - ref[c]).max() <= 1e-12 * scale, c


def test_zero_sources_are_the_plain_step():
    N, r = 7, 0.4
    o = oracle.Oracle3D(N, r)
    f0 = workloads.random_fields3(N, seed=5)
    a = [x.copy() for x in f0]
    b = [x.copy() for x in f0]
    o.step_src(a, [(1, 2, 1, 0.0, 0.0, 0.0, 3.0)], 4)
    o.step(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_fourth_order_convergence_to_the_driven_solution():
    """J = (a_x cos sin sin, a_y sin cos sin, a_z sin sin cos) sin(w t) with (1, 1, 1) . a = 0 and
    (1, 2, 1) . a = 0 (both off resonance); start on the driven solution, run to T."""
    src = [(1, 1, 1, 1.0, -1.0, 0.0, 3.0), (1, 2, 1, 2.0, -1.5, 1.0, 7.0)]
    T, errs = 0.25, []
    for N in (8, 16, 32):
        o = oracle.Oracle3D(N, 0.4, Z=1.2)
        K = int(round(T / o.ht))
        f = o.exact_driven(src, 0.0, 0.5 * o.ht)
        for n in range(K):
            o.step_src(f, src, n)
        ex = o.exact_driven(src, K * o.ht, (K + 0.5) * o.ht)
        errs.append(math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(f, ex)) * o.h ** 3))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert rates[1] > 3.5, (errs, rates)
    # the source terms matter: without them the same run leaves the driven solution at first order
    o = oracle.Oracle3D(16, 0.4, Z=1.2)
    K = int(round(T / o.ht))
    f = o.exact_driven(src, 0.0, 0.5 * o.ht)
    o.run(f, K)
    ex = o.exact_driven(src, K * o.ht, (K + 0.5) * o.ht)
    e_plain = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(f, ex)) * o.h ** 3)
    assert e_plain > 100 * errs[1]
