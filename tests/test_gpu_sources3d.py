"""Current sources on 3D grids (GB300): divergence-free driven modes.

- FP64 against the oracle's source step (oracle/maxwell_oracle3d.c or3d_step_src) on random fields,
  both closures, relative L2 <= 1e-12;
- graph replay equal to single steps bit for bit (the source terms read the step index on the
  device);
- FP32_REFINED against FP64 on the exact driven solution: within 2x the FP64 error and closer to
  FP64 than FP64 is to the driven solution;
- fourth-order convergence to the driven solution through the C ABI (FP64);
- argument checks.
Expected values come only from oracle/ (the oracle's step and its exact driven solution).
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_17263_gb300 as pkg  # noqa: E402

SRC = [(1, 1, 1, 1.0, -1.0, 0.0, 3.0), (1, 2, 1, 2.0, -1.5, 1.0, 7.0), (2, 3, 0, 0.0, 0.0, 0.6, 5.0)]


def _rel(a, b):
    a = np.concatenate([np.ravel(x) for x in a])
    b = np.concatenate([np.ravel(x) for x in b])
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _l2(a, b, h):
    return math.sqrt(sum(float(np.sum((x - y) ** 2)) for x, y in zip(a, b)) * h ** 3)


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
@pytest.mark.parametrize("n", [9, 16])
def test_fp64_matches_oracle(closure, n):
    r, Z, K, n0 = 0.4, 1.3, 4, 3
    init = workloads.random_fields3(n, seed=400 + n)
    o = oracle.Oracle3D(n, r, Z=Z, closure=closure)
    ref = [a.copy() for a in init]
    for k in range(K):
        o.step_src(ref, SRC, n0 + k)
    with pkg.Grid(n, r, z=Z, closure=closure, dim=3) as g:
        g.set_sources3(SRC)
        g.set_fields(*init, step=n0)
        for _ in range(K):
            g.step()
        got = g.get_fields()
    assert _rel(got, ref) <= 1e-12


@pytest.mark.parametrize("prec", [pkg.FP64, pkg.FP32_REFINED])
def test_graph_replay_equals_single_steps(prec):
    n, r, K = 12, 0.4, 19
    init = workloads.random_fields3(n, seed=7)
    out = []
    for mode in ("steps", "run"):
        with pkg.Grid(n, r, precision=prec, dim=3) as g:
            g.set_sources3(SRC)
            g.set_fields(*init)
            if mode == "steps":
                for _ in range(K):
                    g.step()
            else:
                g.run(K)
            out.append(g.get_fields())
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_fp32_within_the_fp64_discretisation_error():
    n, r, T = 32, 0.4, 0.25
    res = {}
    for prec in (pkg.FP64, pkg.FP32_REFINED):
        with pkg.Grid(n, r, z=1.2, precision=prec, dim=3) as g:
            g.set_sources3(SRC)
            g.init_driven3(SRC)
            K = int(round(T / (r / n)))
            g.run(K)
            res[prec] = g.get_fields()
    o = oracle.Oracle3D(n, r, Z=1.2)
    ex = o.exact_driven(SRC, K * o.ht, (K + 0.5) * o.ht)
    e64, e32 = _l2(res[pkg.FP64], ex, o.h), _l2(res[pkg.FP32_REFINED], ex, o.h)
    assert e32 <= 2 * e64, (e32, e64)
    assert _l2(res[pkg.FP32_REFINED], res[pkg.FP64], o.h) <= e64


def test_fourth_order_convergence_through_the_c_abi():
    T, errs = 0.25, []
    for n in (8, 16, 32):
        with pkg.Grid(n, 0.4, z=1.2, dim=3) as g:
            g.set_sources3(SRC)
            g.init_driven3(SRC)
            K = int(round(T / (0.4 / n)))
            g.run(K)
            got = g.get_fields()
        o = oracle.Oracle3D(n, 0.4, Z=1.2)
        errs.append(_l2(got, o.exact_driven(SRC, K * o.ht, (K + 0.5) * o.ht), o.h))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert rates[1] > 3.5, (errs, rates)


def test_argument_checks():
    with pkg.Grid(8, 0.4, dim=3) as g:
        for bad in ([(1, 1, 1, 1.0, 1.0, 0.0, 3.0)],    # a . k != 0
                    [(1, 0, 0, 0.0, 1.0, 0.0, 3.0)],    # one nonzero index
                    [(-1, 1, 1, 1.0, 1.0, 0.0, 3.0)],
                    [(1, 1, 1, float("nan"), -1.0, 0.0, 3.0)]):
            with pytest.raises(pkg.MaxwellError) as e:
                g.set_sources3(bad)
            assert e.value.status == -1
        with pytest.raises(pkg.MaxwellError) as e:  # resonant driving
            g.init_driven3([(1, 1, 0, 0.0, 0.0, 1.0, math.pi * math.sqrt(2.0))])
        assert e.value.status == -1
        g.set_sources3([])
    with pkg.Grid(8, 0.5) as g:
        with pytest.raises(pkg.MaxwellError) as e:
            g.set_sources3(SRC)
        assert e.value.status == -7
