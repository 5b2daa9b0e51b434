"""Current sources on the GB300: FP64 parity with the oracle's forced step, the FP32_REFINED path
within the discretisation error of the exact driven solution, fourth-order convergence through
the C ABI, and graph replay (ms_run) equal to single steps (the source time is read on the
device)."""
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

SRC = [(2, 3, 1.0, 5.0), (1, 1, -0.5, 11.0)]


def _cat(fs):
    return np.concatenate([np.ravel(a) for a in fs])


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
@pytest.mark.parametrize("n,steps", [(12, 3), (37, 20)])
def test_fp64_sources_match_oracle(closure, n, steps):
    r, Z = 0.5, 1.3
    init = workloads.random_fields(n, seed=1300 + n)
    o = oracle.Oracle2D(n, r, Z=Z, closure=closure)
    ref = [a.copy() for a in init]
    for s in range(5, 5 + steps):
        o.step_src(*ref, SRC, s)
    with pkg.Grid(n, r, z=Z, closure=closure) as g:
        g.set_sources(SRC)
        g.set_fields(*init, step=5)
        g.run(steps)
        got = g.get_fields()
    assert np.linalg.norm(_cat(got) - _cat(ref)) <= 1e-12 * np.linalg.norm(_cat(ref))


def test_graph_replay_equals_single_steps():
    n, steps = 40, 37
    outs = []
    for mode in ("step", "run"):
        with pkg.Grid(n, 0.5, precision=pkg.FP32_REFINED) as g:
            g.set_sources(SRC)
            g.init_driven(SRC)
            if mode == "step":
                for _ in range(steps):
                    g.step()
            else:
                g.run(steps)
            outs.append(g.get_fields())
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_convergence_and_fp32_within_discretisation_error():
    T, errs = 0.5, []
    for n in (32, 64, 128):
        res = {}
        for prec in (pkg.FP64, pkg.FP32_REFINED):
            with pkg.Grid(n, 0.5, z=1.3, precision=prec) as g:
                g.set_sources(SRC)
                g.init_driven(SRC)
                g.run(int(round(T / g.ht)))
                res[prec] = (g.get_fields(), g.error_vs_driven(SRC)[0])
        (f64, e64), (f32, e32) = res[pkg.FP64], res[pkg.FP32_REFINED]
        errs.append(e64)
        assert e32 <= 2 * e64
        assert np.linalg.norm(_cat(f32) - _cat(f64)) / n <= e64
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 3.7, (errs, rates)
