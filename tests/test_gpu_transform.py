"""The tensor-core transform solver of P1 on 3D FP32_REFINED grids (GB300 only).

- The transforms alone (sine / cosine GEMMs in bf16 hi + lo, three products) against the oracle's
  CG solve of P1 x = b (Def. "def:operatorsP"), on every component: relative error <= 5e-5, the
  accuracy the refinement sweep count is derived from (measured about 1e-5).
- Whole steps with the transform solver against the Richardson solver and against the oracle on
  random fields (FP32 noise, relative L2 <= 2e-6), and the mixed-path criterion on cavity modes.
Inputs come from workloads.py (seeded); expected values only from oracle/ or the Richardson path.
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
    a = np.concatenate([np.ravel(x) for x in a])
    b = np.concatenate([np.ravel(x) for x in b])
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n", [16, 23, 40])
def test_transform_solve_matches_oracle_cg(n):
    r = 0.4
    o = oracle.Oracle3D(n, r)
    o.set_cg(1e-15, 400)
    fields = workloads.random_fields3(n, seed=100 + n)
    h2 = (1.0 / n) ** 2
    with pkg.Grid(n, r, precision=pkg.FP32_REFINED, dim=3) as g:
        for c in range(6):
            b = fields[c].astype(np.float32)
            b_dev = torch.from_numpy(np.ascontiguousarray(b)).cuda()
            x_dev = torch.full_like(b_dev, 7.0)  # wall points must come back as zero
            g.transform_solve(c, b_dev, x_dev)
            g.sync()
            x = x_dev.cpu().numpy().astype(np.float64)
            # the GPU solves (6 h^2 P1) x = b
            x_ref, _ = o.p1_solve(c, b.astype(np.float64) / (6.0 * h2))
            err = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
            print(f"n={n} comp={c} transform-solve relative error {err:.3e}")
            assert err <= 5e-5, (c, err)
            wall = x_ref == 0.0
            assert np.all(x[wall] == 0.0)


def test_transform_steps_match_richardson_and_oracle():
    n, r, steps = 24, 0.4, 6
    init = workloads.random_fields3(n, seed=31)
    o = oracle.Oracle3D(n, r)
    ref = [a.copy() for a in init]
    o.run(ref, steps)
    out = {}
    for solver in (pkg.SOLVER_RICHARDSON, pkg.SOLVER_TRANSFORM_TC):
        with pkg.Grid(n, r, precision=pkg.FP32_REFINED, dim=3) as g:
            g.set_solver(solver)
            g.set_fields(*init)
            g.run(steps)
            g.sync()
            out[solver] = g.get_fields()
    ts, rich = out[pkg.SOLVER_TRANSFORM_TC], out[pkg.SOLVER_RICHARDSON]
    assert _rel(ts, ref) <= 2e-6
    assert _rel(ts, rich) <= 2e-6


def test_transform_mixed_criterion_on_modes():
    """Cavity modes (3D mode of Maxwell's equations, as in the 3D parity tests): the transform-solver
    step within 2x the FP64 path's error against the exact modes and closer to FP64 than FP64 is
    to the exact modes."""
    n, r, steps = 48, 0.4, 60
    modes = [workloads.mode3(2, 3, 1, 1.0), workloads.mode3(3, 1, 4, -0.7)]
    out = {}
    for prec, solver in ((pkg.FP64, None), (pkg.FP32_REFINED, pkg.SOLVER_TRANSFORM_TC)):
        with pkg.Grid(n, r, precision=prec, dim=3) as g:
            if solver is not None:
                g.set_solver(solver)
            g.init_modes(modes)
            g.run(steps)
            g.sync()
            out[prec] = (g.get_fields(), g.error_vs_exact(modes)[0])
    (f64, e64), (f32, e32) = out[pkg.FP64], out[pkg.FP32_REFINED]
    diff = np.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(f32, f64)) / n ** 3)
    assert e32 <= 2 * e64, (e32, e64)
    assert diff <= e64, (diff, e64)


def test_solver_selection_checks():
    with pkg.Grid(12, 0.5) as g:  # 2D
        with pytest.raises(pkg.MaxwellError) as e:
            g.set_solver(pkg.SOLVER_TRANSFORM_TC)
        assert e.value.status == -7
        g.set_solver(pkg.SOLVER_RICHARDSON)
    with pkg.Grid(8, 0.4, dim=3) as g:  # 3D FP64
        with pytest.raises(pkg.MaxwellError) as e:
            g.set_solver(pkg.SOLVER_TRANSFORM_TC)
        assert e.value.status == -7
    with pkg.Grid(8, 0.4, precision=pkg.FP32_REFINED, dim=3) as g:
        with pytest.raises(pkg.MaxwellError) as e:
            g.set_solver(5)
        assert e.value.status == -1
        g.set_solver(pkg.SOLVER_TRANSFORM_TC)
        g.set_solver(pkg.SOLVER_RICHARDSON)
