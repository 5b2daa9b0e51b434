"""Three-dimensional scheme on the GB300 against the 3D oracle (six components).

FP64: relative L2 <= 1e-12 after several steps, on random fields (ragged sizes, both closures)
and on exact modes.  FP32_REFINED: the acceptance criterion of the mixed path (within 2x the
oracle's error against the exact modes and closer to the oracle than the oracle is to them).
At the full size of the 3D workload (256^3 cells, 500 steps) with the REFLECT closure, the
discrete solution is the closed-form per-mode recurrence, checked on sampled lines."""
import numpy as np
import pytest

import oracle
import workloads
from closed_forms import mode_basis3, mode_step_matrix3

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_17263_gb300 as pkg  # noqa: E402


def _cat(fs):
    return np.concatenate([np.ravel(a) for a in fs])


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
@pytest.mark.parametrize("n,steps", [(8, 2), (13, 3), (20, 2)])
def test_fp64_random_fields_match_oracle(closure, n, steps):
    r, Z = 0.4, 1.3
    init = workloads.random_fields3(n, seed=500 + n)
    o = oracle.Oracle3D(n, r, Z=Z, closure=closure)
    ref = [a.copy() for a in init]
    o.run(ref, steps)
    with pkg.Grid(n, r, z=Z, closure=closure, dim=3) as g:
        g.set_fields(*init)
        g.run(steps)
        got = g.get_fields()
        assert g.step_count == steps
    rel = np.linalg.norm(_cat(got) - _cat(ref)) / np.linalg.norm(_cat(ref))
    assert rel <= 1e-12, rel


def test_fp64_modes_match_oracle_and_error():
    n, r, steps = 16, 0.4, 12
    modes = [workloads.mode3(2, 3, 1, 1.0), workloads.mode3(1, 2, 3, -0.6)]
    o = oracle.Oracle3D(n, r)
    ref = o.init_modes(modes)
    with pkg.Grid(n, r, dim=3) as g:
        g.init_modes(modes)
        got0 = g.get_fields()
        for a, b in zip(got0, ref):
            assert np.abs(a - b).max() <= 1e-14
        g.run(steps)
        got = g.get_fields()
        err = g.error_vs_exact(modes)
    o.run(ref, steps)
    rel = np.linalg.norm(_cat(got) - _cat(ref)) / np.linalg.norm(_cat(ref))
    assert rel <= 1e-12, rel
    oe = o.error(modes, steps, ref)
    assert abs(err[0] - oe[0]) <= 1e-12 and abs(err[2] - oe[2]) <= 1e-12


def test_fp32_refined_modes_within_discretisation_error():
    n, r, steps = 24, 0.4, 30
    modes = [workloads.mode3(2, 3, 1, 1.0), workloads.mode3(3, 1, 2, 0.7)]
    o = oracle.Oracle3D(n, r)
    ref = o.init_modes(modes)
    o.run(ref, steps)
    ex = o.exact(modes, steps * o.ht, (steps + 0.5) * o.ht)
    with pkg.Grid(n, r, precision=pkg.FP32_REFINED, dim=3) as g:
        g.init_modes(modes)
        g.run(steps)
        got = g.get_fields()
    err_o = np.linalg.norm(_cat(ref) - _cat(ex))
    assert np.linalg.norm(_cat(got) - _cat(ex)) <= 2 * err_o
    assert np.linalg.norm(_cat(got) - _cat(ref)) <= err_o


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
def test_fp32_refined_random_fields_close_to_oracle(closure):
    n, r, steps = 12, 0.4, 6
    init = workloads.random_fields3(n, seed=77)
    o = oracle.Oracle3D(n, r, closure=closure)
    ref = [a.copy() for a in init]
    o.run(ref, steps)
    with pkg.Grid(n, r, precision=pkg.FP32_REFINED, closure=closure, dim=3) as g:
        g.set_fields(*init)
        g.run(steps)
        got = g.get_fields()
    rel = np.linalg.norm(_cat(got) - _cat(ref)) / np.linalg.norm(_cat(ref))
    assert rel <= 2e-6, rel


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
@pytest.mark.parametrize("n,steps", [(5, 4), (40, 3), (71, 2)])
def test_fp32_refined_random_fields_ragged_sizes(closure, n, steps):
    """The smallest FP32 grid (n = 5: every Pade row explicit, sweep tiles of two or three
    unknowns) and grids of several filter, term and sweep tiles with ragged tails (40, 71): random
    fields within 2e-6 of the oracle."""
    r = 0.4
    init = workloads.random_fields3(n, seed=300 + n)
    o = oracle.Oracle3D(n, r, closure=closure)
    ref = [a.copy() for a in init]
    o.run(ref, steps)
    with pkg.Grid(n, r, precision=pkg.FP32_REFINED, closure=closure, dim=3) as g:
        g.set_fields(*init)
        g.run(steps)
        got = g.get_fields()
    rel = np.linalg.norm(_cat(got) - _cat(ref)) / np.linalg.norm(_cat(ref))
    assert rel <= 2e-6, rel


@pytest.mark.parametrize("precision,steps", [(pkg.FP32_REFINED, 500), (pkg.FP64, 40)])
def test_full_size_reflect_closed_form(precision, steps):
    """256^3 cells: under the REFLECT closure each mode evolves by its 6x6 step matrix; sampled
    lines of every component against the closed form."""
    c = workloads.config3()
    n, r = c["n"], c["r"]
    modes = c["modes"]
    with pkg.Grid(n, r, precision=precision, closure=pkg.CLOSURE_REFLECT, dim=3) as g:
        g.init_modes(modes)
        init = g.get_fields()
        g.run(steps)
        got = g.get_fields()
    # coefficients of each mode in the initial state, then the closed-form evolution
    want = [np.zeros_like(a) for a in got]
    for (m, q, p, ax, ay, az) in modes:
        basis = mode_basis3(n, m, q, p)
        coef = np.array([np.sum(init[k] * basis[k]) / np.sum(basis[k] ** 2) for k in range(6)])
        coef = np.linalg.matrix_power(mode_step_matrix3(n, r, m, q, p), steps) @ coef
        for k in range(6):
            want[k] += coef[k] * basis[k]
    rng = np.random.default_rng(3)
    worst = 0.0
    for k in range(6):
        nz, ny, nx = got[k].shape
        for _ in range(8):
            z, y = int(rng.integers(0, nz)), int(rng.integers(0, ny))
            worst = max(worst, float(np.abs(got[k][z, y] - want[k][z, y]).max()))
    scale = max(float(np.abs(w).max()) for w in want)
    tol = 1e-10 if precision == pkg.FP64 else 2e-6
    assert worst <= tol * scale, worst / scale


def test_full_size_fp32_refined_within_fp64_discretisation_error():
    """256^3 cells, 500 steps, PAPER closure: the FP32_REFINED state is within 2x the FP64 path's
    error against the exact modes and closer to the FP64 state than FP64 is to the exact modes
    (the FP64 path is the oracle's parity-pinned stand-in at this size)."""
    c = workloads.config3()
    n, r, modes, K = c["n"], c["r"], c["modes"], c["steps"]
    out = {}
    for prec in (pkg.FP64, pkg.FP32_REFINED):
        with pkg.Grid(n, r, precision=prec, dim=3) as g:
            g.init_modes(modes)
            g.run(K)
            out[prec] = (g.get_fields(), g.error_vs_exact(modes)[0])
    (f64, e64), (f32, e32) = out[pkg.FP64], out[pkg.FP32_REFINED]
    diff = np.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(f32, f64)) / n ** 3)
    assert e32 <= 2 * e64, (e32, e64)
    assert diff <= e64, (diff, e64)


# --------------------------------------------------------------------------
# Diagnostics: discrete energy and Pade divergence of H (FP64 3D grids)

@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
@pytest.mark.parametrize("n", [8, 13])
def test_fp64_energy_and_divergence_match_oracle(closure, n):
    r, Z, steps = 0.4, 1.3, 2
    init = workloads.random_fields3(n, seed=700 + n)
    o = oracle.Oracle3D(n, r, Z=Z, closure=closure)
    ref = [a.copy() for a in init]
    with pkg.Grid(n, r, z=Z, closure=closure, dim=3) as g:
        g.set_fields(*init)
        for k in range(steps + 1):
            W, d = g.energy(), g.divergence()
            assert abs(W - o.energy(ref)) <= 1e-12 * abs(o.energy(ref)), k
            d_ref = o.divergence(ref)[0]
            assert abs(d - d_ref) <= 1e-12 * d_ref, k
            g.step()
            o.step(ref)


def test_fp64_reflect_energy_and_divergence_conserved():
    n, r = 12, 0.45
    with pkg.Grid(n, r, closure=pkg.CLOSURE_REFLECT, dim=3) as g:
        g.set_fields(*workloads.random_fields3(n, seed=9))
        W0, d0 = g.energy(), g.divergence()
        g.run(20)
        assert abs(g.energy() - W0) <= 1e-12 * W0
        assert abs(g.divergence() - d0) <= 1e-10 * d0


def test_fp32_energy_and_divergence_match_oracle_on_its_state():
    """FP32_REFINED grids evaluate the diagnostics in FP64 on their float-float state: the same
    values as the oracle on that state (read back exactly through ms_get_fields)."""
    n, r = 9, 0.4
    with pkg.Grid(n, r, precision=pkg.FP32_REFINED, dim=3) as g:
        g.set_fields(*workloads.random_fields3(n, seed=3))
        g.run(3)
        o = oracle.Oracle3D(n, r)
        for _ in range(2):  # twice: the FP64 tables and scratch are made on the first call
            state = [np.ascontiguousarray(a) for a in g.get_fields()]
            W, d = g.energy(), g.divergence()
            assert abs(W - o.energy(state)) <= 1e-12 * abs(o.energy(state))
            d_ref = o.divergence(state)[0]
            assert abs(d - d_ref) <= 1e-12 * d_ref
            g.step()
