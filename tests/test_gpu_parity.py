"""Parity of the CUDA path with the FP64 CPU oracle (GB300 only).

Tolerances:
  - FP64 path: relative L2 difference <= 1e-12 after the whole run;
  - FP32_REFINED path: within 2x the oracle's own error against the exact modes and closer to
    the oracle than the oracle is to the exact modes (the mixed-path criterion); on random
    fields, relative L2 difference <= 2e-6.
Inputs come from workloads.py (seeded); expected values come only from oracle/ or from the
closed forms in tests/closed_forms.py, which are pinned to the oracle by test_oracle_pins.py.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from closed_forms import mode_basis, mode_step_matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_17263_gb300 as pkg  # noqa: E402

F = (oracle.F_EZ, oracle.F_HX, oracle.F_HY)


def _cat(fields):
    return np.concatenate([np.asarray(a).ravel() for a in fields])


def _rel(a, b):
    return np.linalg.norm(_cat(a) - _cat(b)) / np.linalg.norm(_cat(b))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------------------------------
# Operators, one kernel at a time

@pytest.mark.parametrize("N", [8, 37, 64, 200])
@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
def test_operators_match_oracle(N, closure):
    r = 0.5
    o = oracle.Oracle2D(N, r, closure=closure)
    g = pkg.Grid(N, r, closure=closure)
    ez, hx, hy = workloads.random_fields(N, seed=N)
    fields = {oracle.F_EZ: ez, oracle.F_HX: hx, oracle.F_HY: hy}
    names = {oracle.F_EZ: "ez", oracle.F_HX: "hx", oracle.F_HY: "hy"}
    for f in F:
        u = fields[f]
        for op, ref in ((f"filter_{names[f]}", o.filter(f, u)), (f"p1_{names[f]}", o.p1(f, u))):
            out = torch.zeros_like(_dev(u))
            g.apply_op(op, [_dev(u)], [out])
            g.sync()
            got = out.cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)), op
        x_ref, _ = o.p1_solve(f, u)
        out = torch.zeros_like(_dev(u))
        g.apply_op(f"p1solve_{names[f]}", [_dev(u)], [out])
        g.sync()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - x_ref)) <= 1e-12 * np.max(np.abs(x_ref)), f
    # curls (Step 1 and Step 2 right-hand sides)
    R_ref = o.curl_h_to_e(hx, hy)
    R = torch.zeros_like(_dev(ez))
    g.apply_op("curl_he", [_dev(hx), _dev(hy)], [R])
    Rx_ref, Ry_ref = o.curl_e_to_h(ez)
    Rx, Ry = torch.zeros_like(_dev(hx)), torch.zeros_like(_dev(hy))
    g.apply_op("curl_eh", [_dev(ez)], [Rx, Ry])
    g.sync()
    for got, ref in ((R, R_ref), (Rx, Rx_ref), (Ry, Ry_ref)):
        got = got.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    g.close()


# ---------------------------------------------------------------------------------------
# Whole steps

def _oracle_run(N, r, closure, init, steps, Z=1.0):
    o = oracle.Oracle2D(N, r, Z=Z, closure=closure)
    ez, hx, hy = (a.copy() for a in init)
    o.run(ez, hx, hy, steps)
    return o, (ez, hx, hy)


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
def test_fp64_config1_matches_oracle(closure):
    c = workloads.config1()
    N, r = c["n"], c["r"]
    o = oracle.Oracle2D(N, r, closure=closure)
    init = o.init_modes(c["modes"])
    _, ref = _oracle_run(N, r, closure, init, c["steps"])
    with pkg.Grid(N, r, closure=closure) as g:
        g.init_modes(c["modes"])
        g.run(c["steps"])
        got = g.get_fields()
        assert g.step_count == c["steps"]
        assert _rel(got, ref) <= 1e-12
        e = g.error_vs_exact(c["modes"])
    e_ref = o.error(c["modes"], c["steps"], *ref)
    # |err_gpu - err_oracle| <= ||u_gpu - u_oracle||_h, which the field check bounds by 1e-12 ||u||
    assert abs(e[0] - e_ref[0]) <= 1e-12


@pytest.mark.parametrize("N,r,Z,steps", [(37, 0.5, 1.0, 25), (50, 5 / (6 * math.sqrt(2)), 2.5, 20),
                                         (16, 0.1, 0.7, 30), (130, 0.6, 1.0, 8)])
@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
def test_fp64_random_fields_match_oracle(N, r, Z, steps, closure):
    init = workloads.random_fields(N, seed=7 * N)
    _, ref = _oracle_run(N, r, closure, init, steps, Z=Z)
    with pkg.Grid(N, r, z=Z, closure=closure) as g:
        g.set_fields(*init)
        for _ in range(steps // 2):
            g.step()
        g.run(steps - steps // 2)
        got = g.get_fields()
    assert _rel(got, ref) <= 1e-12


@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
def test_mixed_config1_within_twice_oracle_error(closure):
    c = workloads.config1()
    N, r = c["n"], c["r"]
    o = oracle.Oracle2D(N, r, closure=closure)
    init = o.init_modes(c["modes"])
    _, ref = _oracle_run(N, r, closure, init, c["steps"])
    exact = o.exact(c["modes"], c["steps"] * o.ht, (c["steps"] + 0.5) * o.ht)
    with pkg.Grid(N, r, precision=pkg.FP32_REFINED, closure=closure) as g:
        g.init_modes(c["modes"])
        g.run(c["steps"])
        got = g.get_fields()
    err_oracle = np.linalg.norm(_cat(ref) - _cat(exact))
    err_mixed = np.linalg.norm(_cat(got) - _cat(exact))
    diff = np.linalg.norm(_cat(got) - _cat(ref))
    assert err_mixed <= 2 * err_oracle
    assert diff <= err_oracle


@pytest.mark.parametrize("N,steps", [(37, 25), (64, 40)])
def test_mixed_random_fields_close_to_oracle(N, steps):
    r = 0.5
    init = workloads.random_fields(N, seed=N + 1)
    _, ref = _oracle_run(N, r, pkg.CLOSURE_PAPER, init, steps)
    with pkg.Grid(N, r, precision=pkg.FP32_REFINED) as g:
        g.set_fields(*init)
        g.run(steps)
        got = g.get_fields()
    assert _rel(got, ref) <= 2e-6


def test_energy_and_divergence_match_oracle():
    N, r = 40, 0.5
    init = workloads.random_fields(N, seed=3)
    for closure in (pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT):
        o = oracle.Oracle2D(N, r, closure=closure)
        W_ref = o.energy(*init)
        d_ref, _ = o.divergence(init[1], init[2])
        for prec in (pkg.FP64, pkg.FP32_REFINED):
            with pkg.Grid(N, r, precision=prec, closure=closure) as g:
                g.set_fields(*init)
                tol = 1e-12 if prec == pkg.FP64 else 1e-6
                assert abs(g.energy() - W_ref) <= tol * abs(W_ref)
                assert abs(g.divergence() - d_ref) <= tol * d_ref


def test_reflect_energy_conserved_on_gpu():
    N, r = 96, 0.5
    init = workloads.random_fields(N, seed=11)
    for prec, tol in ((pkg.FP64, 1e-12), (pkg.FP32_REFINED, 1e-6)):
        with pkg.Grid(N, r, precision=prec, closure=pkg.CLOSURE_REFLECT) as g:
            g.set_fields(*init)
            W0 = g.energy()
            g.run(200)
            assert abs(g.energy() - W0) <= tol * W0


def test_yee_matches_oracle():
    N, r = 48, 0.6
    init = workloads.random_fields(N, seed=5)
    o = oracle.Oracle2D(N, r)
    ref = tuple(a.copy() for a in init)
    for _ in range(30):
        o.yee_step(*ref)
    with pkg.Grid(N, r, scheme=pkg.SCHEME_YEE2) as g:
        g.set_fields(*init)
        g.run(30)
        got = g.get_fields()
    assert _rel(got, ref) <= 1e-13


# ---------------------------------------------------------------------------------------
# Full size (2048 x 2048, the benchmark's configuration), REFLECT closure: the discrete
# solution is the closed-form per-mode recurrence (pinned to the oracle at small N).

def _closed_form_fields(N, r, modes, steps, rows):
    """Exact discrete solution of the REFLECT scheme on the given rows, from the mode recurrence."""
    h = 1.0 / N
    ez = np.zeros((len(rows), N + 1))
    hx = np.zeros((len(rows), N + 1))
    hy = np.zeros((len(rows), N))
    ht = r * h
    for (kx, ky, a) in modes:
        w = math.pi * math.hypot(kx, ky)
        # initial coefficients of the closed-form init (E at 0, H at h_tau/2)
        c = np.array([a, -a * math.sin(w * ht / 2) / w * math.pi * ky, a * math.sin(w * ht / 2) / w * math.pi * kx])
        c = np.linalg.matrix_power(mode_step_matrix(N, r, kx, ky), steps) @ c
        be, bx, by = mode_basis(N, kx, ky)
        ez += c[0] * be[rows]
        hx += c[1] * bx[rows]
        hy += c[2] * by[rows]
    return ez, hx, hy


@pytest.mark.parametrize("prec", [pkg.FP64, pkg.FP32_REFINED])
def test_full_size_reflect_matches_closed_form(prec):
    c = workloads.config2()
    N, r, modes, steps = c["n"], c["r"], c["modes"], c["steps"]
    rows = np.array([1, 2, 37, 511, 1024, 1500, 2045, 2046])
    with pkg.Grid(N, r, precision=prec, closure=pkg.CLOSURE_REFLECT) as g:
        g.init_modes(modes)
        g.run(steps)
        ez, hx, hy = g.get_fields()
        l2_abs, l2_rel, _, _ = g.error_vs_exact(modes)
    ref = _closed_form_fields(N, r, modes, steps, rows)
    got = (ez[rows], hx[rows], hy[rows])
    if prec == pkg.FP64:
        scale = max(np.max(np.abs(a)) for a in ref)
        diff = max(np.max(np.abs(a - b)) for a, b in zip(got, ref))
        assert diff <= 1e-11 * scale
    else:
        # L2 over the sampled rows: distance to the scheme's discrete solution no larger than
        # the scheme's own error against the exact modes, and error within 2x of it
        exact_rows = oracle.Oracle2D(N, r).exact(modes, steps * r / N, (steps + 0.5) * r / N)
        ex = tuple(e[rows] for e in exact_rows)
        l2 = lambda fields: math.sqrt(sum(float(np.sum(a * a)) for a in fields))
        disc = l2([e - b for e, b in zip(ex, ref)])
        assert l2([a - b for a, b in zip(got, ref)]) <= disc
        assert l2([a - e for a, e in zip(got, ex)]) <= 2 * disc
    assert l2_rel < 1e-4


@pytest.mark.parametrize("N,r,Z,steps", [(129, 0.5, 1.0, 12), (150, 5 / (6 * math.sqrt(2)), 1.6, 10),
                                         (191, 0.45, 0.7, 8)])
@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
def test_mixed_multi_tile_ragged_sizes_close_to_oracle(N, r, Z, steps, closure):
    """FP32_REFINED tile kernels over several curl tiles (64) and solve regions (64 - 2(S-1)) with
    ragged last tiles, against the oracle on random fields (FP32 noise ~1e-7 per step)."""
    init = workloads.random_fields(N, seed=2000 + N)
    o = oracle.Oracle2D(N, r, Z=Z, closure=closure)
    ref = [a.copy() for a in init]
    o.run(*ref, steps)
    with pkg.Grid(N, r, z=Z, precision=pkg.FP32_REFINED, closure=closure) as g:
        g.set_fields(*init)
        g.run(steps)
        got = g.get_fields()
    cat = lambda fs: np.concatenate([np.ravel(a) for a in fs])
    assert np.linalg.norm(cat(got) - cat(ref)) <= 2e-6 * np.linalg.norm(cat(ref))


def test_headline_config_mixed_within_fp64_discretisation_error():
    """The benchmarked workload in full: 2048^2 cells, PAPER closure, the 8 seeded modes, 4000
    steps (T = 0.9765625).  The FP32_REFINED state is within 2x the FP64 path's error against the
    exact modes (Sec. 5.1, Eq. "eq:data") and closer to the FP64 state than FP64 is to the exact
    modes.  The FP64 path is the oracle's parity-pinned stand-in at this size (<= 1e-12 against
    the oracle up to N = 200)."""
    c = workloads.config2()
    N, r, modes, K = c["n"], c["r"], c["modes"], c["steps"]
    out = {}
    for prec in (pkg.FP64, pkg.FP32_REFINED):
        with pkg.Grid(N, r, precision=prec, closure=pkg.CLOSURE_PAPER) as g:
            g.init_modes(modes)
            g.run(K)
            out[prec] = (g.get_fields(), g.error_vs_exact(modes)[0])
    (f64, e64), (f32, e32) = out[pkg.FP64], out[pkg.FP32_REFINED]
    # the same h^2-weighted L2 norm as ms_error_vs_exact (wall values are zero in both states)
    diff = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(f32, f64)) / N ** 2)
    assert e32 <= 2 * e64, (e32, e64)
    assert diff <= e64, (diff, e64)


@pytest.mark.parametrize("N", [5, 6, 7, 12, 56, 57, 58, 59, 114, 115, 116, 117])
@pytest.mark.parametrize("closure", [pkg.CLOSURE_PAPER, pkg.CLOSURE_REFLECT])
def test_mixed_solve_region_edges_close_to_oracle(N, closure):
    """Sizes around the solve regions' output width (64 - 2(S-1) = 58 at r = 0.5): one region that
    reaches past both walls, a last region one or two points wide, Neumann ghost columns and rows at
    either lane of a column pair, and the smallest grids; FP32_REFINED against the oracle on random
    fields (every region at a wall takes the masked path with ghost refills)."""
    r, steps = 0.5, 6
    init = workloads.random_fields(N, seed=3000 + N)
    o = oracle.Oracle2D(N, r, closure=closure)
    ref = [a.copy() for a in init]
    o.run(*ref, steps)
    with pkg.Grid(N, r, precision=pkg.FP32_REFINED, closure=closure) as g:
        g.set_fields(*init)
        g.run(steps)
        got = g.get_fields()
    cat = lambda fs: np.concatenate([np.ravel(a) for a in fs])
    assert np.linalg.norm(cat(got) - cat(ref)) <= 2e-6 * np.linalg.norm(cat(ref))
