"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: polynomial
exactness of the Pade rows, closed-form eigenvalues, a dense Kronecker assembly
from App. A.1, brute-force dense solves, the closed-form per-mode evolution of
the scheme under the REFLECT closure, and the values the paper prints in
Tables "table:cfl" and "table:conv_rates".
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import CLOSURE_PAPER, CLOSURE_REFLECT, F_EZ, F_HX, F_HY, HALF_TO_NODE, NODE_TO_HALF
from closed_forms import d2_symbol, mode_basis, mode_step_matrix, pade_symbol

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Pade derivative, App. A.1 Eq. "eq:lhs"

@pytest.mark.parametrize("M", [5, 8, 13, 31])
@pytest.mark.parametrize("kind", [HALF_TO_NODE, NODE_TO_HALF])
def test_pade_paper_rows_exact_through_degree_4(M, kind):
    """Both the interior row [1,22,1]/24 and the one-sided rows [26,-5,4,-1]/24 are
    fourth order: exact on polynomials of degree <= 4, not on degree 5."""
    h = 1.0
    x = np.arange(M + 1) * h - 0.4 * M
    xm = x[:-1] + h / 2
    for p in range(0, 6):
        fp = oracle.pade_line(x ** p, h, CLOSURE_PAPER, kind)
        exact = p * xm ** (p - 1) if p > 0 else np.zeros(M)
        err = np.max(np.abs(fp - exact)) / max(1.0, np.max(np.abs(exact)))
        if p <= 4:
            assert err < 1e-12, (p, err)
        else:
            assert err > 1e-8, (p, err)


@pytest.mark.parametrize("N", [6, 16, 33])
def test_pade_reflect_rows_exact_on_cavity_modes(N):
    """REFLECT closure: sin on nodes maps to d cos on half-nodes (node->half), cos on
    half-nodes maps to -d sin on interior nodes (half->node), d the Pade symbol."""
    h = 1.0 / N
    for k in range(1, N):
        th = math.pi * k * h
        d = pade_symbol(th, h)
        f = np.sin(th * np.arange(N + 1))
        f[0] = f[-1] = 0.0
        got = oracle.pade_line(f, h, CLOSURE_REFLECT, NODE_TO_HALF)
        assert np.allclose(got, d * np.cos(th * (np.arange(N) + 0.5)), atol=1e-10 * d, rtol=0)
        g = np.cos(th * (np.arange(N) + 0.5))
        got = oracle.pade_line(g, h, CLOSURE_REFLECT, HALF_TO_NODE)
        assert np.allclose(got, -d * np.sin(th * np.arange(1, N)), atol=1e-10 * d, rtol=0)


def test_pade_matrix_rows_match_eq_lhs():
    """The assembled 24*A has the printed rows: first [26,-5,4,-1], interior [1,22,1], last reversed."""
    M = 7
    A = np.array([oracle.pade_matvec24(np.eye(M)[:, j]) for j in range(M)]).T
    assert np.array_equal(A[0, :4], [26, -5, 4, -1])
    assert np.array_equal(A[-1, -4:], [-1, 4, -5, 26])
    for i in range(1, M - 1):
        assert np.array_equal(A[i, i - 1:i + 2], [1, 22, 1])
        assert np.count_nonzero(A[i]) == 3


# --------------------------------------------------------------------------
# D_2, Delta_h, the filter, P1 and P2 (App. A.1, Eq. "eq:ell", Def. "def:operatorsP")

def _dense_d2(n, bc, h):
    """D_2 of App. A.1 (Dirichlet) or with the even ghost of Corollary "cor:ghost_cor" (Neumann)."""
    D = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1))
    if bc == "neu":
        D[0, 0] = D[-1, -1] = -1.0
    return D / h ** 2


def _dense_ops(o, f):
    """Dense D_xx, D_yy on the interior unknowns of field f (x fastest), Kronecker lifts of App. A.1."""
    N, h = o.N, o.h
    bx, by = {F_EZ: ("dir", "dir"), F_HX: ("dir", "neu"), F_HY: ("neu", "dir")}[f]
    nx = N - 1 if bx == "dir" else N
    ny = N - 1 if by == "dir" else N
    Dx, Dy = _dense_d2(nx, bx, h), _dense_d2(ny, by, h)
    Dxx = np.kron(np.eye(ny), Dx)
    Dyy = np.kron(Dy, np.eye(nx))
    return Dxx, Dyy, nx, ny, bx, by


def _interior_slices(f, bx, by):
    return (slice(1, -1) if by == "dir" else slice(None), slice(1, -1) if bx == "dir" else slice(None))


@pytest.mark.parametrize("N", [4, 5, 7])
@pytest.mark.parametrize("f", [F_EZ, F_HX, F_HY])
@pytest.mark.parametrize("r", [0.5, 5 / (6 * math.sqrt(2))])
def test_p1_matches_dense_kronecker_assembly(N, f, r):
    o = oracle.Oracle2D(N, r)
    Dxx, Dyy, nx, ny, bx, by = _dense_ops(o, f)
    P1 = o.c1 * np.eye(nx * ny) - (Dxx + Dyy + o.h ** 2 / 6.0 * Dxx @ Dyy)
    sl = _interior_slices(f, bx, by)
    rng = np.random.default_rng(1)
    for _ in range(3):
        u = o.zeros(f)
        u[sl] = rng.standard_normal((ny, nx))
        got = o.p1(f, u)
        assert np.allclose(got[sl].ravel(), P1 @ u[sl].ravel(), rtol=1e-13, atol=1e-13 * np.abs(P1).max())
        lap = o.laplacian(f, u)
        assert np.allclose(lap[sl].ravel(), (Dxx + Dyy) @ u[sl].ravel(), rtol=1e-13, atol=1e-12 / o.h ** 2)
        G = o.filter(f, u)
        assert np.allclose(G[sl].ravel(), o.beta * u[sl].ravel() + o.h ** 2 / 12 * (Dxx + Dyy) @ u[sl].ravel(),
                           rtol=1e-13, atol=1e-12)
        # Dirichlet boundary points stay zero
        mask = np.ones(o.shape(f), bool)
        mask[sl] = False
        assert np.all(got[mask] == 0.0) and np.all(G[mask] == 0.0)
    # closed-form eigenvalues: mu_x + mu_y - (h^2/6) mu_x mu_y + c1
    kx = range(1, N) if bx == "dir" else range(0, N)
    ky = range(1, N) if by == "dir" else range(0, N)
    mu = lambda k: (4 / o.h ** 2) * math.sin(math.pi * k / (2 * N)) ** 2
    ev = sorted(mu(a) + mu(b) - o.h ** 2 / 6 * mu(a) * mu(b) + o.c1 for a in kx for b in ky)
    assert np.allclose(np.linalg.eigvalsh(P1), ev, rtol=1e-12)


@pytest.mark.parametrize("r", [0.2, 0.5, 5 / (6 * math.sqrt(2)), 1.0])
def test_p1_p2_spectral_bounds(r):
    """App. A.2: (h_tau^2/24) sigma(P1) within [1+2/r^2 - r^2/6, 1+2/r^2 + r^2/2] and
    (h_tau^2/24) sigma(-P2) within [2/r^2, 1+2/r^2]; both SPD (r < sqrt(3+sqrt(21)))."""
    N = 6
    o = oracle.Oracle2D(N, r)
    for f in (F_EZ, F_HX, F_HY):
        Dxx, Dyy, nx, ny, bx, by = _dense_ops(o, f)
        sl = _interior_slices(f, bx, by)
        n = nx * ny
        P1 = np.zeros((n, n))
        P2 = np.zeros((n, n))
        for c in range(n):
            u = o.zeros(f)
            u[sl] = np.eye(n)[c].reshape(ny, nx)
            P1[:, c] = o.p1(f, u)[sl].ravel()
            P2[:, c] = o.p2(f, u)[sl].ravel()
        assert np.allclose(P1, P1.T, rtol=1e-13) and np.allclose(P2, P2.T, rtol=1e-13)
        s1 = np.linalg.eigvalsh(P1) * o.ht ** 2 / 24
        s2 = np.linalg.eigvalsh(-P2) * o.ht ** 2 / 24
        b = 1 + 2 / r ** 2
        assert s1.min() >= b - r ** 2 / 6 - 1e-12 and s1.max() <= b + r ** 2 / 2 + 1e-12
        # sharper bound of the same symbol: [b, b + 2 r^2 / 9]
        assert s1.min() >= b - 1e-12 and s1.max() <= b + 2 * r ** 2 / 9 + 1e-12
        assert s2.min() >= 2 / r ** 2 - 1e-12 and s2.max() <= b + 1e-12


@pytest.mark.parametrize("N", [5, 8])
@pytest.mark.parametrize("f", [F_EZ, F_HX, F_HY])
def test_cg_matches_dense_solve(N, f):
    o = oracle.Oracle2D(N, 0.5)
    Dxx, Dyy, nx, ny, bx, by = _dense_ops(o, f)
    P1 = o.c1 * np.eye(nx * ny) - (Dxx + Dyy + o.h ** 2 / 6.0 * Dxx @ Dyy)
    sl = _interior_slices(f, bx, by)
    rng = np.random.default_rng(2)
    b = o.zeros(f)
    b[sl] = rng.standard_normal((ny, nx))
    x, it = o.p1_solve(f, b)
    ref = np.linalg.solve(P1, b[sl].ravel())
    assert np.allclose(x[sl].ravel(), ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
    assert it <= 8


@pytest.mark.parametrize("N", [16, 32, 64, 128])
def test_cg_needs_about_three_iterations(N):
    """Sec. 6: at fixed CFL number about three CG iterations per solve, independent of N."""
    o = oracle.Oracle2D(N, 5 / (6 * math.sqrt(2)))
    o.set_cg(1e-8)
    m = [(2, 3, 1.0), (5, 1, 0.5)]
    ez, hx, hy = o.init_modes(m)
    o.run(ez, hx, hy, 4)
    it, solves = o.cg_stats()
    assert solves == 12
    assert 2.0 <= it / solves <= 4.0


# --------------------------------------------------------------------------
# Whole step against closed forms

@pytest.mark.parametrize("N,kx,ky", [(12, 1, 1), (16, 2, 3), (16, 7, 2), (21, 5, 11)])
@pytest.mark.parametrize("Z", [1.0, 2.5])
def test_reflect_step_equals_mode_recurrence(N, kx, ky, Z):
    """REFLECT closure: every operator is diagonal on the mode bases, so n steps equal the
    n-th power of the closed-form 3x3 step matrix on the coefficients (e, a, b)."""
    r = 0.5
    o = oracle.Oracle2D(N, r, Z=Z, closure=CLOSURE_REFLECT)
    be, bx_, by_ = mode_basis(N, kx, ky)
    c0 = np.array([0.7, -0.3, 0.45])
    ez, hx, hy = c0[0] * be, c0[1] * bx_, c0[2] * by_
    S = mode_step_matrix(N, r, kx, ky, Z)
    c = c0.copy()
    for n in range(25):
        o.step(ez, hx, hy)
        c = S @ c
    scale = np.abs(c).max()
    assert np.allclose(ez, c[0] * be, atol=1e-12 * scale, rtol=0)
    assert np.allclose(hx, c[1] * bx_, atol=1e-12 * scale, rtol=0)
    assert np.allclose(hy, c[2] * by_, atol=1e-12 * scale, rtol=0)


def test_reflect_step_is_linear_superposition():
    N, r = 20, 0.5
    o = oracle.Oracle2D(N, r, closure=CLOSURE_REFLECT)
    modes = [(1, 2, 1.0), (3, 1, -0.5), (6, 9, 0.25), (13, 4, 0.1)]
    fields = [np.zeros(o.shape(f)) for f in (F_EZ, F_HX, F_HY)]
    expect = [np.zeros(o.shape(f)) for f in (F_EZ, F_HX, F_HY)]
    for kx, ky, a in modes:
        b = mode_basis(N, kx, ky)
        c = np.array([a, 0.3 * a, -0.2 * a])
        for k in range(3):
            fields[k] += c[k] * b[k]
        c = np.linalg.matrix_power(mode_step_matrix(N, r, kx, ky), 10) @ c
        for k in range(3):
            expect[k] += c[k] * b[k]
    for _ in range(10):
        o.step(*fields)
    for k in range(3):
        assert np.allclose(fields[k], expect[k], atol=1e-12, rtol=0)


def test_exact_modes_satisfy_scaled_maxwell():
    """Eq. "eq:data" with general Z solves Eq. "eq:maxwellv" (2D TM_z): checked with
    fourth-order central differences in tau, x and y on a fine grid."""
    N, Z = 200, 1.7
    o = oracle.Oracle2D(N, 0.5, Z=Z)
    m = [(2, 3, 1.0), (1, 4, -0.6)]
    t, dt, h = 0.31, 1e-3, o.h

    def fields(tt):
        return o.exact(m, tt, tt)

    def d_dt(k):
        fm2, fm1, fp1, fp2 = (fields(t + s * dt)[k] for s in (-2, -1, 1, 2))
        return (fm2 - 8 * fm1 + 8 * fp1 - fp2) / (12 * dt)

    ez, hx, hy = fields(t)
    # dE/dt = Z (dHy/dx - dHx/dy) at interior node (i,j): Hy at half-nodes in x, Hx at half-nodes in y
    i, j = 57, 91
    dhy_dx = (hy[j, i - 2] - 27 * hy[j, i - 1] + 27 * hy[j, i] - hy[j, i + 1]) / (24 * h)
    dhx_dy = (hx[j - 2, i] - 27 * hx[j - 1, i] + 27 * hx[j, i] - hx[j + 1, i]) / (24 * h)
    assert abs(d_dt(0)[j, i] - Z * (dhy_dx - dhx_dy)) < 1e-5
    # dHx/dt = -(1/Z) dEz/dy at (x_i, y_{j+1/2}); dHy/dt = (1/Z) dEz/dx at (x_{i+1/2}, y_j)
    dez_dy = (ez[j - 1, i] - 27 * ez[j, i] + 27 * ez[j + 1, i] - ez[j + 2, i]) / (24 * h)
    dez_dx = (ez[j, i - 1] - 27 * ez[j, i] + 27 * ez[j, i + 1] - ez[j, i + 2]) / (24 * h)
    assert abs(d_dt(1)[j, i] + dez_dy / Z) < 1e-5
    assert abs(d_dt(2)[j, i] - dez_dx / Z) < 1e-5


def test_reflect_energy_and_divergence_conserved():
    """Leapfrog invariant W^n and the Pade divergence of H are conserved to round-off."""
    N = 24
    o = oracle.Oracle2D(N, 0.5, closure=CLOSURE_REFLECT)
    rng = np.random.default_rng(5)
    ez, hx, hy = o.zeros(F_EZ), o.zeros(F_HX), o.zeros(F_HY)
    ez[1:-1, 1:-1] = rng.standard_normal((N - 1, N - 1))
    hx[:, 1:-1] = rng.standard_normal((N, N - 1))
    hy[1:-1, :] = rng.standard_normal((N - 1, N))
    W0 = o.energy(ez, hx, hy)
    d0, div0 = o.divergence(hx, hy)
    assert d0 > 1.0  # random H is far from divergence-free
    for _ in range(60):
        o.step(ez, hx, hy)
    assert abs(o.energy(ez, hx, hy) - W0) < 1e-12 * W0
    d1, div1 = o.divergence(hx, hy)
    assert np.max(np.abs(div1 - div0)) < 1e-10 * np.max(np.abs(div0))


def test_paper_closure_energy_bounded():
    """PAPER closure: W is not an exact invariant, but stays within a small band (no growth)."""
    N = 32
    o = oracle.Oracle2D(N, 0.5, closure=CLOSURE_PAPER)
    m = [(2, 3, 1.0), (7, 5, 0.4)]
    ez, hx, hy = o.init_modes(m)
    W = [o.energy(ez, hx, hy)]
    for _ in range(8):
        o.run(ez, hx, hy, 40)
        W.append(o.energy(ez, hx, hy))
    W = np.array(W)
    assert (W.max() - W.min()) / W[0] < 1e-4


# --------------------------------------------------------------------------
# Printed results of Sec. 5

def _mae(N, r, k, T):
    o = oracle.Oracle2D(N, r)
    m = [(k, k, 1.0)]
    ez, hx, hy = o.init_modes(m)
    n = int(round(T / o.ht))
    return o.run(ez, hx, hy, n, m), n, T / o.ht


@pytest.mark.parametrize("k", ["2", "21"])
def test_table_cfl_mean_absolute_error(k):
    """Table "table:cfl", C4 column: MAE vs CFL number r = j/(6 sqrt 2), h = 1/64, T = 4/sqrt 2.
    Where T/h_tau is an integer the oracle is within 15% of the printed value; for j = 5
    (T/h_tau = 307.2, step count rounded) within 20%."""
    gold = json.load(open(os.path.join(GOLDEN, "table_cfl_c4.json")))
    for j, want in zip(gold["r_numerators_over_6sqrt2"], gold["mae"][k]):
        got, n, exact_n = _mae(gold["N"], j / (6 * math.sqrt(2)), int(k), gold["T"])
        tol = 0.15 if abs(exact_n - n) < 1e-9 else 0.20
        assert abs(got - want) <= tol * want, (k, j, got, want)


def test_table_conv_rates_small_cfl():
    """Table "table:conv_rates", r = 1/(6 sqrt 2) (integral step counts): rates within 0.1."""
    gold = json.load(open(os.path.join(GOLDEN, "table_conv_rates_c4.json")))
    for case in gold["cases"]:
        if case["r_num"] != 1:
            continue
        k, r = case["k"], 1 / (6 * math.sqrt(2))
        Ns = [16, 32, 64, 128] if k == 2 else [32, 64, 128]
        maes = [_mae(N, r, k, gold["T"])[0] for N in Ns]
        for a in range(1, len(Ns)):
            want = case["rate"][case["N"].index(Ns[a])]
            got = math.log2(maes[a - 1] / maes[a])
            assert abs(got - want) < 0.1, (k, Ns[a], got, want)


def test_fourth_order_at_paper_cfl():
    """Table "table:conv_rates", r = 5/(6 sqrt 2), k = 2: rates near 5 (printed 5.06, 4.98)."""
    T = 1 / math.sqrt(2)
    r = 5 / (6 * math.sqrt(2))
    m = [_mae(N, r, 2, T)[0] for N in (16, 32, 64)]
    rates = [math.log2(m[0] / m[1]), math.log2(m[1] / m[2])]
    assert all(4.5 < q < 5.5 for q in rates), rates


def test_unstable_at_r_one_over_sqrt2_stable_below():
    """Table "table:cfl": r = 1/sqrt 2 diverges; Sec. 4: r <= 5/(6 sqrt 2) is stable."""
    N = 32
    rng = np.random.default_rng(3)

    def growth(r):
        o = oracle.Oracle2D(N, r)
        ez, hx, hy = o.zeros(F_EZ), o.zeros(F_HX), o.zeros(F_HY)
        ez[1:-1, 1:-1] = rng.standard_normal((N - 1, N - 1))
        n0 = np.linalg.norm(ez)
        o.run(ez, hx, hy, 300)
        return np.linalg.norm(ez) / n0

    assert growth(1 / math.sqrt(2)) > 1e6
    assert growth(5 / (6 * math.sqrt(2))) < 10


def test_exact_fourier_stability_limit():
    """Sec. 4 recurrence sigma^2 - (2 - lambda^2 h_tau^2) sigma + 1 = 0: with the symbols, the
    largest stable r (2D, periodic symbol) lies between the paper's bound 5/(6 sqrt 2) and 1/sqrt 2."""
    def max_amp(r):
        N = 400
        worst = 0.0
        for kx in (N - 1, N - 2, N // 2):
            for ky in (N - 1, N - 3):
                S = mode_step_matrix(N, r, kx, ky)
                worst = max(worst, np.max(np.abs(np.linalg.eigvals(S))))
        return worst
    assert max_amp(5 / (6 * math.sqrt(2))) < 1 + 1e-9
    assert max_amp(1 / math.sqrt(2)) > 1 + 1e-3


# --------------------------------------------------------------------------
# Yee comparator (Sec. 5.2, stencil S with c = 1)

@pytest.mark.parametrize("kx,ky", [(1, 2), (5, 3)])
def test_yee_step_matches_its_symbol(kx, ky):
    """Plain Yee on a mode: the same 3x3 recurrence with d = (2/h) sin(theta/2) and no filter/P1."""
    N, r = 16, 0.6
    o = oracle.Oracle2D(N, r)
    h, ht = o.h, o.ht
    dx, dy = (2 / h) * math.sin(math.pi * kx * h / 2), (2 / h) * math.sin(math.pi * ky * h / 2)
    S1 = np.array([[1, ht * dy, -ht * dx], [0, 1, 0], [0, 0, 1]])
    S2 = np.array([[1, 0, 0], [-ht * dy, 1, 0], [ht * dx, 0, 1]])
    S = S2 @ S1
    be, bx_, by_ = mode_basis(N, kx, ky)
    c = np.array([1.0, 0.2, -0.1])
    ez, hx, hy = c[0] * be, c[1] * bx_, c[2] * by_
    for _ in range(30):
        o.yee_step(ez, hx, hy)
        c = S @ c
    assert np.allclose(ez, c[0] * be, atol=1e-12)
    assert np.allclose(hx, c[1] * bx_, atol=1e-12)
    assert np.allclose(hy, c[2] * by_, atol=1e-12)
    # discrete dispersion sin(w h_tau / 2) = r sqrt(sin^2(pi kx h/2) + sin^2(pi ky h/2))
    lam = np.linalg.eigvals(S)
    w_num = np.max(np.abs(np.angle(lam))) / ht
    w_th = 2 / ht * math.asin(r * math.hypot(math.sin(math.pi * kx * h / 2), math.sin(math.pi * ky * h / 2)))
    assert abs(w_num - w_th) < 1e-10 * w_th
