"""Pins of the oracle's step with currents that do not vanish on the walls (Sec. 3.3, Method 2):
the manufactured solution against Maxwell's equations and the PEC conditions (finite differences),
the ghost data against that solution half a cell outside the walls (fifth order in h), G_E on the
walls against its Laplacian there, the affine ghost part of P1 against the 9-point stencil on an
array extended by the ghost nodes, fourth-order convergence to the manufactured solution, and the
reduction to the sine-mode sources and to the plain step."""
import math

import numpy as np
import pytest

import oracle
from oracle import F_EZ, F_HX, F_HY, manufactured_current, manufactured_field, manufactured_sources

M, N_, A, W, Z = 1, 2, 0.7, 3.0, 1.3


def test_sources_sum_to_the_current():
    rng = np.random.default_rng(3)
    x, y, t = rng.uniform(-0.2, 1.2, 50), rng.uniform(-0.2, 1.2, 50), 0.37
    got = np.zeros(50)
    for m, n, a, w, px, py in manufactured_sources(M, N_, A, W, Z):
        X = np.cos(m * np.pi * x) if px else np.sin(m * np.pi * x)
        Y = np.cos(n * np.pi * y) if py else np.sin(n * np.pi * y)
        got += a * X * Y * np.sin(w * t)
    ref = manufactured_current(M, N_, A, W, Z, x, y, t)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_manufactured_solution_solves_maxwell_with_pec_walls():
    rng = np.random.default_rng(4)
    x, y, t = rng.uniform(0.05, 0.95, 40), rng.uniform(0.05, 0.95, 40), rng.uniform(0.1, 1.0, 40)
    d = 1e-4

    def F(c, xx, yy, tt):
        return manufactured_field(M, N_, A, W, Z, c, xx, yy, tt)

    def dd(c, ax, xx, yy, tt):  # fourth-order central difference
        e = np.eye(3)[ax] * d
        f = [F(c, xx + k * e[0], yy + k * e[1], tt + k * e[2]) for k in (-2, -1, 1, 2)]
        return (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * d)

    J = manufactured_current(M, N_, A, W, Z, x, y, t)
    # Ampere: d_t E_z = Z (d_x H_y - d_y H_x - J_z);  Faraday: d_t H_x = -d_y E_z / Z, d_t H_y = d_x E_z / Z
    amp = dd(F_EZ, 2, x, y, t) - Z * (dd(F_HY, 0, x, y, t) - dd(F_HX, 1, x, y, t) - J)
    far_x = dd(F_HX, 2, x, y, t) + dd(F_EZ, 1, x, y, t) / Z
    far_y = dd(F_HY, 2, x, y, t) - dd(F_EZ, 0, x, y, t) / Z
    for r in (amp, far_x, far_y):
        assert np.abs(r).max() < 1e-7
    s = np.linspace(0, 1, 13)
    for wall in (0.0, 1.0):
        assert np.abs(F(F_EZ, wall, s, 0.4)).max() < 1e-14 and np.abs(F(F_EZ, s, wall, 0.4)).max() < 1e-14
        assert np.abs(F(F_HX, wall, s, 0.4)).max() < 1e-13 and np.abs(F(F_HY, s, wall, 0.4)).max() < 1e-13
    # the Neumann data of the tangential H on the walls is the current, not zero
    assert np.abs(manufactured_current(M, N_, A, W, Z, s, 0.0, 0.4)).max() > 0.1


def _ghost_errors(N, t0, t1, diff):
    o = oracle.Oracle2D(N, 0.5, Z=Z)
    h = o.h
    gxl, gxh, gyl, gyh = o.wall_ghosts(manufactured_sources(M, N_, A, W, Z), t0, t1, diff)
    xi = np.arange(1, N) * h  # unknown columns of H_x, unknown rows of H_y

    def H(c, xx, yy):
        v = manufactured_field(M, N_, A, W, Z, c, xx, yy, t1)
        return (v - manufactured_field(M, N_, A, W, Z, c, xx, yy, t0)) / o.ht if diff else v

    exact = [H(F_HX, xi, h / 2) - H(F_HX, xi, -h / 2), H(F_HX, xi, 1 + h / 2) - H(F_HX, xi, 1 - h / 2),
             H(F_HY, h / 2, xi) - H(F_HY, -h / 2, xi), H(F_HY, 1 + h / 2, xi) - H(F_HY, 1 - h / 2, xi)]
    got = [gxl[1:N], gxh[1:N], gyl[1:N], gyh[1:N]]
    return [float(np.abs(g - e).max()) for g, e in zip(got, exact)], [float(np.abs(e).max()) for e in exact]


@pytest.mark.parametrize("diff", [0, 1])
def test_ghost_data_match_the_solution_outside_the_walls_to_fifth_order(diff):
    t0, t1 = 0.31, 0.31 + 0.5 / 16 if diff else 0.31
    e16, size = _ghost_errors(16, t0, t1, diff)
    e32, _ = _ghost_errors(32, t0, 0.31 + 0.5 / 32 if diff else 0.31, diff)
    for a, b, s in zip(e16, e32, size):
        assert s > 1e-3  # the data are not trivially zero on any wall
        assert a < 1e-3 * s, (e16, size)
        assert a / b > 25.0, (e16, e32)  # h^5: 32; a missing or wrong h^3 term would give 8


def test_ge_on_the_walls_is_the_laplacian_of_e_there():
    o = oracle.Oracle2D(12, 0.5, Z=Z)
    t = 0.23
    ge = o.ge_wall(manufactured_sources(M, N_, A, W, Z), t)
    d = 1e-3
    x = np.arange(o.N + 1) * o.h

    def lap(xx, yy):  # fourth-order central second differences along each axis
        f = lambda a, b: manufactured_field(M, N_, A, W, Z, F_EZ, a, b, t)
        c = [-1 / 12, 4 / 3, -5 / 2, 4 / 3, -1 / 12]
        return sum(ck * (f(xx + k * d, yy) + f(xx, yy + k * d)) for ck, k in zip(c, range(-2, 3))) / d ** 2

    ref = np.zeros_like(ge)
    ref[0, :], ref[-1, :] = lap(x, 0.0), lap(x, 1.0)
    ref[:, 0], ref[:, -1] = lap(0.0, x), lap(1.0, x)
    ref *= o.h ** 2 / 12
    assert np.abs(ge[1:-1, 1:-1]).max() == 0.0
    assert np.abs(ge - ref).max() <= 1e-8 * np.abs(ref).max()
    assert np.abs(ref).max() > 1e-3


@pytest.mark.parametrize("f", [F_HX, F_HY])
def test_p1_ghost_part_is_the_nine_point_stencil_with_ghost_nodes(f):
    N = 9
    o = oracle.Oracle2D(N, 0.45, Z=1.0)
    rng = np.random.default_rng(7 + f)
    glo, ghi = rng.standard_normal(N + 1), rng.standard_normal(N + 1)
    x = rng.standard_normal(o.shape(f))
    # zero the Dirichlet boundary entries of x
    if f == F_HX:
        x[:, 0] = x[:, -1] = 0.0
    else:
        x[0, :] = x[-1, :] = 0.0
    # extended array: one ghost line beyond each Neumann wall, u(-1) = u(0) - g_lo, u(n) = u(n-1) + g_hi;
    # ghosts beside the Dirichlet walls are not reached by any unknown's stencil except through the
    # zero Dirichlet values, which the scheme keeps at zero
    if f == F_HX:
        ext = np.zeros((N + 2, N + 1))
        ext[1:-1] = x
        ext[0, 1:-1] = x[0, 1:-1] - glo[1:-1]
        ext[-1, 1:-1] = x[-1, 1:-1] + ghi[1:-1]
    else:
        ext = np.zeros((N + 1, N + 2))
        ext[:, 1:-1] = x
        ext[1:-1, 0] = x[1:-1, 0] - glo[1:-1]
        ext[1:-1, -1] = x[1:-1, -1] + ghi[1:-1]
    h2 = o.h ** 2
    w9 = np.array([[1, -2, 1], [-2, 4, -2], [1, -2, 1]]) / h2 ** 2  # D_xx D_yy
    ref = np.zeros_like(x)
    for j in range(x.shape[0]):
        for i in range(x.shape[1]):
            if f == F_HX and (i == 0 or i == N):
                continue
            if f == F_HY and (j == 0 or j == N):
                continue
            je, ie = (j + 1, i) if f == F_HX else (j, i + 1)
            blk = ext[je - 1:je + 2, ie - 1:ie + 2]
            lap = (blk[1, 0] + blk[1, 2] + blk[0, 1] + blk[2, 1] - 4 * blk[1, 1]) / h2
            ref[j, i] = o.c1 * blk[1, 1] - lap - h2 / 6 * float(np.sum(w9 * blk))
    got = o.p1(f, x) + o.p1_ghost_shift(f, glo, ghi)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("m,n,Zc", [(1, 1, 1.3), (1, 2, 1.0)])
def test_fourth_order_convergence_to_the_manufactured_solution(m, n, Zc):
    T, errs = 0.5, []
    for N in (16, 32, 64):
        o = oracle.Oracle2D(N, 0.5, Z=Zc)
        src = manufactured_sources(m, n, A, W, Zc)
        K = int(round(T / o.ht))
        f = o.exact_manufactured(m, n, A, W, 0.0, 0.5 * o.ht)
        for s in range(K):
            o.step_src_xy(*f, src, s)
        ex = o.exact_manufactured(m, n, A, W, K * o.ht, (K + 0.5) * o.ht)
        errs.append(math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(f, ex))) / N)
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 3.7, (errs, rates)


def test_sine_rows_reduce_to_the_sine_mode_sources():
    o = oracle.Oracle2D(14, 0.5, Z=1.3)
    src4 = [(2, 3, 1.0, 5.0), (1, 1, -0.5, 11.0)]
    src6 = [s + (0, 0) for s in src4]
    a = list(o.exact_driven(src4, 0.0, 0.5 * o.ht))
    b = [x.copy() for x in a]
    for s in range(4):
        o.step_src(*a, src4, s)
        o.step_src_xy(*b, src6, s)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-13 * np.abs(x).max()


def test_zero_amplitude_rows_equal_the_plain_step():
    import workloads
    o = oracle.Oracle2D(12, 0.5)
    a = list(workloads.random_fields(12, seed=6))
    b = [x.copy() for x in a]
    for s in range(3):
        o.step(*a)
        o.step_src_xy(*b, [(2, 0, 0.0, 3.0, 1, 1), (1, 3, 0.0, 2.0, 0, 1)], s)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
