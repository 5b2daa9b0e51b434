"""Pins of the 3D oracle (six components) against facts other than itself: closed-form spectra
of the compact operators with the boundary types of Table "tab:bc", reduction to the (pinned) 2D
oracle for fields independent of one coordinate, the per-mode recurrence under the REFLECT
closure, exact cavity modes of Maxwell's equations, and fourth-order convergence."""
import math

import numpy as np
import pytest

import oracle
import workloads
from closed_forms import mode_basis3, mode_step_matrix3
from oracle import CLOSURE_PAPER, CLOSURE_REFLECT

pytestmark = pytest.mark.filterwarnings("ignore")


def _spectrum_1d(N, bc):
    k = np.arange(1, N) if bc == 0 else np.arange(0, N)
    return (4.0 * N * N) * np.sin(np.pi * k / (2 * N)) ** 2  # eigenvalues of -D_2


def _dense(o, c, apply):
    shp = o.shape(c)
    mask = np.zeros(shp, dtype=bool)
    nz, ny, nx = shp
    idx = [np.arange(nx), np.arange(ny), np.arange(nz)]
    keep = []
    for a in range(3):
        n_a = [nx, ny, nz][a]
        keep.append(np.arange(1, n_a - 1) if o.bc(c, a) == 0 else np.arange(n_a))
    mask[np.ix_(keep[2], keep[1], keep[0])] = True
    pos = np.flatnonzero(mask.ravel())
    A = np.zeros((pos.size, pos.size))
    for q, pp in enumerate(pos):
        e = np.zeros(shp)
        e.ravel()[pp] = 1.0
        A[:, q] = apply(c, e).ravel()[pos]
    return A


@pytest.mark.parametrize("N", [4, 5])
@pytest.mark.parametrize("c", range(6))
def test_operator_spectra_closed_form(N, c):
    o = oracle.Oracle3D(N, 0.4)
    h = 1.0 / N
    mus = [_spectrum_1d(N, o.bc(c, a)) for a in range(3)]
    mx, my, mz = np.meshgrid(*mus, indexing="ij")
    s1 = (mx + my + mz).ravel()
    s2 = (mx * my + my * mz + mz * mx).ravel()
    for apply, ref in ((o.laplacian, -s1), (o.filter, o.beta - h * h / 12 * s1),
                       (o.p1, o.c1 + s1 - h * h / 6 * s2)):
        A = _dense(o, c, apply)
        assert np.allclose(A, A.T, rtol=0, atol=1e-9 * np.abs(A).max())
        ev = np.sort(np.linalg.eigvalsh(0.5 * (A + A.T)))
        assert np.allclose(ev, np.sort(ref), rtol=1e-12, atol=1e-9 * np.abs(ref).max())


def _extrude(o2_fields, N, axis):
    """3D fields independent of `axis` from a 2D TM_z state (ez, hx, hy) of the plane of the other
    two axes (taken in cyclic order: the 2D x is axis+1, the 2D y is axis+2)."""
    ez, hx, hy = o2_fields
    o3 = oracle.Oracle3D(N, 0.4)
    f = [o3.zeros(c) for c in range(6)]
    # component mapping: 2D E_z -> E_axis, 2D H_x -> H_{axis+1}, 2D H_y -> H_{axis+2}
    m2 = {axis: ez, 3 + (axis + 1) % 3: hx, 3 + (axis + 2) % 3: hy}
    for c, a2 in m2.items():
        # a2 is [y2][x2] with x2 = axis+1, y2 = axis+2; broadcast along `axis` into [z][y][x]
        ax1, ax2 = (axis + 1) % 3, (axis + 2) % 3
        nd = f[c].shape[::-1]  # (nx, ny, nz)
        full = np.empty(nd)  # [x][y][z] indexing by axis number
        src = np.moveaxis(np.broadcast_to(a2.T[:, :, None], (a2.shape[1], a2.shape[0], nd[axis])), [0, 1, 2],
                          [ax1, ax2, axis])
        full[...] = src
        f[c] = np.ascontiguousarray(full.transpose(2, 1, 0))
    return f, m2


@pytest.mark.parametrize("closure", [CLOSURE_PAPER, CLOSURE_REFLECT])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_reduces_to_2d_for_fields_independent_of_one_axis(closure, axis):
    N, r, Z, K = 9, 0.4, 1.3, 3
    o2 = oracle.Oracle2D(N, r, Z=Z, closure=closure)
    o3 = oracle.Oracle3D(N, r, Z=Z, closure=closure)
    s2 = list(workloads.random_fields(N, seed=70 + axis))
    f, m2 = _extrude(s2, N, axis)
    o3.run(f, K)
    for _ in range(K):
        o2.step(*s2)
    ref, _ = _extrude(s2, N, axis)
    for c in range(6):
        scale = max(1.0, np.abs(ref[c]).max())
        assert np.abs(f[c] - ref[c]).max() <= 1e-12 * scale, c


@pytest.mark.parametrize("mnp", [(2, 3, 1), (1, 1, 2), (3, 1, 2)])
def test_reflect_step_is_the_mode_recurrence(mnp):
    N, r, Z, K = 8, 0.4, 1.7, 5
    o = oracle.Oracle3D(N, r, Z=Z, closure=CLOSURE_REFLECT)
    basis = mode_basis3(N, *mnp)
    coef = np.random.default_rng(sum(mnp)).standard_normal(6)
    f = [np.ascontiguousarray(coef[c] * basis[c]) for c in range(6)]
    o.run(f, K)
    want = np.linalg.matrix_power(mode_step_matrix3(N, r, *mnp, Z=Z), K) @ coef
    for c in range(6):
        ref = want[c] * basis[c]
        assert np.abs(f[c] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), c


def _modes231():
    return [(2, 3, 1, -1.0, 2.0 / 3.0, 0.0), (1, 2, 2, 0.6, 0.5, -0.8)]


def test_exact_modes_are_divergence_free_and_satisfy_maxwell():
    """Fourth-order staggered differences of the oracle's exact fields satisfy dE/dt = Z curl H,
    dH/dt = -(1/Z) curl E at interior points, with residual falling like h^4."""
    modes = _modes231()
    for m in modes:
        assert abs(m[0] * m[3] + m[1] * m[4] + m[2] * m[5]) < 1e-15
    Z = 1.4
    res = []
    for N in (16, 32):
        o = oracle.Oracle3D(N, 0.4, Z=Z)
        h, dt = 1.0 / N, 1e-3
        t = 0.3

        def F(tt):
            return o.exact(modes, tt, tt)

        fp, fm, fp2, fm2 = F(t + dt), F(t - dt), F(t + 2 * dt), F(t - 2 * dt)
        f0 = F(t)
        ddt = [(8 * (fp[c] - fm[c]) - (fp2[c] - fm2[c])) / (12 * dt) for c in range(6)]

        def D(u, axis, out_half):
            # fourth-order staggered derivative along axis ([z][y][x] array axis 2 - axis)
            u = np.moveaxis(u, 2 - axis, 0)
            if out_half:  # nodes -> half-nodes: out[q] at q+1/2 from u[q-1..q+2]
                d = (27 * (u[2:-1] - u[1:-2]) - (u[3:] - u[:-3])) / (24 * h)
                lo = 1
            else:  # half-nodes -> nodes: out[q] at node q from u[q-2..q+1]
                d = (27 * (u[2:-1] - u[1:-2]) - (u[3:] - u[:-3])) / (24 * h)
                lo = 2
            return np.moveaxis(d, 0, 2 - axis), lo

        worst, scale = 0.0, 0.0
        # dE_z/dt = Z (d_x H_y - d_y H_x) at E_z points (x_i, y_j, z_{k+1/2})
        dxhy, _ = D(f0[4], 0, False)   # H_y x-half -> x-node; result x index i from 2..N-2
        dyhx, _ = D(f0[3], 1, False)
        a = dxhy[:, 2:-2, :]           # [z][y][x]: trim y of dxhy to match
        b = dyhx[:, :, 2:-2]
        lhs = ddt[2][:, 2:-2, 2:-2]
        rhs = Z * (a - b)
        worst = max(worst, np.abs(lhs - rhs).max())
        scale = max(scale, np.abs(lhs).max())
        # dH_x/dt = -(1/Z)(d_y E_z - d_z E_y) at H_x points (x_i, y_{j+1/2}, z_{k+1/2})
        dyez, _ = D(f0[2], 1, True)    # E_z y-node -> y-half: half index 1..N-2
        dzey, _ = D(f0[1], 2, True)
        lhs = ddt[3][1:-1, 1:-1, :]
        rhs = -(1.0 / Z) * (dyez[1:-1, :, :] - dzey[:, 1:-1, :])
        worst = max(worst, np.abs(lhs - rhs).max())
        # Gauss: d_x E_x + d_y E_y + d_z E_z = 0 at nodes
        gx, _ = D(f0[0], 0, False)
        gy, _ = D(f0[1], 1, False)
        gz, _ = D(f0[2], 2, False)
        div = gx[2:-2, 2:-2, :] + gy[2:-2, :, 2:-2] + gz[:, 2:-2, 2:-2]
        worst = max(worst, np.abs(div).max())
        res.append(worst / scale)
    assert res[1] < 2e-3 and res[0] / res[1] > 10.0


def test_fourth_order_convergence_paper_closure():
    modes = _modes231()
    T = 0.25
    errs = []
    for N in (8, 16, 32):
        o = oracle.Oracle3D(N, 0.4)
        K = int(round(T / o.ht))
        f = o.init_modes(modes)
        o.run(f, K)
        errs.append(o.error(modes, K, f)[0])
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert rates[1] > 3.6, (errs, rates)


# --------------------------------------------------------------------------
# Diagnostics: discrete energy and Pade divergence of H in 3D

@pytest.mark.parametrize("closure", [CLOSURE_PAPER, CLOSURE_REFLECT])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_energy_and_divergence_reduce_to_2d(closure, axis):
    """For fields independent of one coordinate, the 3D energy and the norm of the 3D divergence
    equal those of the pinned 2D oracle on the cross-section (h^3 sums over N copies)."""
    N, r, Z = 9, 0.4, 1.3
    o2 = oracle.Oracle2D(N, r, Z=Z, closure=closure)
    o3 = oracle.Oracle3D(N, r, Z=Z, closure=closure)
    s2 = list(workloads.random_fields(N, seed=80 + axis))
    f, _ = _extrude(s2, N, axis)
    W2, W3 = o2.energy(*s2), o3.energy(f)
    assert abs(W3 - W2) <= 1e-12 * abs(W2)
    d2, d3 = o2.divergence(s2[1], s2[2])[0], o3.divergence(f)[0]
    assert abs(d3 - d2) <= 1e-12 * d2


def test_reflect_energy_and_divergence_conserved_3d():
    """REFLECT closure: the leapfrog invariant and the Pade divergence of H are conserved to
    round-off by the six-component step (random fields, far from divergence-free)."""
    N = 7
    o = oracle.Oracle3D(N, 0.45, Z=1.4, closure=CLOSURE_REFLECT)
    f = list(workloads.random_fields3(N, seed=5))
    W0 = o.energy(f)
    d0, div0 = o.divergence(f)
    assert d0 > 1.0
    for _ in range(8):
        o.step(f)
    assert abs(o.energy(f) - W0) < 1e-12 * W0
    d1, div1 = o.divergence(f)
    assert np.max(np.abs(div1 - div0)) < 1e-10 * np.max(np.abs(div0))


def test_paper_closure_energy_bounded_3d():
    """PAPER closure: W is not an exact invariant, but stays in a narrow band for cavity modes."""
    N = 16
    o = oracle.Oracle3D(N, 0.4, closure=CLOSURE_PAPER)
    f = o.init_modes([workloads.mode3(2, 3, 1, 1.0), workloads.mode3(1, 2, 2, 0.7)])
    W = [o.energy(f)]
    for _ in range(4):
        o.run(f, 8)
        W.append(o.energy(f))
    W = np.array(W)
    assert (W.max() - W.min()) / W[0] < 1e-3
