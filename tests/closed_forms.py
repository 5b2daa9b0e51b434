"""Closed forms that pin the oracle: operator symbols on the cavity-mode bases.

These are derived independently of the oracle's code, from the symbols of the
operators of the paper (App. A.1 Pade and D_2 matrices, Def. "def:operatorsP",
Eq. "eq:ell") acting on the sine / cosine bases of the staggered grids.  Under
the REFLECT closure every operator of the scheme is diagonal in these bases, so
a single cavity mode evolves by a 3x3 matrix per step (the recurrence of Sec. 4,
Eq. "eq:stab1").
"""
import math

import numpy as np

# Per-mode symbols of the operators (closed forms used to pin the oracle).
# For a cavity mode with indices (k_x, k_y), theta = pi k h; the sine / cosine
# bases of each staggered grid are eigenvectors of every operator under the
# REFLECT closure, so one step acts on the mode coefficients as a 3x3 matrix.

def pade_symbol(theta: float, h: float) -> float:
    """Magnitude d of the Pade derivative symbol: i (2/h) sin(theta/2) 24 / (22 + 2 cos theta)."""
    return (2.0 / h) * math.sin(theta / 2) * 24.0 / (22.0 + 2.0 * math.cos(theta))


def d2_symbol(theta: float, h: float) -> float:
    """Eigenvalue of D_2 on sin / cos(theta (j + 1/2)) bases: -(4/h^2) sin^2(theta/2)."""
    return -(4.0 / h ** 2) * math.sin(theta / 2) ** 2


def mode_step_matrix(N: int, r: float, kx: int, ky: int, Z: float = 1.0) -> np.ndarray:
    """Matrix of one full step on the coefficients (e, a, b) of
    E_z = e sin(tx i) sin(ty j), H_x = a sin(tx i) cos(ty (j+1/2)), H_y = b cos(tx (i+1/2)) sin(ty j),
    written from the symbols of D_2, Delta_h, P1, the filter and the Pade derivative."""
    h = 1.0 / N
    ht = r * h
    k2 = 24.0 / ht ** 2
    beta = 1.0 + k2 * h * h / 12.0
    tx, ty = math.pi * kx * h, math.pi * ky * h
    mx, my = -d2_symbol(tx, h), -d2_symbol(ty, h)  # eigenvalues of -D_xx, -D_yy (>= 0)
    filt = beta - (h * h / 12.0) * (mx + my)
    p1 = k2 * beta + mx + my - (h * h / 6.0) * mx * my
    g = k2 * filt / p1
    dx, dy = pade_symbol(tx, h), pade_symbol(ty, h)
    # Step 1: e' = e + ht Z g (dy a - dx b)
    S1 = np.array([[1.0, ht * Z * g * dy, -ht * Z * g * dx], [0, 1, 0], [0, 0, 1]])
    # Step 2: a' = a - (ht/Z) g dy e', b' = b + (ht/Z) g dx e'
    S2 = np.array([[1.0, 0, 0], [-(ht / Z) * g * dy, 1, 0], [(ht / Z) * g * dx, 0, 1]])
    return S2 @ S1


def mode_basis(N: int, kx: int, ky: int):
    """Basis fields (E_z, H_x, H_y) of the mode on the staggered grids."""
    h = 1.0 / N
    i_n = np.arange(N + 1)
    i_h = np.arange(N) + 0.5
    tx, ty = math.pi * kx * h, math.pi * ky * h
    ez = np.outer(np.sin(ty * i_n), np.sin(tx * i_n))
    hx = np.outer(np.cos(ty * i_h), np.sin(tx * i_n))
    hy = np.outer(np.sin(ty * i_n), np.cos(tx * i_h))
    ez[0, :] = ez[-1, :] = 0.0
    ez[:, 0] = ez[:, -1] = 0.0
    hx[:, 0] = hx[:, -1] = 0.0
    hy[0, :] = hy[-1, :] = 0.0
    return ez, hx, hy


def mode_step_matrix3(N: int, r: float, m: int, n: int, p: int, Z: float = 1.0) -> np.ndarray:
    """Matrix of one full 3D step on the coefficients (e_x, e_y, e_z, h_x, h_y, h_z) of the mode
    basis of mode_basis3 (sine on node axes, cosine on half-node axes), from the symbols of D_2,
    P1 (with Upsilon_h), the filter and the Pade derivatives; curl_h as printed in Sec. 3.4."""
    h = 1.0 / N
    ht = r * h
    k2 = 24.0 / ht ** 2
    beta = 1.0 + k2 * h * h / 12.0
    th = [math.pi * m * h, math.pi * n * h, math.pi * p * h]
    mu = [-d2_symbol(t, h) for t in th]
    filt = beta - (h * h / 12.0) * sum(mu)
    p1 = k2 * beta + sum(mu) - (h * h / 6.0) * (mu[0] * mu[1] + mu[1] * mu[2] + mu[2] * mu[0])
    g = k2 * filt / p1
    dx, dy, dz = (pade_symbol(t, h) for t in th)
    # d(half->node) cos -> -d sin, d(node->half) sin -> +d cos
    S1 = np.eye(6)
    S1[0, 4], S1[0, 5] = ht * Z * g * dz, -ht * Z * g * dy    # e_x += ht Z g (dz h_y - dy h_z)
    S1[1, 5], S1[1, 3] = ht * Z * g * dx, -ht * Z * g * dz    # e_y += ht Z g (dx h_z - dz h_x)
    S1[2, 3], S1[2, 4] = ht * Z * g * dy, -ht * Z * g * dx    # e_z += ht Z g (dy h_x - dx h_y)
    S2 = np.eye(6)
    c = ht * g / Z
    S2[3, 1], S2[3, 2] = c * dz, -c * dy                       # h_x += (ht/Z) g (dz e_y - dy e_z)
    S2[4, 2], S2[4, 0] = c * dx, -c * dz                       # h_y += (ht/Z) g (dx e_z - dz e_x)
    S2[5, 0], S2[5, 1] = c * dy, -c * dx                       # h_z += (ht/Z) g (dy e_x - dx e_y)
    return S2 @ S1


def mode_basis3(N: int, m: int, n: int, p: int):
    """Basis fields [z][y][x] of the six components for mode (m, n, p): on each axis a component
    carries sin(theta i) on nodes (Dirichlet axes) and cos(theta (i + 1/2)) on half-nodes."""
    h = 1.0 / N
    th = [math.pi * m * h, math.pi * n * h, math.pi * p * h]
    out = []
    for c in range(6):
        s = c % 3
        node_axes = [a != s for a in range(3)] if c < 3 else [a == s for a in range(3)]
        f1 = []
        for a in range(3):
            if node_axes[a]:
                v = np.sin(th[a] * np.arange(N + 1))
                v[0] = v[-1] = 0.0
            else:
                v = np.cos(th[a] * (np.arange(N) + 0.5))
            f1.append(v)
        out.append(np.einsum("k,j,i->kji", f1[2], f1[1], f1[0]))
    return out


def mode_step_matrix_tracked(N: int, r: float, kx: int, ky: int, Z: float = 1.0) -> np.ndarray:
    """One step of the tracked-Delta-E variant on the coefficients (e, a, b, q) of the mode basis
    (q: the tracked Delta E on the E_z basis): Step 1 as in mode_step_matrix, then
    q' = q + kappa^2 (e' - e) - Z kappa^2 h_tau (d_y a - d_x b) (Eq. "eq:mhe" with the unfiltered
    Pade curl), and Step 2 with G_E = beta e' + (h^2/12) q' (Eq. "eq:helm2")."""
    h = 1.0 / N
    ht = r * h
    k2 = 24.0 / ht ** 2
    beta = 1.0 + k2 * h * h / 12.0
    tx, ty = math.pi * kx * h, math.pi * ky * h
    mx, my = -d2_symbol(tx, h), -d2_symbol(ty, h)
    filt = beta - (h * h / 12.0) * (mx + my)
    p1 = k2 * beta + mx + my - (h * h / 6.0) * mx * my
    g = k2 * filt / p1
    dx, dy = pade_symbol(tx, h), pade_symbol(ty, h)
    S1 = np.eye(4)
    S1[0, 1], S1[0, 2] = ht * Z * g * dy, -ht * Z * g * dx
    # q' = q + k2 (e' - e) - Z k2 ht (dy a - dx b), with e' - e = ht Z g (dy a - dx b)
    c = k2 * ht * Z * (g - 1.0)
    S1[3, 1], S1[3, 2] = c * dy, -c * dx
    S2 = np.eye(4)
    w = ht * k2 / (Z * p1)  # H* = -(k2/Z) curl(G_E) / p1
    # G_E = beta e + (h^2/12) q
    S2[1, 0], S2[1, 3] = -w * dy * beta, -w * dy * h * h / 12.0
    S2[2, 0], S2[2, 3] = w * dx * beta, w * dx * h * h / 12.0
    return S2 @ S1


def mode_step_forced(N, r, m, n, Z, src_amp, w, step):
    """Affine per-mode step (M, f) of the scheme with the current source
    J_z = src_amp sin(m pi x) sin(n pi y) sin(w t) on the coefficients (e, a, b) of mode_basis:
    v_{step+1} = M v_step + f, with P(J) = -Z (kappa^2 - w^2) J at t^{n+1/2} added to Step 1 and
    curl d_t J at t^{n+1} to Step 2, both filtered with the exact Laplacian of the source."""
    h = 1.0 / N
    ht = r * h
    k2 = 24.0 / ht ** 2
    beta = 1.0 + k2 * h * h / 12.0
    tx, ty = math.pi * m * h, math.pi * n * h
    mx, my = -d2_symbol(tx, h), -d2_symbol(ty, h)
    filt = beta - (h * h / 12.0) * (mx + my)
    p1 = k2 * beta + mx + my - (h * h / 6.0) * mx * my
    g = k2 * filt / p1
    dx, dy = pade_symbol(tx, h), pade_symbol(ty, h)
    fj = beta - (h * h / 12.0) * math.pi ** 2 * (m * m + n * n)
    th, tn = (step + 0.5) * ht, (step + 1.0) * ht
    se = -Z * (k2 - w * w) * fj * src_amp * math.sin(w * th)
    shx = fj * src_amp * w * math.pi * n * math.cos(w * tn)
    shy = fj * src_amp * w * math.pi * m * math.cos(w * tn)
    S1 = np.array([[1.0, ht * Z * g * dy, -ht * Z * g * dx], [0, 1, 0], [0, 0, 1]])
    f1 = np.array([ht * se / p1, 0.0, 0.0])
    S2 = np.array([[1.0, 0, 0], [-(ht / Z) * g * dy, 1, 0], [(ht / Z) * g * dx, 0, 1]])
    f2 = np.array([0.0, ht * shx / p1, -ht * shy / p1])
    return S2 @ S1, S2 @ f1 + f2
