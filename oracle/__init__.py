"""FP64 CPU oracle of the compact fourth-order staggered Maxwell scheme (arXiv 2306.17263).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never uses it; the two share no code.

The arithmetic lives in ``maxwell_oracle.c`` (2D) and ``maxwell_oracle3d.c`` (3D)
(plain C, FP64, single thread),
compiled on demand with gcc into ``oracle/_build/liboracle.so``.  This module
only marshals numpy arrays to it.  Each wrapper names the passage of the paper
its C routine follows.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "maxwell_oracle.c"), os.path.join(_HERE, "maxwell_oracle3d.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

F_EZ, F_HX, F_HY = 0, 1, 2
CLOSURE_PAPER, CLOSURE_REFLECT = 0, 1
HALF_TO_NODE, NODE_TO_HALF = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no fast-math) if it is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS)
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            D = ctypes.POINTER(ctypes.c_double)
            V = ctypes.c_void_p
            L.or2d_setup.argtypes = [V, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
            L.or2d_set_cg.argtypes = [V, ctypes.c_double, ctypes.c_int]
            L.or2d_field_size.argtypes = [V, ctypes.c_int]
            L.or2d_field_size.restype = ctypes.c_int
            L.or_pade_line.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, D, D]
            L.or_pade_matvec24.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D]
            for name in ("or2d_laplacian", "or2d_filter", "or2d_p1_apply", "or2d_p2_apply"):
                getattr(L, name).argtypes = [V, ctypes.c_int, D, D]
            L.or2d_p1_solve_cg.argtypes = [V, ctypes.c_int, D, D]
            L.or2d_p1_solve_cg.restype = ctypes.c_int
            L.or2d_curl_h_to_e.argtypes = [V, D, D, D]
            L.or2d_curl_e_to_h.argtypes = [V, D, D, D]
            L.or2d_h_increment.argtypes = [V, D, D, D]
            L.or2d_step.argtypes = [V, D, D, D]
            L.or2d_yee_step.argtypes = [V, D, D, D]
            L.or2d_exact.argtypes = [V, D, ctypes.c_int, ctypes.c_double, ctypes.c_double, D, D, D]
            L.or2d_error.argtypes = [V, D, ctypes.c_int, ctypes.c_double, ctypes.c_double, D, D, D, D]
            L.or2d_energy.argtypes = [V, D, D, D]
            L.or2d_energy.restype = ctypes.c_double
            L.or2d_divergence.argtypes = [V, D, D, D]
            L.or2d_divergence.restype = ctypes.c_double
            L.or2d_run.argtypes = [V, D, D, D, ctypes.c_int, D, ctypes.c_int]
            L.or2d_run.restype = ctypes.c_double
            L.or2d_cg_iters_total.argtypes = [V]
            L.or2d_cg_iters_total.restype = ctypes.c_long
            L.or2d_cg_solves.argtypes = [V]
            L.or2d_cg_solves.restype = ctypes.c_long
            L.or2d_sizeof.restype = ctypes.c_int
            L.or_pade_line_T.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, D, D]
            L.or2d_curl_h_to_e_T.argtypes = [V, D, D, D]
            L.or2d_curl_e_to_h_T.argtypes = [V, D, D, D]
            L.or2d_step_T.argtypes = [V, D, D, D]
            L.or2d_taylor_h.argtypes = [V, D, D, D]
            L.or2d_taylor_h_T.argtypes = [V, D, D, D]
            L.or2d_misfit_grad.argtypes = [V, D, D, ctypes.c_int, D]
            L.or2d_misfit_grad.restype = ctypes.c_double
            L.or_nc_line.argtypes = [ctypes.c_int, ctypes.c_double, D, D]
            L.or2d_nc_step.argtypes = [V, D, D, D]
            L.or2d_step_tracked.argtypes = [V, D, D, D, D]
            L.or2d_step_src.argtypes = [V, D, D, D, D, ctypes.c_int, ctypes.c_long]
            L.or2d_exact_driven.argtypes = [V, D, ctypes.c_int, ctypes.c_double, ctypes.c_double, D, D, D]
            L.or2d_step_src_xy.argtypes = [V, D, D, D, D, ctypes.c_int, ctypes.c_long]
            L.or2d_wall_ghosts.argtypes = [V, D, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           D, D, D, D]
            L.or2d_ge_wall.argtypes = [V, D, ctypes.c_int, ctypes.c_double, D]
            L.or2d_p1_ghost_shift.argtypes = [V, ctypes.c_int, D, D, D]
            PP = ctypes.POINTER(ctypes.c_void_p)
            L.or3d_sizeof.restype = ctypes.c_int
            L.or3d_setup.argtypes = [V, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
            L.or3d_set_cg.argtypes = [V, ctypes.c_double, ctypes.c_int]
            L.or3d_bc.argtypes = [ctypes.c_int, ctypes.c_int]
            L.or3d_bc.restype = ctypes.c_int
            for name in ("or3d_laplacian", "or3d_filter", "or3d_p1_apply"):
                getattr(L, name).argtypes = [V, ctypes.c_int, D, D]
            L.or3d_p1_solve_cg.argtypes = [V, ctypes.c_int, D, D]
            L.or3d_p1_solve_cg.restype = ctypes.c_int
            L.or3d_curl_h_to_e.argtypes = [V, PP, PP]
            L.or3d_curl_e_to_h.argtypes = [V, PP, PP]
            L.or3d_step.argtypes = [V, PP]
            L.or3d_exact.argtypes = [V, D, ctypes.c_int, ctypes.c_double, ctypes.c_double, PP]
            L.or3d_error.argtypes = [V, D, ctypes.c_int, ctypes.c_double, ctypes.c_double, PP, D]
            L.or3d_energy.argtypes = [V, PP]
            L.or3d_energy.restype = ctypes.c_double
            L.or3d_divergence.argtypes = [V, PP, D]
            L.or3d_divergence.restype = ctypes.c_double
            L.or3d_cg_iters_total.argtypes = [V]
            L.or3d_cg_iters_total.restype = ctypes.c_long
            L.or3d_cg_solves.argtypes = [V]
            L.or3d_cg_solves.restype = ctypes.c_long
            L.or3d_step_src.argtypes = [V, PP, D, ctypes.c_int, ctypes.c_long]
            L.or3d_exact_driven.argtypes = [V, D, ctypes.c_int, ctypes.c_double, ctypes.c_double, PP]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pade_line(f: np.ndarray, h: float, closure: int = CLOSURE_PAPER, kind: int = HALF_TO_NODE) -> np.ndarray:
    """Pade first derivative of one line (App. A.1, Eq. "eq:lhs"): A f' = D1 f / h, len(f') = len(f) - 1."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    M = f.size - 1
    out = np.zeros(M)
    lib().or_pade_line(M, closure, kind, h, _p(f), _p(out))
    return out


def pade_line_T(g: np.ndarray, h: float, closure: int = CLOSURE_PAPER, kind: int = HALF_TO_NODE) -> np.ndarray:
    """Transpose of pade_line: D1^T A^{-T} g / h, len(out) = len(g) + 1."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(g.size + 1)
    lib().or_pade_line_T(g.size, closure, kind, h, _p(g), _p(out))
    return out


def nc_line(f: np.ndarray, h: float) -> np.ndarray:
    """Fourth-order staggered first derivative of the NC comparator (Sec. 5.2, stencil K4 with
    a = 0, one-sided fourth-order differences at the ends): len(out) = len(f) - 1."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(f.size - 1)
    lib().or_nc_line(f.size, h, _p(f), _p(out))
    return out


def pade_matvec24(y: np.ndarray, closure: int = CLOSURE_PAPER, kind: int = HALF_TO_NODE) -> np.ndarray:
    """Apply 24 A (the left-hand matrix of Eq. "eq:lhs") to y."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros_like(y)
    lib().or_pade_matvec24(y.size, closure, kind, _p(y), _p(out))
    return out


class Oracle2D:
    """2D TM_z grid of the scheme (Sec. 5: E_z, H_x, H_y on the unit square, PEC walls)."""

    def __init__(self, N: int, r: float, Z: float = 1.0, closure: int = CLOSURE_PAPER):
        L = lib()
        self._buf = ctypes.create_string_buffer(L.or2d_sizeof())
        self.g = ctypes.cast(self._buf, ctypes.c_void_p)
        L.or2d_setup(self.g, int(N), float(r), float(Z), int(closure))
        self.N, self.r, self.Z, self.closure = int(N), float(r), float(Z), int(closure)
        self.h = 1.0 / N
        self.ht = r * self.h
        self.kappa2 = 24.0 / self.ht ** 2
        self.beta = 1.0 + self.kappa2 * self.h ** 2 / 12.0
        self.c1 = self.kappa2 * self.beta

    # shapes (rows = y, cols = x), Eq. "eq:meshes" restricted to TM_z
    def shape(self, f: int):
        N = self.N
        return {F_EZ: (N + 1, N + 1), F_HX: (N, N + 1), F_HY: (N + 1, N)}[f]

    def zeros(self, f: int) -> np.ndarray:
        return np.zeros(self.shape(f))

    def set_cg(self, tol: float, maxit: int = 200):
        lib().or2d_set_cg(self.g, tol, maxit)

    def _unary(self, name, f, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = self.zeros(f)
        getattr(lib(), name)(self.g, f, _p(u), _p(out))
        return out

    def laplacian(self, f, u):
        """Delta_h = D_xx + D_yy with the field's Dirichlet / even-ghost Neumann boundaries."""
        return self._unary("or2d_laplacian", f, u)

    def filter(self, f, u):
        """G = (1 + kappa^2 h^2 / 12) u + (h^2/12) Delta_h u (right side of Eq. "eq:ell")."""
        return self._unary("or2d_filter", f, u)

    def p1(self, f, x):
        """P1 x (Definition "def:operatorsP")."""
        return self._unary("or2d_p1_apply", f, x)

    def p2(self, f, x):
        """P2 x (Definition "def:operatorsP")."""
        return self._unary("or2d_p2_apply", f, x)

    def p1_solve(self, f, b):
        """CG solve of P1 x = b (Sec. 3.2); returns (x, iterations)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = self.zeros(f)
        it = lib().or2d_p1_solve_cg(self.g, f, _p(b), _p(x))
        return x, it

    def curl_h_to_e(self, Gx, Gy):
        """R_E = kappa^2 Z (delta_x G_y - delta_y G_x) (Step 1, Sec. 3.4)."""
        Gx = np.ascontiguousarray(Gx, dtype=np.float64)
        Gy = np.ascontiguousarray(Gy, dtype=np.float64)
        R = self.zeros(F_EZ)
        lib().or2d_curl_h_to_e(self.g, _p(Gx), _p(Gy), _p(R))
        return R

    def curl_e_to_h(self, GE):
        """(R_x, R_y) = (kappa^2/Z) (-delta_y G_E, delta_x G_E) (Step 2, Sec. 3.4)."""
        GE = np.ascontiguousarray(GE, dtype=np.float64)
        Rx, Ry = self.zeros(F_HX), self.zeros(F_HY)
        lib().or2d_curl_e_to_h(self.g, _p(GE), _p(Rx), _p(Ry))
        return Rx, Ry

    def h_increment(self, ez):
        ez = np.ascontiguousarray(ez, dtype=np.float64)
        hxs, hys = self.zeros(F_HX), self.zeros(F_HY)
        lib().or2d_h_increment(self.g, _p(ez), _p(hxs), _p(hys))
        return hxs, hys

    def step(self, ez, hx, hy):
        """One full step in place (Sec. 3.4 Step 1 then Step 2)."""
        lib().or2d_step(self.g, _p(ez), _p(hx), _p(hy))

    def yee_step(self, ez, hx, hy):
        """One plain second-order Yee step in place (Sec. 5.2, stencil S with c = 1)."""
        lib().or2d_yee_step(self.g, _p(ez), _p(hx), _p(hy))

    def step_tracked(self, ez, hx, hy, de):
        """One step of the tracked-Delta-E variant in place (Sec. 3.4 as printed: DE advanced by
        Eq. "eq:mhe", Step 2 filtered with it as in Eq. "eq:helm2")."""
        lib().or2d_step_tracked(self.g, _p(ez), _p(hx), _p(hy), _p(de))

    @staticmethod
    def _src(src):
        a = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, 4))
        return a, a.shape[0]

    def step_src(self, ez, hx, hy, src, n):
        """Step n (E^n -> E^{n+1}) with current sources J_z = a sin(m pi x) sin(n pi y) sin(w t),
        rows (m, n, a, w): P(J) and curl d_t J added to the right-hand sides of Eq. "eq:mh"."""
        s, ns = self._src(src)
        lib().or2d_step_src(self.g, _p(ez), _p(hx), _p(hy), _p(s), ns, int(n))

    def exact_driven(self, src, tE, tH):
        """Exact particular solution driven by the sources (E at tE, H at tH)."""
        s, ns = self._src(src)
        ez, hx, hy = self.zeros(F_EZ), self.zeros(F_HX), self.zeros(F_HY)
        lib().or2d_exact_driven(self.g, _p(s), ns, tE, tH, _p(ez), _p(hx), _p(hy))
        return ez, hx, hy

    # -- sources with sine or cosine profiles, nonzero on the walls (Sec. 3.3, Method 2) --
    @staticmethod
    def _src_xy(src):
        a = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, 6))
        return a, a.shape[0]

    def step_src_xy(self, ez, hx, hy, src, n):
        """Step n with sources J_z = a X(m pi x) Y(n pi y) sin(w t), rows (m, n, a, w, px, py),
        X = sin (px = 0) or cos (px = 1): the inhomogeneous ghosts of the H filter and the H solves,
        and G_E on the walls from d_t J (PAPER closure)."""
        s, ns = self._src_xy(src)
        lib().or2d_step_src_xy(self.g, _p(ez), _p(hx), _p(hy), _p(s), ns, int(n))

    def wall_ghosts(self, src, t0, t1, diff):
        """Ghost data (g_x_lo, g_x_hi, g_y_lo, g_y_hi): H_x by column on y = 0, 1 and H_y by row on
        x = 0, 1; the data of H at t1 (diff = 0) or of (H(t1) - H(t0)) / h_tau (diff = 1)."""
        s, ns = self._src_xy(src)
        out = [np.zeros(self.N + 1) for _ in range(4)]
        lib().or2d_wall_ghosts(self.g, _p(s), ns, float(t0), float(t1), int(diff), *[_p(a) for a in out])
        return out

    def ge_wall(self, src, t):
        """E_z-shaped array whose boundary nodes hold G_E = (h^2/12) Z d_t J_z at time t."""
        s, ns = self._src_xy(src)
        ge = self.zeros(F_EZ)
        lib().or2d_ge_wall(self.g, _p(s), ns, float(t), _p(ge))
        return ge

    def p1_ghost_shift(self, f, glo, ghi):
        """P1 (of H_x or H_y) applied to zero with the given ghost data: the affine part."""
        c = self.zeros(f)
        lib().or2d_p1_ghost_shift(self.g, int(f), _p(np.ascontiguousarray(glo, dtype=np.float64)),
                                  _p(np.ascontiguousarray(ghi, dtype=np.float64)), _p(c))
        return c

    def exact_manufactured(self, m, n, A, w, tE, tH):
        """The manufactured solution of `manufactured_sources` on this grid (E at tE, H at tH)."""
        N, h = self.N, self.h
        xn = np.arange(N + 1) * h
        xh = (np.arange(N) + 0.5) * h
        ez = manufactured_field(m, n, A, w, self.Z, F_EZ, xn[None, :], xn[:, None], tE)
        hx = manufactured_field(m, n, A, w, self.Z, F_HX, xn[None, :], xh[:, None], tH)
        hy = manufactured_field(m, n, A, w, self.Z, F_HY, xh[None, :], xn[:, None], tH)
        return [np.ascontiguousarray(np.broadcast_to(a, self.shape(f)), dtype=np.float64)
                for f, a in ((F_EZ, ez), (F_HX, hx), (F_HY, hy))]

    def nc_step(self, ez, hx, hy):
        """One step of the non-compact fourth-order comparator NC in place (Sec. 5.2, K4, a = 0)."""
        lib().or2d_nc_step(self.g, _p(ez), _p(hx), _p(hy))

    @staticmethod
    def _modes(modes):
        m = np.ascontiguousarray(np.asarray(modes, dtype=np.float64).reshape(-1, 3))
        return m, m.shape[0]

    def exact(self, modes, tE, tH):
        """Exact cavity-mode superposition (Eq. "eq:data"); modes rows are (k_x, k_y, amplitude)."""
        m, nm = self._modes(modes)
        ez, hx, hy = self.zeros(F_EZ), self.zeros(F_HX), self.zeros(F_HY)
        lib().or2d_exact(self.g, _p(m), nm, tE, tH, _p(ez), _p(hx), _p(hy))
        return ez, hx, hy

    def init_modes(self, modes):
        """E^0 and H^{1/2} from the closed form (Sec. 5.1)."""
        return self.exact(modes, 0.0, 0.5 * self.ht)

    def error(self, modes, n, ez, hx, hy):
        """(L2 abs, L2 rel, max abs, sum |err|) of (E^n, H^{n+1/2}) against the exact modes."""
        m, nm = self._modes(modes)
        out = np.zeros(4)
        lib().or2d_error(self.g, _p(m), nm, n * self.ht, (n + 0.5) * self.ht, _p(ez), _p(hx), _p(hy), _p(out))
        return out

    def energy(self, ez, hx, hy):
        """W^n = Z^-1 ||E^n||^2 + Z <H^{n-1/2}, H^{n+1/2}> (h^2-weighted)."""
        return lib().or2d_energy(self.g, _p(ez), _p(hx), _p(hy))

    def divergence(self, hx, hy):
        """(||div_h H||_h, div field) with the node->half-node Pade derivatives."""
        div = np.zeros((self.N, self.N))
        n = lib().or2d_divergence(self.g, _p(hx), _p(hy), _p(div))
        return n, div

    def run(self, ez, hx, hy, nsteps, modes=None):
        """Run nsteps in place; with modes, return the mean absolute error of Sec. 5.1."""
        if modes is None:
            lib().or2d_run(self.g, _p(ez), _p(hx), _p(hy), int(nsteps), None, 0)
            return None
        m, nm = self._modes(modes)
        acc = lib().or2d_run(self.g, _p(ez), _p(hx), _p(hy), int(nsteps), _p(m), nm)
        return acc / (3.0 * nsteps * self.N ** 2)

    def cg_stats(self):
        L = lib()
        return L.or2d_cg_iters_total(self.g), L.or2d_cg_solves(self.g)

    # -- adjoint (transpose) of the step, the Taylor initialisation and the misfit gradient --
    def step_T(self, lez, lhx, lhy):
        """Transpose of one full step, in place on the adjoint state (level n+1 -> n)."""
        lib().or2d_step_T(self.g, _p(lez), _p(lhx), _p(lhy))

    def taylor_h(self, ez0):
        """H^{1/2} from E^0 with H^0 = 0 by the Taylor series of Sec. 5.1 (Eq. "talorh")."""
        ez0 = np.ascontiguousarray(ez0, dtype=np.float64)
        hx, hy = self.zeros(F_HX), self.zeros(F_HY)
        lib().or2d_taylor_h(self.g, _p(ez0), _p(hx), _p(hy))
        return hx, hy

    def taylor_h_T(self, lhx, lhy):
        lhx = np.ascontiguousarray(lhx, dtype=np.float64)
        lhy = np.ascontiguousarray(lhy, dtype=np.float64)
        out = self.zeros(F_EZ)
        lib().or2d_taylor_h_T(self.g, _p(lhx), _p(lhy), _p(out))
        return out

    def misfit_grad(self, ez0, target, K, grad=True):
        """L = (1/2) h^2 sum (E_z^K - target)^2 from (E^0, Taylor H^{1/2}) and dL/dE^0 (interior)."""
        ez0 = np.ascontiguousarray(ez0, dtype=np.float64)
        target = np.ascontiguousarray(target, dtype=np.float64)
        g = self.zeros(F_EZ) if grad else None
        L = lib().or2d_misfit_grad(self.g, _p(ez0), _p(target), int(K), _p(g) if grad else None)
        return (L, g) if grad else L


def manufactured_field(m, n, A, w, Z, comp, x, y, t):
    """A closed-form PEC solution driven by a current that does not vanish on the walls:
        E_z = A cos(w t) P,  P = sin^2(m pi x) sin^2(n pi y),
        H   = (A sin(w t) / (Z w)) (-d_y P, d_x P)          (Faraday's law, H = 0 at t = 0),
        J_z = (A sin(w t) / (Z w)) (Delta P + w^2 P)         (Ampere's law, d_t E = Z (curl H - J)).
    E_z and H.n vanish on the walls; d_n H_t = -/+ J_z does not.  Evaluated at any (x, y), inside or
    outside the square."""
    pi = np.pi
    sx, sy = np.sin(m * pi * x), np.sin(n * pi * y)
    if comp == F_EZ:
        return A * np.cos(w * t) * sx ** 2 * sy ** 2
    c = A * np.sin(w * t) / (Z * w)
    if comp == F_HX:
        return -c * sx ** 2 * (n * pi * np.sin(2 * n * pi * y))
    return c * (m * pi * np.sin(2 * m * pi * x)) * sy ** 2


def manufactured_current(m, n, A, w, Z, x, y, t):
    """J_z of `manufactured_field`, from its definition (Delta P written out term by term)."""
    pi = np.pi
    P = np.sin(m * pi * x) ** 2 * np.sin(n * pi * y) ** 2
    lapP = (2 * (m * pi) ** 2 * np.cos(2 * m * pi * x) * np.sin(n * pi * y) ** 2
            + 2 * (n * pi) ** 2 * np.sin(m * pi * x) ** 2 * np.cos(2 * n * pi * y))
    return A * np.sin(w * t) / (Z * w) * (lapP + w * w * P)


def manufactured_sources(m, n, A, w, Z):
    """Rows (m, n, a, w, px, py) whose sum is J_z of `manufactured_field`: with
    sin^2 = (1 - cos 2.)/2 the current is (A sin(w t) / (4 Z w)) times
        w^2 + (4 m^2 pi^2 - w^2) cos(2 m pi x) + (4 n^2 pi^2 - w^2) cos(2 n pi y)
          + (w^2 - 4 pi^2 (m^2 + n^2)) cos(2 m pi x) cos(2 n pi y)."""
    pi2, c = np.pi ** 2, A / (4.0 * Z * w)
    return [(0, 0, c * w * w, w, 1, 1),
            (2 * m, 0, c * (4 * m * m * pi2 - w * w), w, 1, 1),
            (0, 2 * n, c * (4 * n * n * pi2 - w * w), w, 1, 1),
            (2 * m, 2 * n, c * (w * w - 4 * pi2 * (m * m + n * n)), w, 1, 1)]


E_X, E_Y, E_Z, H_X, H_Y, H_Z = range(6)


def _pp(arrs):
    for a in arrs:
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])


class Oracle3D:
    """3D grid of the scheme: six components on the staggered unit cube (Eq. "eq:meshes"),
    PEC walls, boundary types of Table "tab:bc".  Arrays are [z][y][x]."""

    def __init__(self, N: int, r: float, Z: float = 1.0, closure: int = CLOSURE_PAPER):
        L = lib()
        self._buf = ctypes.create_string_buffer(L.or3d_sizeof())
        self.g = ctypes.cast(self._buf, ctypes.c_void_p)
        L.or3d_setup(self.g, int(N), float(r), float(Z), int(closure))
        self.N, self.r, self.Z, self.closure = int(N), float(r), float(Z), int(closure)
        self.h = 1.0 / N
        self.ht = r * self.h
        self.kappa2 = 24.0 / self.ht ** 2
        self.beta = 1.0 + self.kappa2 * self.h ** 2 / 12.0
        self.c1 = self.kappa2 * self.beta

    @staticmethod
    def bc(c: int, axis: int) -> int:
        """0 = Dirichlet (nodes, wall zeros stored), 1 = Neumann (half-nodes, even ghosts)."""
        return lib().or3d_bc(c, axis)

    def shape(self, c: int):
        """(nz, ny, nx) of component c."""
        d = [self.N + 1 if self.bc(c, a) == 0 else self.N for a in range(3)]
        return d[2], d[1], d[0]

    def zeros(self, c: int) -> np.ndarray:
        return np.zeros(self.shape(c))

    def fields(self):
        return [self.zeros(c) for c in range(6)]

    def set_cg(self, tol: float, maxit: int = 200):
        lib().or3d_set_cg(self.g, tol, maxit)

    def _unary(self, name, c, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = self.zeros(c)
        getattr(lib(), name)(self.g, c, _p(u), _p(out))
        return out

    def laplacian(self, c, u):
        """Delta_h = D_xx + D_yy + D_zz with the component's boundary types."""
        return self._unary("or3d_laplacian", c, u)

    def filter(self, c, u):
        """G = (1 + kappa^2 h^2/12) u + (h^2/12) Delta_h u (right side of Eq. "eq:ell")."""
        return self._unary("or3d_filter", c, u)

    def p1(self, c, x):
        """P1 x = -(Delta_h + (h^2/6) Upsilon_h) x + c1 x (Definition "def:operatorsP")."""
        return self._unary("or3d_p1_apply", c, x)

    def p1_solve(self, c, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = self.zeros(c)
        it = lib().or3d_p1_solve_cg(self.g, c, _p(b), _p(x))
        return x, it

    def curl_h_to_e(self, G):
        """R_E = kappa^2 Z curl_h G_H (Step 1, Sec. 3.4); G = filtered (H_x, H_y, H_z)."""
        G = [np.ascontiguousarray(a, dtype=np.float64) for a in G]
        R = [self.zeros(c) for c in range(3)]
        lib().or3d_curl_h_to_e(self.g, _pp(G), _pp(R))
        return R

    def curl_e_to_h(self, G):
        """R_H = -(kappa^2/Z) curl_h G_E (Step 2, Sec. 3.4); G = filtered (E_x, E_y, E_z)."""
        G = [np.ascontiguousarray(a, dtype=np.float64) for a in G]
        R = [self.zeros(c) for c in range(3, 6)]
        lib().or3d_curl_e_to_h(self.g, _pp(G), _pp(R))
        return R

    def step(self, f):
        """One full step in place on f = [E_x, E_y, E_z, H_x, H_y, H_z] (Sec. 3.4)."""
        lib().or3d_step(self.g, _pp(f))

    def run(self, f, nsteps):
        for _ in range(int(nsteps)):
            self.step(f)

    @staticmethod
    def _modes(modes):
        m = np.ascontiguousarray(np.asarray(modes, dtype=np.float64).reshape(-1, 6))
        return m, m.shape[0]

    def exact(self, modes, tE, tH):
        """Exact cavity modes; rows (m, n, p, A_x, A_y, A_z) with A . (m, n, p) = 0."""
        m, nm = self._modes(modes)
        f = self.fields()
        lib().or3d_exact(self.g, _p(m), nm, tE, tH, _pp(f))
        return f

    def init_modes(self, modes):
        return self.exact(modes, 0.0, 0.5 * self.ht)

    def error(self, modes, n, f):
        """(L2 abs, L2 rel, max abs, sum |err|) of (E^n, H^{n+1/2}) against the exact modes."""
        m, nm = self._modes(modes)
        out = np.zeros(4)
        lib().or3d_error(self.g, _p(m), nm, n * self.ht, (n + 0.5) * self.ht, _pp(f), _p(out))
        return out

    def energy(self, f):
        """W^n = Z^-1 ||E^n||^2 + Z <H^{n-1/2}, H^{n+1/2}> (h^3-weighted) of the six components."""
        return lib().or3d_energy(self.g, _pp(f))

    def divergence(self, f):
        """(||div_h H||_h, div field on the N^3 cell centres) with node->half-node Pade derivatives."""
        div = np.zeros((self.N, self.N, self.N))
        nrm = lib().or3d_divergence(self.g, _pp(f), _p(div))
        return nrm, div

    def cg_stats(self):
        L = lib()
        return L.or3d_cg_iters_total(self.g), L.or3d_cg_solves(self.g)

    @staticmethod
    def _src3(src):
        s = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, 7))
        return s, s.shape[0]

    def step_src(self, f, src, n):
        """Step n in place with current sources, rows (m, n, p, a_x, a_y, a_z, w): divergence-free
        driven modes J = (a_x cos sin sin, a_y sin cos sin, a_z sin sin cos) sin(w t)."""
        s, ns = self._src3(src)
        lib().or3d_step_src(self.g, _pp(f), _p(s), ns, int(n))

    def exact_driven(self, src, tE, tH):
        """The exact driven solution of those sources (E at tE, H at tH)."""
        s, ns = self._src3(src)
        f = self.fields()
        lib().or3d_exact_driven(self.g, _p(s), ns, tE, tH, _pp(f))
        return f
