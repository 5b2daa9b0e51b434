"""GB300 (sm_103a) implementation of the compact fourth-order staggered scheme for the
first-order Maxwell equations (Versano, Turkel & Tsynkov, arXiv 2306.17263).

This module is a thin ctypes binding of ``include/maxwell4.h``: it marshals arguments
and raises on non-zero status codes.  Every step of the scheme runs in the CUDA kernels of
``libmaxwell4.so``; there is no CPU path.  If the library cannot be built or loaded,
importing the binding's entry points raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Grid", "Batch", "MaxwellError", "load", "lib_path", "FP64", "FP32_REFINED", "CLOSURE_PAPER", "CLOSURE_REFLECT",
           "SCHEME_C4", "SCHEME_YEE2", "SCHEME_NC4", "SCHEME_C4_DE", "OPS", "stability_limit"]

FP64, FP32_REFINED = 0, 1
CLOSURE_PAPER, CLOSURE_REFLECT = 0, 1
SCHEME_C4, SCHEME_YEE2, SCHEME_NC4, SCHEME_C4_DE = 0, 1, 2, 3
SOLVER_RICHARDSON, SOLVER_TRANSFORM_TC = 0, 1
OPS = {
    "filter_ez": 0, "filter_hx": 1, "filter_hy": 2, "curl_he": 3, "curl_eh": 4,
    "p1_ez": 5, "p1_hx": 6, "p1_hy": 7, "p1solve_ez": 8, "p1solve_hx": 9, "p1solve_hy": 10,
}
STATUS = {0: "MS_OK", -1: "MS_EINVAL", -2: "MS_ECFL", -3: "MS_ENOMEM", -4: "MS_ECUDA", -5: "MS_ETIMEOUT",
          -6: "MS_ENOTCONV", -7: "MS_EUNSUPPORTED"}


class MaxwellError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("z_imp", ctypes.c_double), ("r", ctypes.c_double),
                ("precision", ctypes.c_int), ("closure", ctypes.c_int), ("scheme", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class _Mode(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("amp", ctypes.c_double)]


class _Source(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("amp", ctypes.c_double), ("omega", ctypes.c_double)]


class _SourceXY(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("cos_x", ctypes.c_int), ("cos_y", ctypes.c_int),
                ("amp", ctypes.c_double), ("omega", ctypes.c_double)]


class _Source3(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("p", ctypes.c_int), ("ax", ctypes.c_double),
                ("ay", ctypes.c_double), ("az", ctypes.c_double), ("omega", ctypes.c_double)]


class _Mode3(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("p", ctypes.c_int), ("ax", ctypes.c_double),
                ("ay", ctypes.c_double), ("az", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Build (in-tree, if stale) and load libmaxwell4.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = ctypes.CDLL(path)
        V, I, D, L_ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
        PD = ctypes.POINTER(ctypes.c_double)
        PPD = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "ms_create_grid": [ctypes.POINTER(_Desc), ctypes.POINTER(V)],
            "ms_destroy": [V],
            "ms_init_modes": [V, ctypes.POINTER(_Mode), I],
            "ms_set_fields": [V, PPD, L_],
            "ms_get_fields": [V, PPD],
            "ms_set_fields_device": [V, PPD, L_],
            "ms_get_fields_device": [V, PPD],
            "ms_step": [V],
            "ms_run": [V, L_],
            "ms_sync": [V],
            "ms_get_step": [V, ctypes.POINTER(L_)],
            "ms_energy": [V, PD],
            "ms_divergence": [V, PD],
            "ms_error_vs_exact": [V, ctypes.POINTER(_Mode), I, PD, PD, PD, PD],
            "ms_apply_op": [V, I, PPD, PPD],
            "ms_launches_per_step": [V, ctypes.POINTER(I)],
            "ms_stability_limit": [I, PD],
            "ms_solver_sweeps": [I, D, I, D, ctypes.POINTER(I)],
            "ms_set_solver": [V, I],
            "ms_set_adjoint_precision": [V, I],
            "ms_set_sources3": [V, ctypes.POINTER(_Source3), I],
            "ms_init_driven3": [V, ctypes.POINTER(_Source3), I],
            "ms_batch_set_plan": [V, ctypes.POINTER(I)],
            "ms_batch_get_plan": [V, ctypes.POINTER(I)],
            "ms_batch_autotune": [V, I, ctypes.POINTER(I), ctypes.POINTER(I)],
            "ms_autotune_cache_get": [ctypes.c_char_p, ctypes.POINTER(I), ctypes.POINTER(I)],
            "ms_autotune_cache_put": [ctypes.c_char_p, ctypes.POINTER(I)],
            "ms_autotune_cache_clear": [],
            "ms_transform_solve3": [V, I, V, V],
            "ms_create_batch": [ctypes.POINTER(_Desc), ctypes.POINTER(I), I, ctypes.POINTER(V)],
            "ms_batch_destroy": [V],
            "ms_batch_init_modes": [V, I, ctypes.POINTER(_Mode), I],
            "ms_batch_set_fields": [V, I, PPD, L_],
            "ms_batch_get_fields": [V, I, PPD],
            "ms_batch_step": [V],
            "ms_batch_run": [V, L_],
            "ms_batch_sync": [V],
            "ms_batch_error_vs_exact": [V, I, ctypes.POINTER(_Mode), I, PD, PD, PD, PD],
            "ms_batch_info": [V, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(I)],
            "ms_step_profiled": [V, I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(I), PD, ctypes.POINTER(I)],
            "ms_init_modes3": [V, ctypes.POINTER(_Mode3), I],
            "ms_save": [V, ctypes.c_char_p],
            "ms_load": [V, ctypes.c_char_p],
            "ms_set_sources": [V, ctypes.POINTER(_Source), I],
            "ms_set_sources_xy": [V, ctypes.POINTER(_SourceXY), I],
            "ms_init_driven": [V, ctypes.POINTER(_Source), I],
            "ms_error_vs_driven": [V, ctypes.POINTER(_Source), I, PD, PD, PD, PD],
            "ms_error_vs_exact3": [V, ctypes.POINTER(_Mode3), I, PD, PD, PD, PD],
            "ms_taylor_init": [V, V],
            "ms_taylor_init_device": [V, V],
            "ms_taylor_init_T": [V, V, V, V],
            "ms_adjoint_run": [V, L_, V, V],
            "ms_adjoint_run_device": [V, L_, V, V],
            "ms_adjoint_steps": [V, L_, PPD],
            "ms_adjoint_steps_device": [V, L_, PPD],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = I
        L.ms_kernel_kind_name.argtypes = [I]
        L.ms_kernel_kind_name.restype = ctypes.c_char_p
        L.ms_last_error.argtypes = []
        L.ms_last_error.restype = ctypes.c_char_p
        L.ms_debug_fail_alloc.argtypes = [I]
        L.ms_debug_fail_alloc.restype = I
        L.ms_debug_live_allocs.argtypes = []
        L.ms_debug_live_allocs.restype = ctypes.c_long
        _lib = L
        return L


def _check(status: int):
    if status != 0:
        raise MaxwellError(status, load().ms_last_error().decode())


def _modes(modes):
    modes = list(modes)
    arr = (_Mode * max(1, len(modes)))()
    for k, (m, n, a) in enumerate(modes):
        arr[k].m, arr[k].n, arr[k].amp = int(m), int(n), float(a)
    return arr, len(modes)


def _modes3(modes):
    modes = list(modes)
    arr = (_Mode3 * max(1, len(modes)))()
    for k, (m, n, p, ax, ay, az) in enumerate(modes):
        arr[k].m, arr[k].n, arr[k].p = int(m), int(n), int(p)
        arr[k].ax, arr[k].ay, arr[k].az = float(ax), float(ay), float(az)
    return arr, len(modes)


def _sources(src):
    src = list(src)
    arr = (_Source * max(1, len(src)))()
    for k, (m, n, a, w) in enumerate(src):
        arr[k].m, arr[k].n, arr[k].amp, arr[k].omega = int(m), int(n), float(a), float(w)
    return arr, len(src)


def _sources_xy(src):
    src = list(src)
    arr = (_SourceXY * max(1, len(src)))()
    for k, (m, n, a, w, px, py) in enumerate(src):
        arr[k].m, arr[k].n, arr[k].cos_x, arr[k].cos_y = int(m), int(n), int(px), int(py)
        arr[k].amp, arr[k].omega = float(a), float(w)
    return arr, len(src)


def _sources3(src):
    """Rows (m, n, p, a_x, a_y, a_z, omega) as a ctypes array."""
    rows = list(src)
    arr = (_Source3 * max(len(rows), 1))()
    for k, r in enumerate(rows):
        arr[k] = _Source3(int(r[0]), int(r[1]), int(r[2]), float(r[3]), float(r[4]), float(r[5]), float(r[6]))
    return arr, len(rows)


def _ptrs(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(int(p)) for p in ptrs])


def autotune_cache_get(key: str):
    """Cached launch plan of `key` (memory, then the MS_AUTOTUNE_CACHE file), or None; no GPU."""
    p = (ctypes.c_int * 3)()
    found = ctypes.c_int()
    _check(load().ms_autotune_cache_get(key.encode(), p, ctypes.byref(found)))
    return tuple(p) if found.value else None


def autotune_cache_put(key: str, plan):
    """Store a launch plan in the cache (and append it to the MS_AUTOTUNE_CACHE file); no GPU."""
    _check(load().ms_autotune_cache_put(key.encode(), (ctypes.c_int * 3)(*[int(v) for v in plan])))


def autotune_cache_clear():
    """Forget the in-memory cache (the file stays); no GPU."""
    _check(load().ms_autotune_cache_clear())


def stability_limit(dim: int = 2) -> float:
    """Largest stable CFL number of the scheme (from its Fourier symbol); needs no GPU."""
    v = ctypes.c_double()
    _check(load().ms_stability_limit(int(dim), ctypes.byref(v)))
    return v.value


def solver_sweeps(dim: int, r: float, precision: int, tol: float) -> int:
    """Richardson sweeps of the GPU elliptic solve for error reduction `tol` (App. A.2 bound);
    raises MaxwellError (MS_ENOTCONV) when the solve kernels cannot hold that many; needs no GPU."""
    v = ctypes.c_int()
    _check(load().ms_solver_sweeps(int(dim), float(r), int(precision), float(tol), ctypes.byref(v)))
    return v.value


def debug_fail_alloc(n: int) -> None:
    """Test hook: the n-th device allocation of the library from now on fails as out of memory
    (host-side injection, nothing is allocated); 0 disarms."""
    _check(load().ms_debug_fail_alloc(int(n)))


def debug_live_allocs() -> int:
    """Device allocations the library holds now (leak checks in tests)."""
    return int(load().ms_debug_live_allocs())


class Grid:
    """A 2D TM_z cavity (unit square, PEC walls) advanced by the compact scheme on the GPU.

    precision: FP64 or FP32_REFINED; closure: CLOSURE_PAPER or CLOSURE_REFLECT;
    scheme: SCHEME_C4 (the paper's scheme), SCHEME_YEE2 (plain Yee comparator) or SCHEME_NC4
    (the paper's non-compact fourth-order comparator NC) or SCHEME_C4_DE (the compact scheme with
    Delta E tracked as in Step 1 / Step 2 as printed).
    stream: a cudaStream_t handle (int), "torch" for torch's current stream, or None.
    dim: 2 (E_z, H_x, H_y) or 3 (E_x, E_y, E_z, H_x, H_y, H_z on the unit cube, arrays [z][y][x]).
    """

    def __init__(self, n: int, r: float, z: float = 1.0, precision: int = FP64, closure: int = CLOSURE_PAPER,
                 scheme: int = SCHEME_C4, stream=None, dim: int = 2):
        L = load()
        if stream == "torch":
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        d = _Desc(int(dim), int(n), float(z), float(r), int(precision), int(closure), int(scheme),
                  ctypes.c_void_p(int(stream)) if stream else None)
        h = ctypes.c_void_p()
        _check(L.ms_create_grid(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.dim = int(dim)
        self.n, self.r, self.z = int(n), float(r), float(z)
        self.precision, self.closure, self.scheme = int(precision), int(closure), int(scheme)
        self.h = 1.0 / n
        self.ht = r * self.h

    # ------------------------------------------------------------------
    def shapes(self):
        N = self.n
        if self.dim == 3:
            out = []
            for c in range(6):
                node = [(a != c % 3) if c < 3 else (a == c % 3) for a in range(3)]
                nx, ny, nz = (N + 1 if q else N for q in node)
                out.append((nz, ny, nx))
            return tuple(out)
        return (N + 1, N + 1), (N, N + 1), (N + 1, N)

    def close(self):
        if self._h:
            load().ms_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------
    def init_modes(self, modes):
        """2D: rows (m, n, amp); 3D: rows (m, n, p, a_x, a_y, a_z) with a . (m, n, p) = 0."""
        if self.dim == 3:
            arr, nm = _modes3(modes)
            _check(load().ms_init_modes3(self._h, arr, nm))
            return
        arr, nm = _modes(modes)
        _check(load().ms_init_modes(self._h, arr, nm))

    def set_fields(self, *fields, step: int = 0):
        """Host FP64 arrays (numpy) in the full staggered layout (3 in 2D, 6 in 3D)."""
        if len(fields) == len(self.shapes()) + 1:  # trailing positional step
            *fields, step = fields
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in fields]
        if len(arrs) != len(self.shapes()):
            raise ValueError(f"expected {len(self.shapes())} arrays")
        for a, s in zip(arrs, self.shapes()):
            if a.shape != s:
                raise ValueError(f"expected shape {s}, got {a.shape}")
        _check(load().ms_set_fields(self._h, _ptrs([a.ctypes.data for a in arrs]), int(step)))

    def get_fields(self):
        out = [np.zeros(s) for s in self.shapes()]
        _check(load().ms_get_fields(self._h, _ptrs([a.ctypes.data for a in out])))
        return tuple(out)

    def set_fields_device(self, *fields, step: int = 0):
        """torch CUDA float64 tensors (contiguous) in the full staggered layout."""
        if len(fields) == len(self.shapes()) + 1:
            *fields, step = fields
        if len(fields) != len(self.shapes()):
            raise ValueError(f"expected {len(self.shapes())} tensors")
        for t, s in zip(fields, self.shapes()):
            if tuple(t.shape) != s or not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch.float64":
                raise ValueError("expected contiguous CUDA float64 tensors of the staggered shapes")
        _check(load().ms_set_fields_device(self._h, _ptrs([t.data_ptr() for t in fields]), int(step)))

    def get_fields_device(self, *fields):
        if len(fields) != len(self.shapes()):
            raise ValueError(f"expected {len(self.shapes())} tensors")
        _check(load().ms_get_fields_device(self._h, _ptrs([t.data_ptr() for t in fields])))

    def step(self):
        _check(load().ms_step(self._h))

    def run(self, nsteps: int):
        _check(load().ms_run(self._h, int(nsteps)))

    def sync(self):
        _check(load().ms_sync(self._h))

    @property
    def step_count(self) -> int:
        v = ctypes.c_long()
        _check(load().ms_get_step(self._h, ctypes.byref(v)))
        return v.value

    @property
    def launches_per_step(self) -> int:
        v = ctypes.c_int()
        _check(load().ms_launches_per_step(self._h, ctypes.byref(v)))
        return v.value

    def energy(self) -> float:
        v = ctypes.c_double()
        _check(load().ms_energy(self._h, ctypes.byref(v)))
        return v.value

    def divergence(self) -> float:
        v = ctypes.c_double()
        _check(load().ms_divergence(self._h, ctypes.byref(v)))
        return v.value

    def error_vs_exact(self, modes):
        """(l2_abs, l2_rel, max_abs, sum_abs) of the state against the exact modes."""
        arr, nm = _modes3(modes) if self.dim == 3 else _modes(modes)
        out = [ctypes.c_double() for _ in range(4)]
        fn = load().ms_error_vs_exact3 if self.dim == 3 else load().ms_error_vs_exact
        _check(fn(self._h, arr, nm, *[ctypes.byref(v) for v in out]))
        return tuple(v.value for v in out)

    def set_sources3(self, src):
        """3D current sources: divergence-free driven modes, rows (m, n, p, a_x, a_y, a_z, omega)."""
        arr, n = _sources3(src)
        _check(load().ms_set_sources3(self._h, arr, n))

    def init_driven3(self, src):
        """E^0, H^{1/2} = the exact driven solution of 3D sources (step counter 0)."""
        arr, n = _sources3(src)
        _check(load().ms_init_driven3(self._h, arr, n))

    def set_adjoint_precision(self, precision: int):
        """Arithmetic of the reverse pass (FP64, or FP32_REFINED on FP32_REFINED grids, their default)."""
        _check(load().ms_set_adjoint_precision(self._h, int(precision)))

    def set_solver(self, solver: int):
        """Select the P1 solver (SOLVER_RICHARDSON, or SOLVER_TRANSFORM_TC on 3D FP32_REFINED grids)."""
        _check(load().ms_set_solver(self._h, int(solver)))

    def transform_solve(self, comp: int, b, x):
        """x ~ (6 h^2 P1)^{-1} b by the tensor-core transforms alone (device float32 tensors in the
        component's layout), asynchronous on the grid's stream."""
        _check(load().ms_transform_solve3(self._h, int(comp), ctypes.c_void_p(b.data_ptr()),
                                           ctypes.c_void_p(x.data_ptr())))

    def step_profiled(self, cap: int = 512):
        """One step with an event after every launch: list of (kernel kind, ms, algorithmic bytes)."""
        L = load()
        ms = (ctypes.c_float * cap)()
        kinds = (ctypes.c_int * cap)()
        nbytes = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        _check(L.ms_step_profiled(self._h, cap, ms, kinds, nbytes, ctypes.byref(n)))
        return [(L.ms_kernel_kind_name(kinds[k]).decode(), ms[k], nbytes[k]) for k in range(min(n.value, cap))]

    def apply_op(self, op: str, ins, outs):
        """Operator entry point on CUDA float64 tensors (see maxwell4.h, ms_apply_op)."""
        _check(load().ms_apply_op(self._h, OPS[op], _ptrs([t.data_ptr() for t in ins]),
                                  _ptrs([t.data_ptr() for t in outs])))

    # -- checkpoint / resume (maxwell4.h, ms_save / ms_load) --
    def save(self, path: str):
        _check(load().ms_save(self._h, os.fsencode(path)))

    def load_state(self, path: str):
        _check(load().ms_load(self._h, os.fsencode(path)))

    # -- current sources J_z = amp sin(pi m x) sin(pi n y) sin(omega t) (maxwell4.h, ms_set_sources) --
    def set_sources(self, src):
        """Rows (m, n, amp, omega); an empty list removes the sources."""
        arr, ns = _sources(src)
        _check(load().ms_set_sources(self._h, arr, ns))

    def set_sources_xy(self, src):
        """Rows (m, n, amp, omega, cos_x, cos_y): J_z = amp X(pi m x) Y(pi n y) sin(omega t) with X = sin
        (cos_x = 0) or cos (cos_x = 1), Y likewise; cosine profiles need the PAPER closure
        (maxwell4.h, ms_set_sources_xy)."""
        arr, ns = _sources_xy(src)
        _check(load().ms_set_sources_xy(self._h, arr, ns))

    def init_driven(self, src):
        """E^0, H^{1/2} = the exact particular solution driven by the sources."""
        arr, ns = _sources(src)
        _check(load().ms_init_driven(self._h, arr, ns))

    def error_vs_driven(self, src):
        arr, ns = _sources(src)
        out = [ctypes.c_double() for _ in range(4)]
        _check(load().ms_error_vs_driven(self._h, arr, ns, *[ctypes.byref(v) for v in out]))
        return tuple(v.value for v in out)

    # -- non-mode initial data and the reverse pass (maxwell4.h, ms_taylor_init / ms_adjoint_*) --
    def _host(self, a, shape):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != shape:
            raise ValueError(f"expected shape {shape}, got {a.shape}")
        return a

    @staticmethod
    def _dev(t, shape):
        if tuple(t.shape) != shape or not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch.float64":
            raise ValueError(f"expected a contiguous CUDA float64 tensor of shape {shape}")
        return ctypes.c_void_p(t.data_ptr())

    def taylor_init(self, ez0):
        """E_z^0 = ez0 and H^{1/2} by the Taylor series with H^0 = 0; step counter reset."""
        a = self._host(ez0, self.shapes()[0])
        _check(load().ms_taylor_init(self._h, a.ctypes.data_as(ctypes.c_void_p)))

    def taylor_init_device(self, ez0):
        _check(load().ms_taylor_init_device(self._h, self._dev(ez0, self.shapes()[0])))

    def taylor_init_T(self, l_hx, l_hy):
        """Transpose of the map E^0 -> H^{1/2}: returns an (N+1)^2 array."""
        _, sx, sy = self.shapes()
        a, b = self._host(l_hx, sx), self._host(l_hy, sy)
        out = np.zeros(self.shapes()[0])
        _check(load().ms_taylor_init_T(self._h, a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p),
                                       out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def adjoint_run(self, nsteps: int, dL_dEzT):
        """dL/dE_z^0 of a loss of E_z after nsteps steps from taylor_init data (host arrays)."""
        a = self._host(dL_dEzT, self.shapes()[0])
        out = np.zeros(self.shapes()[0])
        _check(load().ms_adjoint_run(self._h, int(nsteps), a.ctypes.data_as(ctypes.c_void_p),
                                     out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def adjoint_run_device(self, nsteps: int, dL_dEzT, dL_dEz0):
        s = self.shapes()[0]
        _check(load().ms_adjoint_run_device(self._h, int(nsteps), self._dev(dL_dEzT, s), self._dev(dL_dEz0, s)))

    def adjoint_steps(self, nsteps: int, l_ez, l_hx, l_hy):
        """(M^T)^nsteps applied to an adjoint state (host arrays); returns the new state."""
        arrs = [self._host(a, s).copy() for a, s in zip((l_ez, l_hx, l_hy), self.shapes())]
        _check(load().ms_adjoint_steps(self._h, int(nsteps), _ptrs([a.ctypes.data for a in arrs])))
        return tuple(arrs)

    def adjoint_steps_device(self, nsteps: int, l_ez, l_hx, l_hy):
        ptrs = [self._dev(t, s).value for t, s in zip((l_ez, l_hx, l_hy), self.shapes())]
        _check(load().ms_adjoint_steps_device(self._h, int(nsteps), _ptrs(ptrs)))


class Batch:
    """Many independent 2D TM_z cavities of uneven sizes advanced together (FP32_REFINED).

    sizes: cells per side of each cavity; the other arguments are shared, as in Grid.
    """

    def __init__(self, sizes, r: float, z: float = 1.0, closure: int = CLOSURE_PAPER, stream=None):
        L = load()
        if stream == "torch":
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        sizes = [int(n) for n in sizes]
        arr = (ctypes.c_int * len(sizes))(*sizes)
        d = _Desc(2, 0, float(z), float(r), FP32_REFINED, int(closure), SCHEME_C4,
                  ctypes.c_void_p(int(stream)) if stream else None)
        h = ctypes.c_void_p()
        _check(L.ms_create_batch(ctypes.byref(d), arr, len(sizes), ctypes.byref(h)))
        self._h = h
        self.sizes, self.r, self.z, self.closure = sizes, float(r), float(z), int(closure)

    def shapes(self, cavity: int):
        N = self.sizes[cavity]
        return (N + 1, N + 1), (N, N + 1), (N + 1, N)

    def close(self):
        if self._h:
            load().ms_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init_modes(self, cavity: int, modes):
        arr, nm = _modes(modes)
        _check(load().ms_batch_init_modes(self._h, int(cavity), arr, nm))

    def set_fields(self, cavity: int, ez, hx, hy, step: int = 0):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (ez, hx, hy)]
        for a, s in zip(arrs, self.shapes(cavity)):
            if a.shape != s:
                raise ValueError(f"expected shape {s}, got {a.shape}")
        _check(load().ms_batch_set_fields(self._h, int(cavity), _ptrs([a.ctypes.data for a in arrs]), int(step)))

    def get_fields(self, cavity: int):
        out = [np.zeros(s) for s in self.shapes(cavity)]
        _check(load().ms_batch_get_fields(self._h, int(cavity), _ptrs([a.ctypes.data for a in out])))
        return tuple(out)

    def step(self):
        _check(load().ms_batch_step(self._h))

    def run(self, nsteps: int):
        _check(load().ms_batch_run(self._h, int(nsteps)))

    def sync(self):
        _check(load().ms_batch_sync(self._h))

    def set_plan(self, order: int, chunk: int, persistent: int):
        """Launch plan: work-list order (0, 1, 2), steps per captured graph, persistent launches."""
        _check(load().ms_batch_set_plan(self._h, (ctypes.c_int * 3)(int(order), int(chunk), int(persistent))))

    def plan(self):
        p = (ctypes.c_int * 3)()
        _check(load().ms_batch_get_plan(self._h, p))
        return tuple(p)

    def autotune(self, trial_steps: int = 16):
        """Choose the launch plan by timing the candidates (before any fields are set); returns
        (plan, from_cache)."""
        p = (ctypes.c_int * 3)()
        hit = ctypes.c_int()
        _check(load().ms_batch_autotune(self._h, int(trial_steps), p, ctypes.byref(hit)))
        return tuple(p), bool(hit.value)

    def error_vs_exact(self, cavity: int, modes):
        arr, nm = _modes(modes)
        out = [ctypes.c_double() for _ in range(4)]
        _check(load().ms_batch_error_vs_exact(self._h, int(cavity), arr, nm, *[ctypes.byref(v) for v in out]))
        return tuple(v.value for v in out)

    def info(self):
        """(cavities, cells advanced per step, kernel launches per step)."""
        c, cells, nl = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int()
        _check(load().ms_batch_info(self._h, ctypes.byref(c), ctypes.byref(cells), ctypes.byref(nl)))
        return c.value, cells.value, nl.value
