"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, exports every
entry point that include/maxwell4.h declares, and validates descriptors before touching CUDA."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_2306_17263_gb300 as pkg
from closed_forms import mode_step_matrix, mode_step_matrix3

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "maxwell4.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ms_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    L = pkg.load()
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n


def _desc(**kw):
    d = dict(dim=2, n=64, z_imp=1.0, r=0.5, precision=0, closure=0, scheme=0, stream=None)
    d.update(kw)
    return pkg._Desc(d["dim"], d["n"], d["z_imp"], d["r"], d["precision"], d["closure"], d["scheme"], d["stream"])


@pytest.mark.parametrize("kw,status", [
    (dict(dim=1), -1), (dict(dim=3, r=0.58), -2), (dict(dim=3, n=600, r=0.4), -1),
    (dict(dim=3, r=0.4, scheme=1), -7), (dict(dim=3, r=0.4, precision=7), -1), (dict(n=3), -1), (dict(n=40000), -1), (dict(z_imp=0.0), -1),
    (dict(r=-0.1), -1), (dict(r=float("nan")), -1), (dict(precision=5), -1), (dict(closure=9), -1),
    (dict(scheme=4), -1), (dict(r=0.70), -2), (dict(r=1 / math.sqrt(2)), -2),
    (dict(scheme=1, r=0.75), -2), (dict(scheme=1, precision=1), -7),
    (dict(scheme=2, r=0.61), -2), (dict(scheme=2, precision=1), -7), (dict(scheme=4), -1),
    (dict(scheme=3, r=0.70), -2),
])
def test_descriptor_validation(kw, status):
    L = pkg.load()
    h = ctypes.c_void_p()
    d = _desc(**kw)
    assert L.ms_create_grid(ctypes.byref(d), ctypes.byref(h)) == status
    assert not h.value
    assert L.ms_last_error().decode() != ""


def test_null_arguments_rejected():
    L = pkg.load()
    h = ctypes.c_void_p()
    assert L.ms_create_grid(None, ctypes.byref(h)) == -1
    assert L.ms_step(None) == -1
    assert L.ms_run(None, 5) == -1
    assert L.ms_destroy(None) == 0


def test_stability_limit_matches_mode_recurrence():
    """The exported limit agrees with the closed-form per-mode step matrix (Sec. 4 recurrence)."""
    rmax = pkg.stability_limit(2)
    assert 5 / (6 * math.sqrt(2)) < rmax < 1 / math.sqrt(2)
    N = 512

    def amp(r):
        return max(np.max(np.abs(np.linalg.eigvals(mode_step_matrix(N, r, kx, ky))))
                   for kx in (N - 1, N - 2) for ky in (N - 1, N - 2))
    assert amp(rmax * 0.999) < 1 + 1e-9
    assert amp(rmax * 1.003) > 1 + 1e-6


def test_stability_limit_3d_matches_mode_recurrence():
    """3D: the exported limit agrees with the closed-form 6x6 per-mode step matrix."""
    rmax = pkg.stability_limit(3)
    assert 5 / (6 * math.sqrt(3)) < rmax < 0.6
    N = 512

    def amp(r):
        return max(np.max(np.abs(np.linalg.eigvals(mode_step_matrix3(N, r, a, b, c))))
                   for a in (N - 1, N - 3) for b in (N - 1, N - 3) for c in (N - 1, N - 3))
    assert amp(rmax * 0.999) < 1 + 1e-9
    assert amp(rmax * 1.003) > 1 + 1e-6


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("r", [0.2, 0.4, 0.5])
def test_solver_sweeps_follow_the_contraction_bound(dim, r):
    """App. A.2: h^2 P1 has its spectrum in [c1 h^2, c1 h^2 + 16/3], so Richardson contracts the
    error by (16/3) / (2 c1 h^2 + 16/3) per sweep; the count is the smallest S with rho^S <= tol."""
    c1h2 = (24 / r ** 2) * (1 + 2 / r ** 2)
    rho = (16 / 3) / (2 * c1h2 + 16 / 3)
    for prec, tol in ((pkg.FP64, 1e-17), (pkg.FP32_REFINED, 1e-10)):
        s = pkg.solver_sweeps(dim, r, prec, tol)
        assert rho ** s <= tol < rho ** (s - 1)


def test_solver_sweeps_not_converged_and_invalid():
    """MS_ENOTCONV when the tolerance needs more sweeps than the solve kernels hold; the other
    failures are MS_ECFL (r at the stability limit) and MS_EINVAL."""
    L = pkg.load()
    v = ctypes.c_int(7)
    assert L.ms_solver_sweeps(2, 0.5, pkg.FP32_REFINED, 1e-40, ctypes.byref(v)) == -6
    assert v.value == 0 and "sweeps" in L.ms_last_error().decode()
    assert L.ms_solver_sweeps(3, 0.4, pkg.FP32_REFINED, 1e-60, ctypes.byref(v)) == -6
    assert L.ms_solver_sweeps(2, 0.5, pkg.FP64, 1e-300, ctypes.byref(v)) == -6
    with pytest.raises(pkg.MaxwellError):
        pkg.solver_sweeps(2, 0.5, pkg.FP32_REFINED, 1e-40)
    assert L.ms_solver_sweeps(2, 0.69, pkg.FP64, 1e-10, ctypes.byref(v)) == -2
    assert L.ms_solver_sweeps(3, 0.57, pkg.FP64, 1e-10, ctypes.byref(v)) == -2
    for args in ((4, 0.5, 0, 1e-10), (2, 0.5, 3, 1e-10), (2, -0.5, 0, 1e-10), (2, 0.5, 0, 0.0),
                 (2, 0.5, 0, 1.0), (2, float("nan"), 0, 1e-10)):
        assert L.ms_solver_sweeps(*args, ctypes.byref(v)) == -1, args
    assert L.ms_solver_sweeps(2, 0.5, 0, 1e-10, None) == -1


def test_autotune_cache_memory_and_file(tmp_path, monkeypatch):
    """The batch autotuner's plan cache: a stored plan is found again in memory, survives the loss of
    the memory copy through the MS_AUTOTUNE_CACHE file (last line of a key wins), and keys and plans
    are validated; no GPU involved."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("MS_AUTOTUNE_CACHE", str(path))
    pkg.autotune_cache_clear()
    assert pkg.autotune_cache_get("batch:abc;r=0.5") is None
    pkg.autotune_cache_put("batch:abc;r=0.5", (1, 32, 0))
    assert pkg.autotune_cache_get("batch:abc;r=0.5") == (1, 32, 0)
    pkg.autotune_cache_put("batch:abc;r=0.5", (2, 8, 1))
    assert path.read_text().splitlines() == ["batch:abc;r=0.5 1 32 0", "batch:abc;r=0.5 2 8 1"]
    pkg.autotune_cache_clear()
    assert pkg.autotune_cache_get("batch:abc;r=0.5") == (2, 8, 1)  # from the file
    assert pkg.autotune_cache_get("batch:other") is None
    monkeypatch.delenv("MS_AUTOTUNE_CACHE")
    pkg.autotune_cache_clear()
    assert pkg.autotune_cache_get("batch:abc;r=0.5") is None  # memory only now
    for key, plan in (("bad key", (0, 16, 0)), ("", (0, 16, 0)), ("k", (3, 16, 0)), ("k", (0, 0, 0)),
                      ("k", (0, 300, 0)), ("k", (0, 16, 2))):
        with pytest.raises(pkg.MaxwellError) as e:
            pkg.autotune_cache_put(key, plan)
        assert e.value.status == -1


def test_alloc_failure_hook_host_side():
    """The allocation-failure hook arms, disarms and rejects a negative count without a GPU, and
    descriptor validation runs before any allocation (an armed failure is not consumed)."""
    assert pkg.debug_live_allocs() == 0
    with pytest.raises(pkg.MaxwellError) as e:
        pkg.debug_fail_alloc(-1)
    assert e.value.status == -1
    L = pkg.load()
    pkg.debug_fail_alloc(1)
    try:
        h = ctypes.c_void_p()
        d = _desc(dim=1)
        assert L.ms_create_grid(ctypes.byref(d), ctypes.byref(h)) == -1
        assert not h.value
        assert pkg.debug_live_allocs() == 0
    finally:
        pkg.debug_fail_alloc(0)
