"""The form in which the tile kernels apply interior rows of A^{-1} (App. A.1, Eq. "eq:lhs"),
checked in FP64 against a dense solve of A = (1/24) tridiag(1, 22, 1) and against the closed-form
band 24 (-rho) rho^|d| / (1 - rho^2):

- A factors as (1 - rho E^-1)(1 - rho E) / (1 - rho)^2 with rho = -11 + sqrt(120), so A^{-1} d is a
  forward recurrence z_i = d_i + rho z_{i-1}, a backward one y_i = z_i + rho y_{i+1} and the scale
  (1 - rho)^2 (the 2D curl tiles);
- by partial fractions the same is (1 - rho) / (1 + rho) (f + g - d) with f, g the forward and the
  backward recurrence over d (the 3D Pade terms);
- each recurrence starts KR + 1 = 7 rows before its first output from the steady state of the value
  there, an error below |rho|^7 times the change of d over those rows;
- with rho rounded to FP32 and the scale formed from that rounded rho, the DC gain is exactly 1.
No GPU: these are the identities the kernels are built on, written out in numpy."""
import numpy as np

RHO = -11.0 + np.sqrt(120.0)
KR = 6
SEG = 8


def dense_inverse_apply(d):
    """A^{-1} d on a line of len(d) points with the interior rows of A everywhere (the rows far from
    the ends are those of the infinite Toeplitz operator to far below FP64 precision)."""
    m = len(d)
    A = (np.diag(np.full(m, 22.0)) + np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)) / 24.0
    return np.linalg.solve(A, d)


def sequential_segment(d, rf, rho=RHO, scale=None):
    """Outputs rf .. rf+SEG-1 by the forward then the backward recurrence (2D curl form)."""
    if scale is None:
        scale = (1.0 - rho) ** 2
    z = d[rf - KR - 1] / (1.0 - rho)
    zs = {}
    for i in range(rf - KR, rf + SEG + KR):
        z = d[i] + rho * z
        zs[i] = z
    y = z / (1.0 - rho)
    out = np.empty(SEG)
    for i in range(rf + SEG + KR - 1, rf - 1, -1):
        y = zs[i] + rho * y
        if i < rf + SEG:
            out[i - rf] = scale * y
    return out


def partial_fraction_segment(d, rf, rho=RHO):
    """The same outputs as (1 - rho)/(1 + rho) (f + g - d), f and g independent (3D term form)."""
    f = d[rf - KR - 1] / (1.0 - rho)
    fs = {}
    for i in range(rf - KR, rf + SEG):
        f = d[i] + rho * f
        fs[i] = f
    g = d[rf + SEG + KR] / (1.0 - rho)
    out = np.empty(SEG)
    for i in range(rf + SEG + KR - 1, rf - 1, -1):
        g = d[i] + rho * g
        if i < rf + SEG:
            out[i - rf] = (1.0 - rho) / (1.0 + rho) * (fs[i] + g - d[i])
    return out


def test_rho_and_the_factorisation():
    assert abs(RHO * RHO + 22.0 * RHO + 1.0) < 1e-14
    assert abs((1.0 - RHO) ** 2 + 24.0 * RHO) < 1e-14
    # the symbol of the factors equals that of A on a few frequencies
    for th in (0.0, 0.3, 1.0, 2.5, np.pi):
        a = (22.0 + 2.0 * np.cos(th)) / 24.0
        e = np.exp(1j * th)
        fac = (1.0 - RHO / e) * (1.0 - RHO * e) / (1.0 - RHO) ** 2
        assert abs(fac - a) < 1e-15


def test_recurrences_match_a_dense_solve_and_the_band():
    rng = np.random.default_rng(7)
    m = 400
    x = np.linspace(0.0, 1.0, m)
    # a smooth line (resolved modes) plus a little noise at every wavenumber
    d = np.sin(7.0 * x) + 0.3 * np.cos(23.0 * x) + 1e-3 * rng.standard_normal(m)
    ref = dense_inverse_apply(d)
    band = np.array([24.0 * (-RHO) * RHO ** abs(k) / (1.0 - RHO * RHO) for k in range(-30, 31)])
    for rf in (100, 173, 250):
        seq = sequential_segment(d, rf)
        pf = partial_fraction_segment(d, rf)
        want = ref[rf:rf + SEG]
        via_band = np.array([band @ d[r - 30:r + 31] for r in range(rf, rf + SEG)])
        assert np.max(np.abs(via_band - want)) < 1e-13
        # warm-up error: |rho|^7 ~ 4e-10 times the change of d over the rows before the segment
        assert np.max(np.abs(seq - want)) < 2e-9 * np.max(np.abs(d))
        assert np.max(np.abs(pf - want)) < 2e-9 * np.max(np.abs(d))


def test_warm_up_error_falls_like_rho_to_the_warm_up_length():
    """A step in d just before the warm-up start: the error at the segment is that step damped by
    |rho|^(KR+1) (within a factor of a few), and a constant d is reproduced exactly."""
    m = 200
    rf = 100
    const = np.full(m, 3.0)
    assert np.max(np.abs(sequential_segment(const, rf) - 3.0)) < 1e-14
    d = np.zeros(m)
    d[: rf - KR - 1] = 1.0  # a unit step ending where the forward recurrence starts
    ref = dense_inverse_apply(d)
    err = np.max(np.abs(sequential_segment(d, rf) - ref[rf:rf + SEG]))
    assert err < 5.0 * abs(RHO) ** (KR + 1)
    assert err > 0.01 * abs(RHO) ** (KR + 1)


def test_dc_gain_is_exact_with_the_fp32_rho():
    """The kernels round rho to FP32 and form the scale (1 - rho_f)^2 from that rounded value in
    extended precision (split hi + lo): the recurrences then reproduce a constant exactly, while a
    scale taken from the exact rho would be off by ~2 |rho - rho_f| / (1 - rho) ~ 1e-8, a coherent
    error of the derivative in every step."""
    rho_f = float(np.float32(RHO))
    one_m = 1.0 - rho_f
    scale_f = one_m * one_m
    # DC gain of the recurrences with rho_f: scale / (1 - rho_f)^2
    assert abs(scale_f / one_m ** 2 - 1.0) < 1e-15
    assert abs((1.0 - rho_f) / (1.0 + rho_f) * (2.0 / (1.0 - rho_f) - 1.0) - 1.0) < 1e-15
    wrong = (1.0 - RHO) ** 2 / one_m ** 2
    assert 1e-10 < abs(wrong - 1.0) < 1e-7
    # the change rho -> rho_f moves A's symbol by ~1e-11 at the benchmark's wavenumbers
    th = np.pi * 40 / 2048
    sym = lambda r: (1.0 - r * np.exp(-1j * th)) * (1.0 - r * np.exp(1j * th)) / (1.0 - r) ** 2
    assert abs(sym(rho_f) - sym(RHO)) < 1e-10
