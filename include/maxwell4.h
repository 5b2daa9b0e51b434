/*
 * maxwell4.h -- C ABI of the GB300 (sm_103a) implementation of the compact
 * fourth-order staggered scheme for the first-order Maxwell equations
 * (Versano, Turkel & Tsynkov, arXiv 2306.17263).
 *
 * One time step is the paper's Step 1 / Step 2 (Sec. 3.4):
 *   P1^E E* = kappa^2 Z curl_h[(1 + kappa^2 h^2/12) H^{n+1/2} + (h^2/12) Delta_h H^{n+1/2}]
 *   E^{n+1} = E^n + h_tau E*
 *   P1^H H* = -(kappa^2/Z) curl_h[(1 + kappa^2 h^2/12) E^{n+1} + (h^2/12) Delta_h E^{n+1}]
 *   H^{n+3/2} = H^{n+1/2} + h_tau H*
 * with kappa^2 = 24/h_tau^2 (Sec. 3.2), P1 = -(Delta_h + (h^2/6) Upsilon_h) + kappa^2(1 + 2/r^2)
 * (Definition "def:operatorsP"), curl_h the Pade compact curl of App. A.1 (Eq. "eq:lhs"),
 * Dirichlet / even-ghost Neumann boundaries of Table "tab:bc" and Corollary "cor:ghost_cor".
 * J defaults to zero (rho = 0 throughout).  The source entry points (ms_set_sources,
 * ms_set_sources_xy) add a current J_z: Step 1 then gains the filtered Z P(J) term of Eq. "eq:pj"
 * on its right-hand side and Step 2 the filtered curl d_t J term (Sec. 3.1, 3.4), and currents
 * that do not vanish on the walls bring the inhomogeneous ghosts of Sec. 3.3 (Method 2).
 *
 * Conventions for every entry point:
 *   - Status codes are returned, never thrown.  On failure a message is available from
 *     ms_last_error() (thread-local, valid until the next call on the same thread).
 *   - Pointers passed in are borrowed for the duration of the call only; nothing is retained.
 *   - Host field arrays are FP64 in the full staggered layout (boundary points included),
 *     row-major with x fastest.  2D TM_z (Sec. 5, Eq. "maxwell2d"), N cells per side:
 *         comps[0] = E_z : (N+1) rows x (N+1) cols, point (x_i, y_j)
 *         comps[1] = H_x : N rows     x (N+1) cols, point (x_i, y_{j+1/2})
 *         comps[2] = H_y : (N+1) rows x N cols,     point (x_{i+1/2}, y_j)
 *     E is at time n h_tau and H at (n + 1/2) h_tau (Sec. 2).  Boundary values of the
 *     Dirichlet components are zero on input and output (PEC walls, Eq. "eq:bc_E=0").
 *   - The grid owns all device memory it needs; it is allocated in ms_create_grid and
 *     released in ms_destroy.  All work is issued on the grid's stream.
 *   - A grid handle must not be used from two threads at once.
 */
#ifndef MAXWELL4_H
#define MAXWELL4_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ms_grid ms_grid;

typedef enum {
  MS_OK = 0,
  MS_EINVAL = -1,        /* invalid argument or descriptor */
  MS_ECFL = -2,          /* CFL number at or above the stability limit */
  MS_ENOMEM = -3,        /* device or host allocation failed */
  MS_ECUDA = -4,         /* a CUDA runtime call failed */
  MS_ETIMEOUT = -5,      /* a bounded device-side wait gave up */
  MS_ENOTCONV = -6,      /* an iterative solve did not reach its tolerance */
  MS_EUNSUPPORTED = -7   /* valid but not implemented combination */
} ms_status;

/* Arithmetic of the time step.
 *   MS_FP64:          every kernel computes in FP64.
 *   MS_FP32_REFINED:  FP32 arithmetic; every scalar coefficient that is not exact in FP32 is
 *                     applied as an error-free hi+lo pair, the elliptic and Pade solves are
 *                     iterated to convergence against residuals with those exact coefficients,
 *                     and the state is kept as an unevaluated FP32 hi+lo sum updated with
 *                     error-free transformations (about 48 significant bits). */
typedef enum { MS_FP64 = 0, MS_FP32_REFINED = 1 } ms_precision;

/* Rows of the Pade matrix A at the two ends of each line (App. A.1, Eq. "eq:lhs").
 *   MS_CLOSURE_PAPER:   the printed one-sided rows [26,-5,4,-1]/24 at both ends.
 *   MS_CLOSURE_REFLECT: rows from the parity of the field about the wall ([23,1]/24 on the
 *                       node-to-half-node lines, [22,1]/24 on half-node-to-node lines); with it
 *                       every operator of the step is diagonal on the cavity modes. */
typedef enum { MS_CLOSURE_PAPER = 0, MS_CLOSURE_REFLECT = 1 } ms_closure;

/* Time-stepping scheme.  MS_SCHEME_C4 is the paper's compact scheme (Sec. 3.4);
 * MS_SCHEME_YEE2 is the plain second-order Yee update (Sec. 5.2, stencil S with c = 1);
 * MS_SCHEME_NC4 is the paper's non-compact fourth-order comparator NC (Sec. 5.2, stencil K4 of
 * Eq. "eq:K4" with a = 0: the (9/8, -1/24) staggered difference, the standard fourth-order
 * one-sided difference (-23, 21, 3, -1)/24 at the line ends, leapfrog in time).  The two
 * comparators run in FP64 on 2D grids; NC needs r < 1 / (sqrt 2 (9/8 + 1/24)) = 0.606.
 * MS_SCHEME_C4_DE is the compact scheme in the form Step 1 / Step 2 print it: Delta E_z is
 * carried as state DE, advanced after Step 1 by Eq. "eq:mhe" (DE += kappa^2 (E^{n+1} - E^n)
 * - Z (24/h_tau) curl_h H^{n+1/2}), and Step 2 filters E with it (Eq. "eq:helm2") instead of
 * with Delta_h E.  2D, both precisions (in MS_FP32_REFINED DE is a float-float field and its
 * update, the small difference of two large terms, is formed in float-float); not for batches,
 * sources or the reverse pass.  DE starts as the exact Delta E of the modes (ms_init_modes) or as
 * Delta_h E^0 (ms_set_fields); it is internal state, not returned by ms_get_fields. */
typedef enum { MS_SCHEME_C4 = 0, MS_SCHEME_YEE2 = 1, MS_SCHEME_NC4 = 2, MS_SCHEME_C4_DE = 3 } ms_scheme;

typedef struct {
  int dim;          /* 2 (TM_z: E_z, H_x, H_y) or 3 (six components, see below) */
  int n;            /* cells per side of the unit square / cube, h = 1/n; 4 <= n <= 32768 (2D), 512 (3D) */
  double z_imp;     /* Z = sqrt(mu/epsilon) of Eq. "eq:maxwellv"; > 0 (1.0 in the paper) */
  double r;         /* CFL number h_tau / h, 0 < r < stability limit (Sec. 4) */
  int precision;    /* ms_precision */
  int closure;      /* ms_closure */
  int scheme;       /* ms_scheme */
  void* stream;     /* cudaStream_t to issue work on, or NULL for a stream the grid creates */
} ms_grid_desc;

/* A cavity mode of the 2D TM_z problem (Sec. 5.1, Eq. "eq:data"):
 *   E_z = amp cos(w t) sin(pi m x) sin(pi n y),  w = pi sqrt(m^2 + n^2),
 *   H_x = -amp (1/Z) (sin(w t)/w) pi n sin(pi m x) cos(pi n y),
 *   H_y =  amp (1/Z) (sin(w t)/w) pi m cos(pi m x) sin(pi n y).
 * m, n >= 1. */
typedef struct {
  int m, n;
  double amp;
} ms_mode;

/* Three-dimensional grids (dim = 3): the six components of Eq. "eq:meshes" on the unit cube,
 * host and device arrays in the layout [z][y][x] (x fastest), comps[0..5] = E_x, E_y, E_z, H_x,
 * H_y, H_z.  A component has n+1 points along the axes on which it sits on nodes (Dirichlet,
 * wall values zero) and n points along its half-node axes (Neumann), Table "tab:bc":
 *   E_x (n, n+1, n+1)  E_y (n+1, n, n+1)  E_z (n+1, n+1, n)
 *   H_x (n+1, n, n)    H_y (n, n+1, n)    H_z (n, n, n+1)      as (nx, ny, nz).
 * One step is Step 1 / Step 2 of Sec. 3.4 with the full curl_h, the 7-point Delta_h and the
 * 19-point P1 (Upsilon_h = D_zz D_xx + D_yy D_zz + D_xx D_yy).  ms_set_fields, ms_get_fields
 * (and _device), ms_step, ms_run, ms_sync, ms_get_step, ms_step_profiled and
 * ms_launches_per_step take 3D grids with six arrays; the mode calls are ms_init_modes3 and
 * ms_error_vs_exact3; the other diagnostics, the operator entry points, batches and the reverse
 * pass are 2D only (MS_EUNSUPPORTED, or MS_EINVAL for the 2D mode calls). */

/* Create a grid.  Validates the descriptor (MS_EINVAL), rejects r at or above the exact
 * Fourier stability limit of the scheme (MS_ECFL; about 0.6895 in 2D and 0.5607 in 3D, Sec. 4
 * gives the sufficient bounds 5/(6 sqrt 2) and 5/(6 sqrt 3)), allocates the state and all
 * scratch on the device, and zeroes the fields.  *out receives the handle; it is NULL on failure. */
ms_status ms_create_grid(const ms_grid_desc* desc, ms_grid** out);

/* Release the grid's device memory and stream.  NULL is accepted. */
ms_status ms_destroy(ms_grid* g);

/* Set E^0 and H^{1/2} to the exact superposition of nmodes cavity modes (Eq. "eq:data") at
 * t = 0 and t = h_tau/2, and reset the step counter to 0.  modes is a host array. */
ms_status ms_init_modes(ms_grid* g, const ms_mode* modes, int nmodes);

/* A cavity mode of the 3D problem (not in the paper; derived from Eq. "eq:maxwellv" with PEC
 * walls): with (a, b, c) = pi (m, n, p) and w = |(a, b, c)|,
 *   E = (ax cos(a x) sin(b y) sin(c z), ay sin(a x) cos(b y) sin(c z), az sin(a x) sin(b y) cos(c z)) cos(w t),
 *   H = -(1/(Z w)) curl(E / cos(w t)) sin(w t),
 * which needs (ax, ay, az) . (m, n, p) = 0 (MS_EINVAL otherwise) and m, n, p >= 1. */
typedef struct {
  int m, n, p;
  double ax, ay, az;
} ms_mode3;

/* 3D grids: E^0 and H^{1/2} from a superposition of exact modes; step counter reset to 0.
 * Synchronous. */
ms_status ms_init_modes3(ms_grid* g, const ms_mode3* modes, int nmodes);

/* 3D grids: error of the state against exact modes at t_E = n h_tau, t_H = (n + 1/2) h_tau
 * over the six components (l2 with weight h^3), as ms_error_vs_exact.  Synchronous. */
ms_status ms_error_vs_exact3(ms_grid* g, const ms_mode3* modes, int nmodes, double* l2_abs, double* l2_rel,
                             double* max_abs, double* sum_abs);

/* Current sources on 3D grids (both precisions): divergence-free driven modes shaped like a
 * cavity mode's E,
 *   J = (ax cos(pi m x) sin(pi n y) sin(pi p z), ay sin cos sin, az sin sin cos) sin(omega t),
 * with (ax, ay, az) . (m, n, p) = 0 (so div J = 0 and rho stays 0), m, n, p >= 0 with at least two
 * of them >= 1.  Their tangential components vanish on every wall with all the derivatives the
 * Neumann data of Sec. 3.3 involve, and d_n E_n = rho = 0, so the even ghosts of Cor.
 * "cor:ghost_cor" stay exact.  Step 1 gains the filtered P(J) = Z(-kappa^2 J + grad div J - d_tt J)
 * at t^{n+1/2} and Step 2 the filtered curl d_t J at t^{n+1} (Sec. 3.1, 3.4, the filter of
 * Eq. "eq:ell" with the exact Laplacian of the source).  A source with p = 0 is the 2D TM_z source
 * a_z sin sin extended along z.  ms_set_sources3 replaces the grid's sources (nsrc = 0 removes
 * them; at most 64) and drops the captured step graphs; the step index that times them is the
 * grid's step counter.  ms_init_driven3 sets E^0, H^{1/2} to the exact driven solution of the
 * sources (the particular solution E = A cos(omega t) (ax, ay, az) (E-mode shapes),
 * A = Z omega / (omega^2 - pi^2 (m^2 + n^2 + p^2)), H from Faraday's law; MS_EINVAL at resonance)
 * and the step counter to 0.  MS_EINVAL for invalid rows, MS_EUNSUPPORTED on 2D grids. */
typedef struct {
  int m, n, p;
  double ax, ay, az;
  double omega;
} ms_source3;
ms_status ms_set_sources3(ms_grid* g, const ms_source3* src, int nsrc);
ms_status ms_init_driven3(ms_grid* g, const ms_source3* src, int nsrc);

/* Copy host FP64 fields (layout above) to the device state and set the step counter to
 * `step` (E at step h_tau, H at (step + 1/2) h_tau).  Dirichlet boundary entries are ignored
 * and stored as zero. */
ms_status ms_set_fields(ms_grid* g, const double* const* comps, long step);

/* Copy the device state to host FP64 arrays (layout above). */
ms_status ms_get_fields(ms_grid* g, double* const* comps);

/* Same as ms_set_fields / ms_get_fields with device FP64 arrays (no host copy). */
ms_status ms_set_fields_device(ms_grid* g, const double* const* comps, long step);
ms_status ms_get_fields_device(ms_grid* g, double* const* comps);

/* Advance one full time step (Step 1 then Step 2), asynchronously on the grid's stream. */
ms_status ms_step(ms_grid* g);

/* Advance nsteps steps (nsteps >= 0), replaying a CUDA graph of the step captured on first
 * use; asynchronous on the grid's stream. */
ms_status ms_run(ms_grid* g, long nsteps);

/* Wait for all work issued on the grid's stream; returns MS_ECUDA if any of it failed. */
ms_status ms_sync(ms_grid* g);

/* Current step counter n (E at n h_tau). */
ms_status ms_get_step(ms_grid* g, long* step);

/* Discrete energy at the current state, FP64 reductions:
 *   W^n = Z^{-1} h^d sum E^n.E^n + Z h^d sum H^{n-1/2}.H^{n+1/2}   (d = 2 or 3; all components),
 * with H^{n-1/2} = H^{n+1/2} - h_tau H*(E^n) recomputed on the device.  This is the
 * leapfrog invariant of the scheme in the form of Sec. 4, Eq. "eq:eh" (the paper states
 * no discrete energy); exact under MS_CLOSURE_REFLECT, bounded under MS_CLOSURE_PAPER.
 * 3D grids are evaluated in FP64; an MS_FP32_REFINED 3D grid joins its float-float state into
 * FP64 copies and, on its first call, allocates the FP64 tables and scratch this needs (kept
 * until ms_destroy).  Synchronous. */
ms_status ms_energy(ms_grid* g, double* W);

/* L2 norm sqrt(h^d sum div^2) of the Pade divergence of H on the n^d cell centres,
 * div_h H = delta_x H_x + delta_y H_y (+ delta_z H_z in 3D), node-to-half-node derivatives of
 * App. A.1 along each component's own axis.  3D grids are evaluated in FP64, as ms_energy.
 * Synchronous. */
ms_status ms_divergence(ms_grid* g, double* norm);

/* Error of the current state against a superposition of exact modes at t_E = n h_tau,
 * t_H = (n + 1/2) h_tau, FP64 on the device:
 *   l2_abs = sqrt(h^2 sum (u - u_exact)^2) over E_z, H_x, H_y;  l2_rel = l2_abs / sqrt(h^2 sum u_exact^2);
 *   max_abs = max |u - u_exact|;  sum_abs = sum |u - u_exact| (the summand of the mean absolute
 *   error of Sec. 5.1).  Any output pointer may be NULL.  Synchronous. */
ms_status ms_error_vs_exact(ms_grid* g, const ms_mode* modes, int nmodes, double* l2_abs, double* l2_rel,
                            double* max_abs, double* sum_abs);

/* Operator-level entry points on device FP64 arrays in the full staggered layout (used to
 * check each kernel against the oracle).  Available on MS_FP64 grids (MS_EUNSUPPORTED otherwise).
 *   MS_OP_FILTER_{EZ,HX,HY}: out[0] = (1 + kappa^2 h^2/12) in[0] + (h^2/12) Delta_h in[0]
 *                            (right side of Eq. "eq:ell"; zero on Dirichlet boundary points).
 *   MS_OP_CURL_HE:  out[0] = kappa^2 Z (delta_x in[1] - delta_y in[0]), in = (G_x, G_y) (Step 1).
 *   MS_OP_CURL_EH:  out[0] = -(kappa^2/Z) delta_y in[0], out[1] = (kappa^2/Z) delta_x in[0] (Step 2).
 *   MS_OP_P1_{EZ,HX,HY}:       out[0] = P1 in[0] (Definition "def:operatorsP").
 *   MS_OP_P1SOLVE_{EZ,HX,HY}:  out[0] = P1^{-1} in[0], iterated to the FP64 tolerance.
 * in / out point to 1 or 2 device pointers as listed; inputs and outputs must not overlap.
 * Asynchronous on the grid's stream. */
typedef enum {
  MS_OP_FILTER_EZ = 0, MS_OP_FILTER_HX = 1, MS_OP_FILTER_HY = 2,
  MS_OP_CURL_HE = 3, MS_OP_CURL_EH = 4,
  MS_OP_P1_EZ = 5, MS_OP_P1_HX = 6, MS_OP_P1_HY = 7,
  MS_OP_P1SOLVE_EZ = 8, MS_OP_P1SOLVE_HX = 9, MS_OP_P1SOLVE_HY = 10
} ms_op;
ms_status ms_apply_op(ms_grid* g, int op, const double* const* in, double* const* out);

/* Largest CFL number r for which every Fourier mode of the scheme is neutrally stable
 * (Sec. 4: a mode is stable iff |h_tau lambda| <= 2 in sigma^2 - (2 - lambda^2 h_tau^2) sigma + 1 = 0),
 * computed from the symbols of the operators.  dim is 2 or 3.  Needs no GPU. */
ms_status ms_stability_limit(int dim, double* rmax);

/* Advance one step like ms_step, recording a CUDA event on the grid's stream after every
 * kernel launch, then wait for it.  On return count = number of launches (at most cap are
 * written), launch_ms[k] = time between the end of launch k-1 (or the step's start) and the
 * end of launch k, kinds[k] = kernel kind (see ms_kernel_kind_name), bytes[k] = the launch's
 * algorithmic bytes (each input array element read once, each output element written once).
 * Synchronous. */
ms_status ms_step_profiled(ms_grid* g, int cap, float* launch_ms, int* kinds, double* bytes, int* count);

/* Name of a kernel kind reported by ms_step_profiled ("" for an unknown kind). */
const char* ms_kernel_kind_name(int kind);

/* P1 solve that allocates no device memory.  The paper has no counterpart: this is a
 * library-usage variant of MS_OP_P1SOLVE_{EZ,HX,HY} for callers that cannot call cudaMalloc,
 * e.g. code in a latency-critical loop where an allocation may synchronise the device, or an
 * application (or plugin host) that owns all device memory through its own pool or a fixed
 * budget.  It needs no grid handle.
 *   n:      cells per side, 4 <= n <= MS_STATIC_MAX_N (MS_EINVAL otherwise, with a message);
 *   r:      CFL number (> 0), which with n fixes P1 (Definition "def:operatorsP");
 *   field:  0 = E_z, 1 = H_x, 2 = H_y (boundary types of Table "tab:bc");
 *   b, x:   distinct device FP64 arrays of that field in the full staggered layout, owned by
 *           the caller; x receives P1^{-1} b (zero on Dirichlet boundary points);
 *   stream: cudaStream_t to issue the work on (NULL: the legacy default stream).
 * The iteration's two scratch planes live in one file-scope __device__ array of
 * MS_STATIC_SCRATCH_BYTES, which every GPU that loads this library keeps until the process
 * exits.  The first call on a device looks up the array's device address with that device
 * current (cudaGetSymbolAddress); make that first call before any stream capture.  Every call
 * uses the same array: calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it and must be serialised by the caller.  Nothing in the array needs clearing, since
 * every sweep writes all points before the next reads them.  Asynchronous on `stream`. */
#define MS_STATIC_MAX_N 512
#define MS_STATIC_SCRATCH_BYTES (2u * (MS_STATIC_MAX_N + 1u) * (MS_STATIC_MAX_N + 1u) * 8u)
ms_status ms_p1_solve_static(int n, double r, int field, const double* b, double* x, void* stream);

/* Richardson sweeps the GPU elliptic solves take to reduce the error of P1 x = b by the factor
 * tol from x = 0, from the spectral bound of App. A.2: h^2 P1 has its spectrum in
 * [c1 h^2, c1 h^2 + 16/3] (2D and 3D), c1 h^2 = (24/r^2)(1 + 2/r^2), so one sweep with the
 * optimal relaxation contracts the error by (16/3) / (2 c1 h^2 + 16/3) (about 0.003 at r = 0.5).
 *   dim: 2 or 3;  r: CFL number, 0 < r < the stability limit (MS_ECFL at or above it);
 *   precision: ms_precision; it fixes the largest sweep count the solve kernels hold (FP64: 64;
 *              FP32_REFINED: 6 in 2D, 8 in 3D);  tol: in (0, 1).
 * *sweeps receives the count (0 on failure).  Returns MS_ENOTCONV, with a message, when tol needs
 * more sweeps than the kernels hold, i.e. when the solve would stop short of tol.  Grid creation
 * runs the same check with tol = 1e-17 (FP64) and 1e-10 (FP32_REFINED) and fails with the same
 * status.  Needs no GPU. */
ms_status ms_solver_sweeps(int dim, double r, int precision, double tol, int* sweeps);

/* P1 solver of a grid.  MS_SOLVER_RICHARDSON (every grid's default): Richardson sweeps of the 9- or
 * 19-point operator, their count fixed by the spectral bound of App. A.2 (ms_solver_sweeps).
 * MS_SOLVER_TRANSFORM_TC (3D FP32_REFINED grids only): the separable solve.  Every 1D operator of P1
 * (Def. "def:operatorsP") is a Kronecker lift of D_2 (App. A.1), diagonalised per axis by the
 * orthonormal sine transform (Dirichlet axes) or cosine transform (Neumann axes with even ghosts,
 * Table "tab:bc"), so P1^{-1} is three transforms, a division by the eigenvalues and three inverse
 * transforms.  Each transform is a dense GEMM on the tensor cores (bf16 operands split hi + lo, three
 * products, FP32 accumulation in tensor memory), and the result is refined by Richardson sweeps
 * with the exact residual until the App. A.2 bound reaches the Richardson path's tolerance.
 *   ms_set_solver: MS_EINVAL for an unknown solver, MS_EUNSUPPORTED for the transform solver on
 *     other grids, MS_ENOMEM / MS_ECUDA if its set-up (two padded working copies of a component,
 *     transform matrices) fails.  The first selection allocates; a selection drops the captured
 *     step graphs.  Synchronises the grid's stream.
 *   ms_transform_solve3: x ~ (6 h^2 P1)^{-1} b for component comp (0..5) of a 3D FP32_REFINED grid by
 *     the transforms alone, without refinement; b and x are distinct device FP32 arrays in the
 *     component's full layout (wall points of x are set to zero).  Asynchronous on the grid's stream.
 * A transform kernel whose bounded wait for its tensor-core work gives up records it; the next
 * ms_sync of the grid returns MS_ETIMEOUT (and clears the record). */
typedef enum { MS_SOLVER_RICHARDSON = 0, MS_SOLVER_TRANSFORM_TC = 1 } ms_solver;
ms_status ms_set_solver(ms_grid* g, int solver);
ms_status ms_transform_solve3(ms_grid* g, int comp, const float* b, float* x);

/* Number of kernel launches one ms_step issues (for launch accounting). */
ms_status ms_launches_per_step(ms_grid* g, int* launches);

/* ---------------------------------------------------------------------------------------
 * Current sources (2D TM_z, J = J_z z, so div J = 0 and rho stays 0): a superposition of driven
 * sine modes
 *   J_z = amp sin(pi m x) sin(pi n y) sin(omega t),  m, n >= 1,
 * which vanish on the walls with every derivative the Neumann data of Sec. 3.3 involve, so the
 * boundary treatment of the homogeneous scheme stays exact.  The modified Helmholtz equations of
 * Eq. "eq:mh" gain, from the Taylor expansion of Sec. 3.1 written out with Faraday's and Ampere's
 * laws, P(J) = Z (-kappa^2 J + grad div J - d_tt J) at t^{n+1/2} on the E side and curl d_t J at
 * t^{n+1} on the H side, each through the right-hand-side filter of Eq. "eq:ell" with the exact
 * Laplacian of the source.  (The printed P(J) of Eq. "eq:pj" and the J term of the H expansion
 * differ from this derivation; the derived form is the fourth-order one.)
 *
 * ms_set_sources: replaces the grid's sources (nsrc = 0 removes them); 2D MS_SCHEME_C4 grids in
 *   either precision (MS_EUNSUPPORTED otherwise); at most 64 sources.  The step index that fixes
 *   the source time is kept on the device, so ms_run's captured graphs stay valid.
 * ms_init_driven: E^0, H^{1/2} = the exact particular solution the sources drive (omega^2 must
 *   differ from pi^2 (m^2 + n^2)):
 *     E_z = A cos(omega t) sin(pi m x) sin(pi n y),  A = Z amp omega / (omega^2 - pi^2 (m^2 + n^2)),
 *     H_x = -(A pi n / (Z omega)) sin(omega t) sin(pi m x) cos(pi n y),
 *     H_y =  (A pi m / (Z omega)) sin(omega t) cos(pi m x) sin(pi n y);  step counter 0.
 * ms_error_vs_driven: as ms_error_vs_exact against that solution at t_E = n h_tau, t_H = (n+1/2) h_tau. */
typedef struct {
  int m, n;
  double amp, omega;
} ms_source;
ms_status ms_set_sources(ms_grid* g, const ms_source* src, int nsrc);
ms_status ms_init_driven(ms_grid* g, const ms_source* src, int nsrc);
ms_status ms_error_vs_driven(ms_grid* g, const ms_source* src, int nsrc, double* l2_abs, double* l2_rel,
                             double* max_abs, double* sum_abs);

/* Sources with sine or cosine profiles:
 *   J_z = amp X(pi m x) Y(pi n y) sin(omega t),  X = sin (cos_x = 0, m >= 1) or cos (cos_x = 1, m >= 0),
 * Y likewise with cos_y and n.  A cosine profile does not vanish on the walls, and the Neumann data of
 * Sec. 3.3 become inhomogeneous; they are discretised by Method 2 of Sec. 3.3 (the Taylor ghost of
 * Eq. "eq:gst2"), with the wall data from Ampere's law on the PEC walls:
 *   on x = 0, 1:  d_x H_y = J_z,   d_xxx H_y = (d_tt + d_xx - d_yy) J_z;
 *   on y = 0, 1:  d_y H_x = -J_z,  d_yyy H_x = -(d_tt + d_yy - d_xx) J_z;
 * the H filter of Step 1 takes the ghosts of H^{n+1/2}, the H solves of Step 2 those of
 * H* = (H^{n+3/2} - H^{n+1/2}) / h_tau, and G_E on the boundary nodes is (h^2/12) Z d_t J_z at t^{n+1}
 * (Delta E_z = Z d_t J_z on a PEC wall).  The data must be compatible at the corners (J_z = 0 there,
 * since H.n = 0 on both walls); ghost values at the corner points are not used.
 * ms_set_sources_xy: replaces the grid's sources like ms_set_sources (rows with cos_x = cos_y = 0 are
 *   exactly ms_set_sources rows).  Rows with a cosine profile need MS_CLOSURE_PAPER (the REFLECT
 *   rows assume even data at the walls): MS_EUNSUPPORTED otherwise; both precisions (FP32_REFINED
 *   adds the wall terms to its right-hand sides as their Pade responses); MS_EINVAL for an index
 *   below its minimum or a flag other than 0 / 1.  Initial data come from ms_set_fields. */
typedef struct {
  int m, n;
  int cos_x, cos_y;
  double amp, omega;
} ms_source_xy;
ms_status ms_set_sources_xy(ms_grid* g, const ms_source_xy* src, int nsrc);

/* ---------------------------------------------------------------------------------------
 * Initial data that is not a cavity mode, and the reverse (adjoint) pass.
 *
 * ms_taylor_init sets E_z^0 = ez0 (boundary entries ignored, stored as zero) and H^{1/2} by the
 * Taylor series of Sec. 5.1 (Eq. "talorh") with H^0 = 0 and J = 0:
 *   H^{1/2} = Z^{-1} (t1 + (t1^3/6) Delta_h) (-delta_y E^0, delta_x E^0),  t1 = h_tau / 2,
 * with delta the node -> half-node Pade derivative of App. A.1 and Delta_h the 5-point Laplacian
 * with the ghost rules of Table "tab:bc" (the discrete reading of the continuous curl and
 * Laplacian in the series).  The step counter is reset to 0.  ez0: (N+1)^2 FP64, host (or
 * device for _device).
 *
 * The step is linear in the state, so a misfit L(E_z^K) has dL/dE_z^0 = T0^T (M^T)^K dL/dE_z^K,
 * with M the matrix of one step (Sec. 3.4, Step 1 then Step 2) on the unknowns and T0 the
 * map E^0 -> (E^0, H^{1/2}) above.  The paper has no reverse pass; this is its exact transpose:
 *   Step 2^T:  u_H = P1_H^{-1} l_H,  l_E += h_tau F_E (kappa^2/Z) (delta_x^T u_y - delta_y^T u_x)
 *   Step 1^T:  u_E = P1_E^{-1} l_E,  l_H += h_tau F_H kappa^2 Z (-delta_y^T u_E, delta_x^T u_E)
 * (F the right-hand-side filter of Eq. "eq:ell", symmetric like P1 on the unknowns; delta^T
 * the transpose of the truncated Pade band the forward kernels apply).  Because the step does
 * not depend on the state, the reverse pass reads no forward trajectory: no checkpoints are
 * stored and memory is that of one state.  The reverse pass computes in FP64 on both
 * precisions (on an MS_FP32_REFINED grid it is the transpose of the exact step, which the
 * refined forward reproduces to its stated accuracy).  It leaves the forward state untouched.
 *
 * ms_adjoint_run:  dL_dEz0 = T0^T (M^T)^nsteps (dL_dEzT, 0, 0): the gradient with respect to
 *   E_z^0 of a loss of E_z after nsteps steps from ms_taylor_init data, given its gradient
 *   dL_dEzT.  Both (N+1)^2 FP64; boundary entries of dL_dEzT are ignored and those of dL_dEz0
 *   are zero.  Host arrays: synchronous.  _device: device arrays, asynchronous on the grid's
 *   stream.
 * ms_adjoint_steps: lam (3 arrays in the full layout of comps) <- (M^T)^nsteps lam, in place;
 *   boundary entries are zeroed.  Host arrays: synchronous.  _device: asynchronous.
 * ms_taylor_init_T: dEz0 = T0_H^T (l_Hx, l_Hy), the transpose of the H^{1/2} part of T0. */
ms_status ms_taylor_init(ms_grid* g, const double* ez0);
ms_status ms_taylor_init_device(ms_grid* g, const double* ez0);
ms_status ms_adjoint_run(ms_grid* g, long nsteps, const double* dL_dEzT, double* dL_dEz0);
ms_status ms_adjoint_run_device(ms_grid* g, long nsteps, const double* dL_dEzT, double* dL_dEz0);
ms_status ms_adjoint_steps(ms_grid* g, long nsteps, double* const* lam);
ms_status ms_adjoint_steps_device(ms_grid* g, long nsteps, double* const* lam);
ms_status ms_taylor_init_T(ms_grid* g, const double* l_hx, const double* l_hy, double* dEz0);

/* Arithmetic of the reverse pass: MS_FP64 (every grid), or MS_FP32_REFINED (FP32_REFINED grids,
 * their default).  The FP32 reverse pass keeps the adjoint state as float-float pairs and is the
 * transpose of the FP32_REFINED forward operator (its truncated Pade tables): the adjoint solve
 * u = P1^{-1} l returns its last Richardson iterate and correction as a pair, the transposed band
 * W^T u is accumulated in float-float, and only the difference D^T W^T u (the transposed Pade
 * derivative) is rounded to FP32, so a smooth adjoint field loses no accuracy to cancellation.
 * ms_adjoint_run / _steps convert at the FP64 interface; the Taylor transpose stays FP64.
 * MS_EINVAL for an unknown precision, MS_EUNSUPPORTED for FP32 on an FP64 grid. */
ms_status ms_set_adjoint_precision(ms_grid* g, int precision);

/* ---------------------------------------------------------------------------------------
 * Batches: many independent 2D cavities of uneven sizes advanced together.  Each cavity is the
 * problem of ms_create_grid with n = n[b] cells per side; all share the rest of the descriptor
 * (z_imp, r, precision, closure, scheme, stream).  Every kernel of a step is one launch for the
 * whole batch (its blocks walk a list of (cavity, tile) entries), and ms_batch_run replays a
 * captured CUDA graph.  Requires MS_FP32_REFINED and MS_SCHEME_C4 (MS_EUNSUPPORTED otherwise).
 * Cavity indices are 0 .. count-1; the per-cavity calls behave like their ms_* counterparts. */
typedef struct ms_batch ms_batch;
ms_status ms_create_batch(const ms_grid_desc* desc, const int* n, int count, ms_batch** out);
ms_status ms_batch_destroy(ms_batch* b);
ms_status ms_batch_init_modes(ms_batch* b, int cavity, const ms_mode* modes, int nmodes);
ms_status ms_batch_set_fields(ms_batch* b, int cavity, const double* const* comps, long step);
ms_status ms_batch_get_fields(ms_batch* b, int cavity, double* const* comps);
ms_status ms_batch_step(ms_batch* b);
ms_status ms_batch_run(ms_batch* b, long nsteps);
ms_status ms_batch_sync(ms_batch* b);
ms_status ms_batch_error_vs_exact(ms_batch* b, int cavity, const ms_mode* modes, int nmodes, double* l2_abs,
                                  double* l2_rel, double* max_abs, double* sum_abs);
/* count: cavities; cells: sum of n[b]^2 (Yee cells advanced per step); launches: kernels per step. */
ms_status ms_batch_info(ms_batch* b, int* count, long long* cells, int* launches);

/* Launch plan of a batch: plan[0] = work-list order (0: cavity by cavity, tiles row by row; 1: the
 * boundary-ring tiles of every cavity first, since they take the general and slower paths; 2:
 * largest cavities first), plan[1] = steps per captured graph in ms_batch_run (1..256), plan[2] = 1
 * for persistent launches (as many blocks as are resident at once, each striding over the work
 * list), 0 for one block per work item.  Every plan runs exactly the same arithmetic per cavity;
 * only the order and the launch shape change.  The default is {0, 16, 0}.  ms_batch_set_plan drops
 * the captured graphs (MS_EINVAL for an invalid plan).
 *
 * ms_batch_autotune: chooses the plan by measurement.  Candidates: orders 0..2 x 8 or 32 steps per
 * graph x persistent or not; each is captured and timed with CUDA events over about trial_steps
 * steps (1..4096), and the fastest per step is applied.  The trials step the batch's current state,
 * so the call must come before any cavity's fields are set (the state is then zero and stays zero;
 * MS_EINVAL otherwise); step counters are not advanced.  The choice is cached under a key of the
 * cavity sizes, r, Z, closure and the device (SM count and name): in memory for the process, and
 * appended to the file named by the environment variable MS_AUTOTUNE_CACHE if it is set, so a later
 * process with the same key reuses it without trials.  plan (3 ints, may be NULL) receives the
 * applied plan, *from_cache (may be NULL) whether it came from the cache.  Synchronous.
 *
 * The cache itself (host only, no GPU needed): keys of 1..512 characters from [A-Za-z0-9:;._-=,];
 * ms_autotune_cache_get sets *found and, if found, plan (memory first, then the cache file, whose
 * last line for a key wins); ms_autotune_cache_put stores a valid plan in memory and appends it to
 * the file (MS_EINVAL if the file cannot be written); ms_autotune_cache_clear empties the memory
 * copy (the file stays). */
ms_status ms_batch_set_plan(ms_batch* b, const int* plan);
ms_status ms_batch_get_plan(ms_batch* b, int* plan);
ms_status ms_batch_autotune(ms_batch* b, int trial_steps, int* plan, int* from_cache);
ms_status ms_autotune_cache_get(const char* key, int* plan, int* found);
ms_status ms_autotune_cache_put(const char* key, const int* plan);
ms_status ms_autotune_cache_clear(void);

/* Checkpoint / resume (the paper has none).  ms_save writes the grid's state (the fields in their
 * working representation: FP64 arrays, or the exact FP32 hi and lo arrays of MS_FP32_REFINED, plus
 * the tracked Delta E_z of MS_SCHEME_C4_DE), its step counter and its descriptor to `path`;
 * ms_load restores them into a grid created with the same dim, n, precision, closure, scheme,
 * z_imp and r (MS_EINVAL otherwise, or for a file that is not a checkpoint), so a resumed run is
 * bit-identical to an uninterrupted one.  Sources are configuration, not state, and are not
 * saved.  Little-endian raw format described in ckpt.cu.  Synchronous; not for batch cavities. */
ms_status ms_save(ms_grid* g, const char* path);
ms_status ms_load(ms_grid* g, const char* path);

/* Message of the last failed call on this thread ("" if none). */
const char* ms_last_error(void);

/* Test hooks for the failure paths (host side; no device work).  ms_debug_fail_alloc(n) makes the
 * n-th device allocation the library makes from now on fail as an out-of-memory device would
 * (nothing is allocated; the call reports MS_ENOMEM, or the status of the operation that needed
 * the memory), then disarms itself; n = 0 disarms, n < 0 is MS_EINVAL.  ms_debug_live_allocs
 * returns the number of device allocations the library holds, so a test can check that a failed
 * creation released everything.  Process-wide, not thread-safe against concurrent creations. */
ms_status ms_debug_fail_alloc(int n);
long ms_debug_live_allocs(void);

#ifdef __cplusplus
}
#endif
#endif /* MAXWELL4_H */
