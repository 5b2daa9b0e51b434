/*
 * Plain FP64 CPU oracle of the compact fourth-order staggered scheme for the
 * first-order Maxwell equations (Versano, Turkel & Tsynkov, arXiv 2306.17263).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the scheme computes.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  The CUDA library in
 * paper_2306_17263_gb300/ never calls, links or includes anything from here,
 * and nothing here is shared with it.
 *
 * Every routine is written straight from the paper's definitions, with no
 * blocking, fusion or reordering beyond them:
 *   - meshes and PEC boundary values: Sec. 2, Eq. (2.1) "eq:meshes", "eq:bc_E=0";
 *   - Dirichlet / Neumann type of each time derivative: Table "tab:bc";
 *   - compact modified-Helmholtz scheme: Sec. 3.2, Eq. "eq:ell";
 *   - operators P1, P2: Definition "def:operatorsP" and App. A.2;
 *   - even ghost reflection for homogeneous Neumann: Corollary "cor:ghost_cor";
 *   - Pade first derivative A f' = D1 f / h: App. A.1, Eq. "eq:lhs";
 *   - D2 and the Kronecker lifts D_xx, D_yy: App. A.1;
 *   - the time step (Step 1 then Step 2): Sec. 3.4;
 *   - conjugate-gradient solves of the SPD systems: Sec. 3.2 and Sec. 6;
 *   - exact PEC cavity modes and the mean absolute error: Sec. 5.1, Eq. "eq:data";
 *   - Yee updating rules with the second-order stencil (c=1): Sec. 5.2;
 *   - the non-compact fourth-order comparator NC (stencil K4, a = 0, one-sided
 *     fourth-order differences at the line ends): Sec. 5.2, Eq. "eq:K4";
 *   - current sources J_z: the source terms of the Taylor expansion of Sec. 3.1, and for
 *     currents that do not vanish on the walls the Taylor ghosts of Method 2, Sec. 3.3,
 *     Eq. "eq:gst2" (readings at or2d_wall_ghosts).
 *
 * Readings of points the paper leaves open:
 *   - the third rows of Step 1 / Step 2 are E_z and H_z (the printed E_y, H_y
 *     rows are typos);
 *   - the Laplacian inside the right-hand-side filter is Delta_h for both
 *     half-steps (the form analysed in Sec. 4);
 *   - the filter is applied on the source grid and then the Pade curl;
 *   - closure PAPER uses the one-sided rows [26,-5,4,-1]/24 of Eq. "eq:lhs" at
 *     both ends of every Pade system; closure REFLECT replaces them by the rows
 *     that follow from the field's parity about the wall (see pade_row);
 *   - G_E = 0 on the PEC boundary nodes (E_z = 0 and Delta E_z = d_tt E_z = 0), and
 *     (h^2/12) Z d_t J_z there when a current does not vanish on the wall;
 *   - boundary values of the Dirichlet components are held at zero.
 *
 * Array layout (2D TM_z, N cells per side, h = 1/N): row-major [y][x].
 *   E_z : (N+1) x (N+1) at (x_i, y_j)           Dirichlet in x and y
 *   H_x : N rows x (N+1) cols at (x_i, y_{j+1/2}) Dirichlet in x, Neumann in y
 *   H_y : (N+1) rows x N cols at (x_{i+1/2}, y_j) Neumann in x, Dirichlet in y
 * 3D: array [z][y][x]; the six components follow Eq. "eq:meshes".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { BC_DIR = 0, BC_NEU = 1 };
enum { CLOSURE_PAPER = 0, CLOSURE_REFLECT = 1 };
/* Pade direction: HALF_TO_NODE maps N half-node values to the N-1 interior
 * nodes; NODE_TO_HALF maps the N+1 node values to the N half-nodes. */
enum { HALF_TO_NODE = 0, NODE_TO_HALF = 1 };
enum { F_EZ = 0, F_HX = 1, F_HY = 2 };

typedef struct {
  int N;
  double r, Z, h, ht, kappa2, beta, c1;
  int closure;
  double cg_tol;
  int cg_maxit;
  long cg_iters_total; /* CG iterations summed over all solves since setup */
  long cg_solves;
} or_grid2d;

/* ------------------------------------------------------------------ */
/* Grid constants: h = 1/N, h_tau = r h, kappa^2 = 24 / h_tau^2 (Sec. 3.2),
 * beta = 1 + kappa^2 h^2 / 12 = 1 + 2/r^2, c1 = kappa^2 beta (Def. "def:operatorsP"). */
void or2d_setup(or_grid2d* g, int N, double r, double Z, int closure) {
  g->N = N;
  g->r = r;
  g->Z = Z;
  g->h = 1.0 / N;
  g->ht = r * g->h;
  g->kappa2 = 24.0 / (g->ht * g->ht);
  g->beta = 1.0 + g->kappa2 * g->h * g->h / 12.0;
  g->c1 = g->kappa2 * g->beta;
  g->closure = closure;
  g->cg_tol = 1e-14;
  g->cg_maxit = 200;
  g->cg_iters_total = 0;
  g->cg_solves = 0;
}

void or2d_set_cg(or_grid2d* g, double tol, int maxit) {
  g->cg_tol = tol;
  g->cg_maxit = maxit;
}

/* Field shapes and boundary types (Eq. "eq:meshes", Table "tab:bc"). */
static void field_dims(const or_grid2d* g, int f, int* nx, int* ny, int* bcx, int* bcy) {
  int N = g->N;
  if (f == F_EZ) { *nx = N + 1; *ny = N + 1; *bcx = BC_DIR; *bcy = BC_DIR; }
  else if (f == F_HX) { *nx = N + 1; *ny = N; *bcx = BC_DIR; *bcy = BC_NEU; }
  else { *nx = N; *ny = N + 1; *bcx = BC_NEU; *bcy = BC_DIR; }
}

int or2d_field_size(const or_grid2d* g, int f) {
  int nx, ny, bx, by;
  field_dims(g, f, &nx, &ny, &bx, &by);
  return nx * ny;
}

/* interior test on one axis: Dirichlet axes (N+1 nodes) exclude 0 and N */
static int axis_interior(int bc, int i, int n) {
  return bc == BC_NEU ? 1 : (i > 0 && i < n - 1);
}

/* ------------------------------------------------------------------ */
/* 1D Pade row coefficients, App. A.1 Eq. "eq:lhs" (scaled by 24).
 * Row i of the M x M matrix 24*A.  Writes up to 4 (col, value) pairs.
 *  interior rows: [1, 22, 1];
 *  PAPER closure: first row [26,-5,4,-1], last row [-1,4,-5,26];
 *  REFLECT closure: NODE_TO_HALF first/last rows [23,1] / [1,23] (the derivative of a
 *  field that vanishes at the wall is even about it); HALF_TO_NODE first/last rows
 *  [22,1] / [1,22] (the derivative of a field that is even about the wall is zero there). */
static int pade_row(int M, int closure, int kind, int i, int* col, double* val) {
  int n = 0;
  if (i == 0 || i == M - 1) {
    int first = (i == 0);
    if (closure == CLOSURE_PAPER) {
      static const double rowc[4] = {26.0, -5.0, 4.0, -1.0};
      for (int k = 0; k < 4; ++k) {
        col[n] = first ? k : M - 1 - k;
        val[n] = rowc[k];
        ++n;
      }
      return n;
    } else {
      double d = (kind == NODE_TO_HALF) ? 23.0 : 22.0;
      col[n] = i; val[n] = d; ++n;
      col[n] = first ? i + 1 : i - 1; val[n] = 1.0; ++n;
      return n;
    }
  }
  col[n] = i - 1; val[n] = 1.0; ++n;
  col[n] = i; val[n] = 22.0; ++n;
  col[n] = i + 1; val[n] = 1.0; ++n;
  return n;
}

/* Solve (24 A) y = rhs for one line by banded Gaussian elimination without
 * pivoting (A is strictly diagonally dominant by rows).  Band half-width 3. */
#define PB 3
static void pade_solve24(int M, int closure, int kind, double* rhs, double* y) {
  /* band[i][k] holds entry (i, i - PB + k), k in [0, 2 PB] */
  double* band = (double*)calloc((size_t)M * (2 * PB + 1), sizeof(double));
  for (int i = 0; i < M; ++i) {
    int col[4];
    double val[4];
    int n = pade_row(M, closure, kind, i, col, val);
    for (int k = 0; k < n; ++k) band[(size_t)i * (2 * PB + 1) + (col[k] - i + PB)] += val[k];
  }
  for (int k = 0; k < M; ++k) {
    double piv = band[(size_t)k * (2 * PB + 1) + PB];
    for (int i = k + 1; i <= k + PB && i < M; ++i) {
      double* ri = band + (size_t)i * (2 * PB + 1);
      double* rk = band + (size_t)k * (2 * PB + 1);
      double a = ri[k - i + PB];
      if (a == 0.0) continue;
      double l = a / piv;
      for (int j = k; j <= k + PB && j < M; ++j) ri[j - i + PB] -= l * rk[j - k + PB];
      rhs[i] -= l * rhs[k];
    }
  }
  for (int i = M - 1; i >= 0; --i) {
    double* ri = band + (size_t)i * (2 * PB + 1);
    double s = rhs[i];
    for (int j = i + 1; j <= i + PB && j < M; ++j) s -= ri[j - i + PB] * y[j];
    y[i] = s / ri[PB];
  }
  free(band);
}

/* Pade derivative of one line: f has M+1 samples, fp receives M derivative values,
 * A fp = D1 f / h (Eq. "eq:lhs"; D1 is the (M) x (M+1) two-point difference). */
void or_pade_line(int M, int closure, int kind, double h, const double* f, double* fp) {
  double* rhs = (double*)malloc(sizeof(double) * M);
  for (int i = 0; i < M; ++i) rhs[i] = 24.0 * (f[i + 1] - f[i]) / h;
  pade_solve24(M, closure, kind, rhs, fp);
  free(rhs);
}

/* Apply 24*A (the matrix of Eq. "eq:lhs" times 24) to a vector: used by tests. */
void or_pade_matvec24(int M, int closure, int kind, const double* y, double* out) {
  for (int i = 0; i < M; ++i) {
    int col[4];
    double val[4];
    int n = pade_row(M, closure, kind, i, col, val);
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += val[k] * y[col[k]];
    out[i] = s;
  }
}

/* ------------------------------------------------------------------ */
/* D_2 along one axis (App. A.1) of a field with its boundary type:
 * Dirichlet axes use the stored zeros at nodes 0 and N; Neumann axes use the
 * even ghosts u(-1) = u(0), u(n) = u(n-1) (Corollary "cor:ghost_cor").
 * Result is written at interior points and set to 0 at Dirichlet boundary points. */
static void d2_axis(const or_grid2d* g, int f, int axis, const double* u, double* out) {
  int nx, ny, bx, by;
  field_dims(g, f, &nx, &ny, &bx, &by);
  double ih2 = 1.0 / (g->h * g->h);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t p = (size_t)j * nx + i;
      if (!axis_interior(bx, i, nx) || !axis_interior(by, j, ny)) { out[p] = 0.0; continue; }
      double um, up;
      if (axis == 0) {
        um = (i - 1 >= 0) ? u[p - 1] : u[p];            /* i-1 < 0 only on Neumann axes */
        up = (i + 1 < nx) ? u[p + 1] : u[p];
      } else {
        um = (j - 1 >= 0) ? u[p - nx] : u[p];
        up = (j + 1 < ny) ? u[p + nx] : u[p];
      }
      out[p] = (um - 2.0 * u[p] + up) * ih2;
    }
}

/* Delta_h = D_xx + D_yy (Sec. 3.2). */
void or2d_laplacian(const or_grid2d* g, int f, const double* u, double* out) {
  int n = or2d_field_size(g, f);
  double* t = (double*)malloc(sizeof(double) * n);
  d2_axis(g, f, 0, u, out);
  d2_axis(g, f, 1, u, t);
  for (int p = 0; p < n; ++p) out[p] += t[p];
  free(t);
}

/* Right-hand-side filter of Eq. "eq:ell": G = (1 + kappa^2 h^2/12) u + (h^2/12) Delta_h u,
 * written on interior points, 0 on Dirichlet boundary points. */
void or2d_filter(const or_grid2d* g, int f, const double* u, double* G) {
  int nx, ny, bx, by;
  field_dims(g, f, &nx, &ny, &bx, &by);
  int n = nx * ny;
  or2d_laplacian(g, f, u, G);
  double h2_12 = g->h * g->h / 12.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t p = (size_t)j * nx + i;
      if (!axis_interior(bx, i, nx) || !axis_interior(by, j, ny)) G[p] = 0.0;
      else G[p] = g->beta * u[p] + h2_12 * G[p];
    }
  (void)n;
}

/* P1 = -(D_xx + D_yy + (h^2/6) D_xx D_yy) + c1 (Def. "def:operatorsP", 2D: Upsilon_h = D_xx D_yy).
 * Applied as the Kronecker composition of App. A.1. */
void or2d_p1_apply(const or_grid2d* g, int f, const double* x, double* y) {
  int n = or2d_field_size(g, f);
  double* dxx = (double*)malloc(sizeof(double) * n);
  double* dyy = (double*)malloc(sizeof(double) * n);
  double* dxxdyy = (double*)malloc(sizeof(double) * n);
  d2_axis(g, f, 0, x, dxx);
  d2_axis(g, f, 1, x, dyy);
  d2_axis(g, f, 0, dyy, dxxdyy);
  int nx, ny, bx, by;
  field_dims(g, f, &nx, &ny, &bx, &by);
  double h2_6 = g->h * g->h / 6.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t p = (size_t)j * nx + i;
      if (!axis_interior(bx, i, nx) || !axis_interior(by, j, ny)) { y[p] = 0.0; continue; }
      y[p] = g->c1 * x[p] - (dxx[p] + dyy[p] + h2_6 * dxxdyy[p]);
    }
  free(dxx);
  free(dyy);
  free(dxxdyy);
}

/* P2 = (24/h_tau^2)(-1 - 2/r^2 - (h^2/12) Delta_h) (Def. "def:operatorsP"). */
void or2d_p2_apply(const or_grid2d* g, int f, const double* x, double* y) {
  int nx, ny, bx, by;
  field_dims(g, f, &nx, &ny, &bx, &by);
  or2d_laplacian(g, f, x, y);
  double k = 24.0 / (g->ht * g->ht), b = 1.0 + 2.0 / (g->r * g->r), h2_12 = g->h * g->h / 12.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t p = (size_t)j * nx + i;
      if (!axis_interior(bx, i, nx) || !axis_interior(by, j, ny)) y[p] = 0.0;
      else y[p] = k * (-b * x[p] - h2_12 * y[p]);
    }
}

static double dot_interior(const or_grid2d* g, int f, const double* a, const double* b) {
  int n = or2d_field_size(g, f);
  double s = 0.0;
  for (int p = 0; p < n; ++p) s += a[p] * b[p]; /* boundary entries are zero */
  return s;
}

/* Conjugate gradients for P1 x = b (the paper's solver, Sec. 3.2 and Sec. 6),
 * started from x = 0, stopped when ||r||_2 <= tol ||b||_2.  Returns iterations. */
int or2d_p1_solve_cg(or_grid2d* g, int f, const double* b, double* x) {
  int n = or2d_field_size(g, f);
  double* r = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  double* Ap = (double*)malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; p[i] = b[i]; }
  double bb = dot_interior(g, f, b, b), rr = bb;
  int it = 0;
  if (bb > 0.0) {
    while (it < g->cg_maxit && rr > g->cg_tol * g->cg_tol * bb) {
      or2d_p1_apply(g, f, p, Ap);
      double alpha = rr / dot_interior(g, f, p, Ap);
      for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; }
      double rr2 = dot_interior(g, f, r, r);
      double beta = rr2 / rr;
      for (int i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
      rr = rr2;
      ++it;
    }
  }
  g->cg_iters_total += it;
  g->cg_solves += 1;
  free(r);
  free(p);
  free(Ap);
  return it;
}

/* ------------------------------------------------------------------ */
/* Pade derivative of a whole field along an axis (App. A.1, delta_s = a_s^{-1} D_s).
 * src is a field of type fs, dst a field of type fd.  HALF_TO_NODE: the axis of src is
 * Neumann type (N half-nodes) and dst's is Dirichlet type (values at nodes 1..N-1, 0 at
 * the boundary nodes).  NODE_TO_HALF: the reverse (N+1 nodes -> N half-nodes).
 * Lines of the other axis are copied index for index (same extent in both fields). */
static void pade_field(const or_grid2d* g, int fs, int fd, int axis, int kind, const double* src, double* dst) {
  int snx, sny, sbx, sby, dnx, dny, dbx, dby;
  field_dims(g, fs, &snx, &sny, &sbx, &sby);
  field_dims(g, fd, &dnx, &dny, &dbx, &dby);
  int N = g->N;
  int M = (kind == HALF_TO_NODE) ? N - 1 : N;
  int nl = (axis == 0) ? sny : snx;  /* number of lines */
  double* f = (double*)malloc(sizeof(double) * (M + 1));
  double* fp = (double*)malloc(sizeof(double) * M);
  memset(dst, 0, sizeof(double) * (size_t)dnx * dny);
  for (int l = 0; l < nl; ++l) {
    for (int k = 0; k <= M; ++k) f[k] = (axis == 0) ? src[(size_t)l * snx + k] : src[(size_t)k * snx + l];
    or_pade_line(M, g->closure, kind, g->h, f, fp);
    for (int k = 0; k < M; ++k) {
      int o = (kind == HALF_TO_NODE) ? k + 1 : k; /* derivative at node k+1, or half-node k */
      if (axis == 0) dst[(size_t)l * dnx + o] = fp[k];
      else dst[(size_t)o * dnx + l] = fp[k];
    }
  }
  free(f);
  free(fp);
}

/* Zero the Dirichlet boundary points of a field. */
static void zero_boundary(const or_grid2d* g, int f, double* u) {
  int nx, ny, bx, by;
  field_dims(g, f, &nx, &ny, &bx, &by);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (!axis_interior(bx, i, nx) || !axis_interior(by, j, ny)) u[(size_t)j * nx + i] = 0.0;
}

/* Step 1 right-hand side (Sec. 3.4): R_E = kappa^2 Z (delta_x G_y - delta_y G_x),
 * with G_x, G_y the filtered H fields (third row of curl_h, App. A.1). */
void or2d_curl_h_to_e(const or_grid2d* g, const double* Gx, const double* Gy, double* R) {
  int n = or2d_field_size(g, F_EZ);
  double* a = (double*)malloc(sizeof(double) * n);
  double* b = (double*)malloc(sizeof(double) * n);
  pade_field(g, F_HY, F_EZ, 0, HALF_TO_NODE, Gy, a); /* delta_x G_y */
  pade_field(g, F_HX, F_EZ, 1, HALF_TO_NODE, Gx, b); /* delta_y G_x */
  for (int p = 0; p < n; ++p) R[p] = g->kappa2 * g->Z * (a[p] - b[p]);
  zero_boundary(g, F_EZ, R);
  free(a);
  free(b);
}

/* Step 2 right-hand side (Sec. 3.4): -(kappa^2/Z) curl_h G_E restricted to TM_z:
 * R_x = -(kappa^2/Z) delta_y G_E, R_y = +(kappa^2/Z) delta_x G_E. */
void or2d_curl_e_to_h(const or_grid2d* g, const double* GE, double* Rx, double* Ry) {
  int nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  pade_field(g, F_EZ, F_HX, 1, NODE_TO_HALF, GE, Rx); /* delta_y G_E */
  pade_field(g, F_EZ, F_HY, 0, NODE_TO_HALF, GE, Ry); /* delta_x G_E */
  double s = g->kappa2 / g->Z;
  for (int p = 0; p < nx_; ++p) Rx[p] *= -s;
  for (int p = 0; p < ny_; ++p) Ry[p] *= s;
  zero_boundary(g, F_HX, Rx);
  zero_boundary(g, F_HY, Ry);
}

/* The H increment of Step 2 for a given E: P1^{H} H* = R_H(E).  hxs, hys receive H*. */
void or2d_h_increment(or_grid2d* g, const double* ez, double* hxs, double* hys) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* GE = (double*)malloc(sizeof(double) * ne);
  double* Rx = (double*)malloc(sizeof(double) * nx_);
  double* Ry = (double*)malloc(sizeof(double) * ny_);
  or2d_filter(g, F_EZ, ez, GE);
  or2d_curl_e_to_h(g, GE, Rx, Ry);
  or2d_p1_solve_cg(g, F_HX, Rx, hxs);
  or2d_p1_solve_cg(g, F_HY, Ry, hys);
  free(GE);
  free(Rx);
  free(Ry);
}

/* One full time step (Sec. 3.4, Step 1 then Step 2), J = rho = 0:
 *   P1^{E} E* = kappa^2 Z curl_h[(1 + kappa^2 h^2/12) H + (h^2/12) Delta_h H],  E += h_tau E*;
 *   P1^{H} H* = -(kappa^2/Z) curl_h[(1 + kappa^2 h^2/12) E + (h^2/12) Delta_h E], H += h_tau H*. */
void or2d_step(or_grid2d* g, double* ez, double* hx, double* hy) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* Gx = (double*)malloc(sizeof(double) * nx_);
  double* Gy = (double*)malloc(sizeof(double) * ny_);
  double* R = (double*)malloc(sizeof(double) * ne);
  double* Es = (double*)malloc(sizeof(double) * ne);
  double* Hxs = (double*)malloc(sizeof(double) * nx_);
  double* Hys = (double*)malloc(sizeof(double) * ny_);
  or2d_filter(g, F_HX, hx, Gx);
  or2d_filter(g, F_HY, hy, Gy);
  or2d_curl_h_to_e(g, Gx, Gy, R);
  or2d_p1_solve_cg(g, F_EZ, R, Es);
  for (int p = 0; p < ne; ++p) ez[p] += g->ht * Es[p];
  or2d_h_increment(g, ez, Hxs, Hys);
  for (int p = 0; p < nx_; ++p) hx[p] += g->ht * Hxs[p];
  for (int p = 0; p < ny_; ++p) hy[p] += g->ht * Hys[p];
  free(Gx);
  free(Gy);
  free(R);
  free(Es);
  free(Hxs);
  free(Hys);
}

/* ------------------------------------------------------------------ */
/* Exact PEC cavity modes (Sec. 5.1, Eq. "eq:data"), superposed.  modes[3m..3m+2] =
 * (k_x, k_y, amplitude).  omega = pi sqrt(k_x^2 + k_y^2); for general Z the H fields
 * carry 1/Z (Faraday's law, Eq. "maxh").  E at time tE, H at time tH. */
void or2d_exact(const or_grid2d* g, const double* modes, int nmodes, double tE, double tH, double* ez,
                double* hx, double* hy) {
  int N = g->N;
  double h = g->h, pi = M_PI;
  memset(ez, 0, sizeof(double) * (N + 1) * (N + 1));
  memset(hx, 0, sizeof(double) * N * (N + 1));
  memset(hy, 0, sizeof(double) * N * (N + 1));
  for (int m = 0; m < nmodes; ++m) {
    double kx = modes[3 * m], ky = modes[3 * m + 1], A = modes[3 * m + 2];
    double w = pi * sqrt(kx * kx + ky * ky);
    double ce = A * cos(w * tE), sh = A * sin(w * tH) / (w * g->Z);
    for (int j = 1; j < N; ++j)
      for (int i = 1; i < N; ++i)
        ez[(size_t)j * (N + 1) + i] += ce * sin(pi * kx * i * h) * sin(pi * ky * j * h);
    for (int j = 0; j < N; ++j)
      for (int i = 1; i < N; ++i)
        hx[(size_t)j * (N + 1) + i] += -sh * pi * ky * sin(pi * kx * i * h) * cos(pi * ky * (j + 0.5) * h);
    for (int j = 1; j < N; ++j)
      for (int i = 0; i < N; ++i)
        hy[(size_t)j * N + i] += sh * pi * kx * cos(pi * kx * (i + 0.5) * h) * sin(pi * ky * j * h);
  }
}

/* Error of the state against the exact modes at t_E = n h_tau, t_H = (n + 1/2) h_tau.
 * out[0] = L2 abs = sqrt(h^2 sum (u - u_ex)^2) over the three fields, out[1] = L2 rel,
 * out[2] = max abs, out[3] = sum |u - u_ex| (the summand of the mean absolute error, Sec. 5.1). */
void or2d_error(const or_grid2d* g, const double* modes, int nmodes, double tE, double tH, const double* ez,
                const double* hx, const double* hy, double* out) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* e = (double*)malloc(sizeof(double) * ne);
  double* a = (double*)malloc(sizeof(double) * nx_);
  double* b = (double*)malloc(sizeof(double) * ny_);
  or2d_exact(g, modes, nmodes, tE, tH, e, a, b);
  double s2 = 0.0, r2 = 0.0, mx = 0.0, s1 = 0.0;
  const double* num[3] = {ez, hx, hy};
  const double* ex[3] = {e, a, b};
  int sz[3] = {ne, nx_, ny_};
  for (int f = 0; f < 3; ++f)
    for (int p = 0; p < sz[f]; ++p) {
      double d = num[f][p] - ex[f][p];
      s2 += d * d;
      r2 += ex[f][p] * ex[f][p];
      s1 += fabs(d);
      if (fabs(d) > mx) mx = fabs(d);
    }
  double h2 = g->h * g->h;
  out[0] = sqrt(h2 * s2);
  out[1] = r2 > 0 ? sqrt(s2 / r2) : 0.0;
  out[2] = mx;
  out[3] = s1;
  free(e);
  free(a);
  free(b);
}

/* Discrete energy W^n = Z^{-1} ||E^n||_h^2 + Z <H^{n-1/2}, H^{n+1/2}>_h, with h^2-weighted sums.
 * (The paper is silent on a discrete energy; this is the leapfrog invariant of the scheme
 * written as in Sec. 4, Eq. "eq:eh".)  H^{n-1/2} = H^{n+1/2} - h_tau H*(E^n). */
double or2d_energy(or_grid2d* g, const double* ez, const double* hx, const double* hy) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* hxs = (double*)malloc(sizeof(double) * nx_);
  double* hys = (double*)malloc(sizeof(double) * ny_);
  or2d_h_increment(g, ez, hxs, hys);
  double se = 0.0, sh = 0.0;
  for (int p = 0; p < ne; ++p) se += ez[p] * ez[p];
  for (int p = 0; p < nx_; ++p) sh += (hx[p] - g->ht * hxs[p]) * hx[p];
  for (int p = 0; p < ny_; ++p) sh += (hy[p] - g->ht * hys[p]) * hy[p];
  free(hxs);
  free(hys);
  double h2 = g->h * g->h;
  return h2 * (se / g->Z + g->Z * sh);
}

/* Pade divergence of H on the N x N cell centres: div_h H = delta_x H_x + delta_y H_y
 * (App. A.1 delta operators, node -> half-node direction).  Returns sqrt(h^2 sum div^2). */
double or2d_divergence(const or_grid2d* g, const double* hx, const double* hy, double* div_out) {
  int N = g->N, M = N;
  double* f = (double*)malloc(sizeof(double) * (N + 1));
  double* fp = (double*)malloc(sizeof(double) * N);
  double* div = div_out ? div_out : (double*)malloc(sizeof(double) * N * N);
  for (int j = 0; j < N; ++j) { /* rows of H_x: nodes i = 0..N at y_{j+1/2} */
    for (int i = 0; i <= N; ++i) f[i] = hx[(size_t)j * (N + 1) + i];
    or_pade_line(M, g->closure, NODE_TO_HALF, g->h, f, fp);
    for (int i = 0; i < N; ++i) div[(size_t)j * N + i] = fp[i];
  }
  for (int i = 0; i < N; ++i) { /* columns of H_y: nodes j = 0..N at x_{i+1/2} */
    for (int j = 0; j <= N; ++j) f[j] = hy[(size_t)j * N + i];
    or_pade_line(M, g->closure, NODE_TO_HALF, g->h, f, fp);
    for (int j = 0; j < N; ++j) div[(size_t)j * N + i] += fp[j];
  }
  double s = 0.0;
  for (int p = 0; p < N * N; ++p) s += div[p] * div[p];
  free(f);
  free(fp);
  if (!div_out) free(div);
  return sqrt(g->h * g->h * s);
}

/* Run nsteps steps from (E^0, H^{1/2}); if modes != NULL, accumulate the mean-absolute-error
 * summand of Sec. 5.1 over steps n = 1..nsteps (errors of E^n and H^{n+1/2}).  Returns the
 * summand; mae = summand / (3 nsteps N^2). */
double or2d_run(or_grid2d* g, double* ez, double* hx, double* hy, int nsteps, const double* modes, int nmodes) {
  double acc = 0.0, e[4];
  for (int n = 1; n <= nsteps; ++n) {
    or2d_step(g, ez, hx, hy);
    if (modes) {
      or2d_error(g, modes, nmodes, n * g->ht, (n + 0.5) * g->ht, ez, hx, hy, e);
      acc += e[3];
    }
  }
  return acc;
}

/* ------------------------------------------------------------------ */
/* Plain second-order Yee step (Sec. 5.2 updating rules with stencil S, c = 1, a = b = d = 0):
 *   E_z += h_tau Z (D_x H_y - D_y H_x);  H_x -= (h_tau/Z) D_y E_z;  H_y += (h_tau/Z) D_x E_z. */
void or2d_yee_step(const or_grid2d* g, double* ez, double* hx, double* hy) {
  int N = g->N;
  double c = g->ht / g->h;
  for (int j = 1; j < N; ++j)
    for (int i = 1; i < N; ++i) {
      double dxhy = hy[(size_t)j * N + i] - hy[(size_t)j * N + i - 1];
      double dyhx = hx[(size_t)j * (N + 1) + i] - hx[(size_t)(j - 1) * (N + 1) + i];
      ez[(size_t)j * (N + 1) + i] += c * g->Z * (dxhy - dyhx);
    }
  for (int j = 0; j < N; ++j)
    for (int i = 1; i < N; ++i)
      hx[(size_t)j * (N + 1) + i] -= c / g->Z * (ez[(size_t)(j + 1) * (N + 1) + i] - ez[(size_t)j * (N + 1) + i]);
  for (int j = 1; j < N; ++j)
    for (int i = 0; i < N; ++i)
      hy[(size_t)j * N + i] += c / g->Z * (ez[(size_t)j * (N + 1) + i + 1] - ez[(size_t)j * (N + 1) + i]);
}

long or2d_cg_iters_total(const or_grid2d* g) { return g->cg_iters_total; }
long or2d_cg_solves(const or_grid2d* g) { return g->cg_solves; }
int or2d_sizeof(void) { return (int)sizeof(or_grid2d); }

/* ------------------------------------------------------------------ */
/* Adjoint (transpose) of the step, for gradients of a misfit.  The step of Sec. 3.4 is linear
 * in (E, H); its transpose is built from the transposes of its factors:
 *   the filter and P1 are symmetric on the unknowns (Dirichlet zeros, even Neumann ghosts);
 *   the Pade derivative fp = A^{-1} D1 f / h has the transpose D1^T A^{-T} g / h, with A^{-T}
 *   applied by a banded solve of A^T z = g (A is not symmetric under the one-sided closure). */

/* Solve (24 A)^T y = rhs (banded elimination on the transposed band, no pivoting: A^T is
 * column diagonally dominant). */
static void pade_solve24_T(int M, int closure, int kind, double* rhs, double* y) {
  double* band = (double*)calloc((size_t)M * (2 * PB + 1), sizeof(double));
  for (int i = 0; i < M; ++i) {
    int col[4];
    double val[4];
    int n = pade_row(M, closure, kind, i, col, val);
    /* entry (i, col) of 24A is entry (col, i) of the transpose */
    for (int k = 0; k < n; ++k) band[(size_t)col[k] * (2 * PB + 1) + (i - col[k] + PB)] += val[k];
  }
  for (int k = 0; k < M; ++k) {
    double piv = band[(size_t)k * (2 * PB + 1) + PB];
    for (int i = k + 1; i <= k + PB && i < M; ++i) {
      double* ri = band + (size_t)i * (2 * PB + 1);
      double* rk = band + (size_t)k * (2 * PB + 1);
      double a = ri[k - i + PB];
      if (a == 0.0) continue;
      double l = a / piv;
      for (int j = k; j <= k + PB && j < M; ++j) ri[j - i + PB] -= l * rk[j - k + PB];
      rhs[i] -= l * rhs[k];
    }
  }
  for (int i = M - 1; i >= 0; --i) {
    double* ri = band + (size_t)i * (2 * PB + 1);
    double s = rhs[i];
    for (int j = i + 1; j <= i + PB && j < M; ++j) s -= ri[j - i + PB] * y[j];
    y[i] = s / ri[PB];
  }
  free(band);
}

/* Transpose of or_pade_line: g has M values, out receives M+1 values, out = D1^T A^{-T} g / h. */
void or_pade_line_T(int M, int closure, int kind, double h, const double* g, double* out) {
  double* rhs = (double*)malloc(sizeof(double) * M);
  double* z = (double*)malloc(sizeof(double) * M);
  for (int i = 0; i < M; ++i) rhs[i] = 24.0 * g[i];
  pade_solve24_T(M, closure, kind, rhs, z);
  /* (D1^T z)_k = z_{k-1} - z_k with z_{-1} = z_M = 0 */
  for (int k = 0; k <= M; ++k) out[k] = ((k >= 1 ? z[k - 1] : 0.0) - (k < M ? z[k] : 0.0)) / h;
  free(rhs);
  free(z);
}

/* Transpose of pade_field: reads the dst-shaped array at the positions pade_field writes and
 * accumulates into the src-shaped array (which it first zeroes). */
static void pade_field_T(const or_grid2d* g, int fs, int fd, int axis, int kind, const double* dsrc, double* out) {
  int snx, sny, sbx, sby, dnx, dny, dbx, dby;
  field_dims(g, fs, &snx, &sny, &sbx, &sby);
  field_dims(g, fd, &dnx, &dny, &dbx, &dby);
  int N = g->N;
  int M = (kind == HALF_TO_NODE) ? N - 1 : N;
  int nl = (axis == 0) ? sny : snx;
  double* gl = (double*)malloc(sizeof(double) * M);
  double* o = (double*)malloc(sizeof(double) * (M + 1));
  memset(out, 0, sizeof(double) * (size_t)snx * sny);
  for (int l = 0; l < nl; ++l) {
    for (int k = 0; k < M; ++k) {
      int oo = (kind == HALF_TO_NODE) ? k + 1 : k;
      gl[k] = (axis == 0) ? dsrc[(size_t)l * dnx + oo] : dsrc[(size_t)oo * dnx + l];
    }
    or_pade_line_T(M, g->closure, kind, g->h, gl, o);
    for (int k = 0; k <= M; ++k) {
      if (axis == 0) out[(size_t)l * snx + k] += o[k];
      else out[(size_t)k * snx + l] += o[k];
    }
  }
  free(gl);
  free(o);
}

/* Transposes of the two right-hand-side curls (Sec. 3.4), on arrays whose Dirichlet
 * boundary entries are zero. */
void or2d_curl_h_to_e_T(const or_grid2d* g, const double* lR, double* lGx, double* lGy) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* mu = (double*)malloc(sizeof(double) * ne);
  memcpy(mu, lR, sizeof(double) * ne);
  zero_boundary(g, F_EZ, mu);
  pade_field_T(g, F_HY, F_EZ, 0, HALF_TO_NODE, mu, lGy);
  pade_field_T(g, F_HX, F_EZ, 1, HALF_TO_NODE, mu, lGx);
  double s = g->kappa2 * g->Z;
  for (int p = 0; p < ny_; ++p) lGy[p] *= s;
  for (int p = 0; p < nx_; ++p) lGx[p] *= -s;
  free(mu);
}

void or2d_curl_e_to_h_T(const or_grid2d* g, const double* lRx, const double* lRy, double* lGE) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* mx = (double*)malloc(sizeof(double) * nx_);
  double* my = (double*)malloc(sizeof(double) * ny_);
  double* t = (double*)malloc(sizeof(double) * ne);
  memcpy(mx, lRx, sizeof(double) * nx_);
  memcpy(my, lRy, sizeof(double) * ny_);
  zero_boundary(g, F_HX, mx);
  zero_boundary(g, F_HY, my);
  double s = g->kappa2 / g->Z;
  pade_field_T(g, F_EZ, F_HX, 1, NODE_TO_HALF, mx, lGE);
  pade_field_T(g, F_EZ, F_HY, 0, NODE_TO_HALF, my, t);
  for (int p = 0; p < ne; ++p) lGE[p] = s * (t[p] - lGE[p]);
  free(mx);
  free(my);
  free(t);
}

/* Transpose of one full step: (lE, lHx, lHy) at level n+1 are replaced by the adjoint state at
 * level n.  Reverse order of Sec. 3.4: adjoint of Step 2, then of Step 1. */
void or2d_step_T(or_grid2d* g, double* lE, double* lHx, double* lHy) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* ux = (double*)malloc(sizeof(double) * nx_);
  double* uy = (double*)malloc(sizeof(double) * ny_);
  double* v = (double*)malloc(sizeof(double) * ne);
  double* w = (double*)malloc(sizeof(double) * ne);
  double* vx = (double*)malloc(sizeof(double) * nx_);
  double* vy = (double*)malloc(sizeof(double) * ny_);
  double* wx = (double*)malloc(sizeof(double) * nx_);
  double* wy = (double*)malloc(sizeof(double) * ny_);
  zero_boundary(g, F_EZ, lE);
  zero_boundary(g, F_HX, lHx);
  zero_boundary(g, F_HY, lHy);
  /* Step 2: H += h_tau P1_H^{-1} curl_EH(F_E E)  =>  lE += h_tau F_E curl_EH^T(P1_H^{-1} lH) */
  or2d_p1_solve_cg(g, F_HX, lHx, ux);
  or2d_p1_solve_cg(g, F_HY, lHy, uy);
  or2d_curl_e_to_h_T(g, ux, uy, v);
  zero_boundary(g, F_EZ, v);
  or2d_filter(g, F_EZ, v, w);
  for (int p = 0; p < ne; ++p) lE[p] += g->ht * w[p];
  /* Step 1: E += h_tau P1_E^{-1} curl_HE(F_H H)  =>  lH += h_tau F_H curl_HE^T(P1_E^{-1} lE) */
  or2d_p1_solve_cg(g, F_EZ, lE, v);
  or2d_curl_h_to_e_T(g, v, vx, vy);
  zero_boundary(g, F_HX, vx);
  zero_boundary(g, F_HY, vy);
  or2d_filter(g, F_HX, vx, wx);
  or2d_filter(g, F_HY, vy, wy);
  for (int p = 0; p < nx_; ++p) lHx[p] += g->ht * wx[p];
  for (int p = 0; p < ny_; ++p) lHy[p] += g->ht * wy[p];
  free(ux);
  free(uy);
  free(v);
  free(w);
  free(vx);
  free(vy);
  free(wx);
  free(wy);
}

/* Taylor initialisation of H^{1/2} from E^0 with H^0 = 0 (Sec. 5.1, Eq. "talorh"): with J = 0,
 * d_t H = -Z^{-1} curl E = Z^{-1} (-d_y E, d_x E), d_tt H = 0 at t = 0 (it is the curl of d_t E,
 * which vanishes with H), d_ttt H = Delta d_t H and d_tttt H = 0, so
 *   H^{1/2} = Z^{-1} (t1 + (t1^3/6) Delta_h) c,  c = (-delta_y E^0, delta_x E^0),  t1 = h_tau / 2,
 * with delta the node -> half-node Pade derivative of App. A.1. */
void or2d_taylor_h(const or_grid2d* g, const double* ez, double* hx, double* hy) {
  int nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* cx = (double*)malloc(sizeof(double) * nx_);
  double* cy = (double*)malloc(sizeof(double) * ny_);
  double* lx = (double*)malloc(sizeof(double) * nx_);
  double* ly = (double*)malloc(sizeof(double) * ny_);
  pade_field(g, F_EZ, F_HX, 1, NODE_TO_HALF, ez, cx); /* delta_y E */
  pade_field(g, F_EZ, F_HY, 0, NODE_TO_HALF, ez, cy); /* delta_x E */
  for (int p = 0; p < nx_; ++p) cx[p] = -cx[p];
  zero_boundary(g, F_HX, cx);
  zero_boundary(g, F_HY, cy);
  or2d_laplacian(g, F_HX, cx, lx);
  or2d_laplacian(g, F_HY, cy, ly);
  double t1 = 0.5 * g->ht, c3 = t1 * t1 * t1 / 6.0;
  for (int p = 0; p < nx_; ++p) hx[p] = (t1 * cx[p] + c3 * lx[p]) / g->Z;
  for (int p = 0; p < ny_; ++p) hy[p] = (t1 * cy[p] + c3 * ly[p]) / g->Z;
  zero_boundary(g, F_HX, hx);
  zero_boundary(g, F_HY, hy);
  free(cx);
  free(cy);
  free(lx);
  free(ly);
}

/* Transpose of or2d_taylor_h: lez (output) = T^T (lhx, lhy). */
void or2d_taylor_h_T(const or_grid2d* g, const double* lhx, const double* lhy, double* lez) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* ax = (double*)malloc(sizeof(double) * nx_);
  double* ay = (double*)malloc(sizeof(double) * ny_);
  double* lx = (double*)malloc(sizeof(double) * nx_);
  double* ly = (double*)malloc(sizeof(double) * ny_);
  double* t = (double*)malloc(sizeof(double) * ne);
  memcpy(ax, lhx, sizeof(double) * nx_);
  memcpy(ay, lhy, sizeof(double) * ny_);
  zero_boundary(g, F_HX, ax);
  zero_boundary(g, F_HY, ay);
  or2d_laplacian(g, F_HX, ax, lx);
  or2d_laplacian(g, F_HY, ay, ly);
  double t1 = 0.5 * g->ht, c3 = t1 * t1 * t1 / 6.0;
  for (int p = 0; p < nx_; ++p) ax[p] = (t1 * ax[p] + c3 * lx[p]) / g->Z;
  for (int p = 0; p < ny_; ++p) ay[p] = (t1 * ay[p] + c3 * ly[p]) / g->Z;
  zero_boundary(g, F_HX, ax);
  zero_boundary(g, F_HY, ay);
  /* curl_h^T: cx = -delta_y E -> -pade_T_y(ax); cy = delta_x E -> pade_T_x(ay) */
  pade_field_T(g, F_EZ, F_HX, 1, NODE_TO_HALF, ax, lez);
  pade_field_T(g, F_EZ, F_HY, 0, NODE_TO_HALF, ay, t);
  for (int p = 0; p < ne; ++p) lez[p] = t[p] - lez[p];
  zero_boundary(g, F_EZ, lez);
  free(ax);
  free(ay);
  free(lx);
  free(ly);
  free(t);
}

/* Final-time misfit L = (1/2) h^2 sum_interior (E_z^K - target)^2 after K steps from
 * (E^0, H^{1/2} = Taylor(E^0)), and its gradient with respect to the interior of E^0:
 * the reverse pass applies the transposed step K times, then the transposed initialisation. */
double or2d_misfit_grad(or_grid2d* g, const double* ez0, const double* target, int K, double* grad) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* ez = (double*)malloc(sizeof(double) * ne);
  double* hx = (double*)malloc(sizeof(double) * nx_);
  double* hy = (double*)malloc(sizeof(double) * ny_);
  memcpy(ez, ez0, sizeof(double) * ne);
  zero_boundary(g, F_EZ, ez);
  or2d_taylor_h(g, ez, hx, hy);
  for (int n = 0; n < K; ++n) or2d_step(g, ez, hx, hy);
  /* d = E^K - target on the interior (boundary entries of target do not enter); lE = h^2 d */
  double h2 = g->h * g->h, L = 0.0;
  for (int p = 0; p < ne; ++p) ez[p] -= target[p];
  zero_boundary(g, F_EZ, ez);
  for (int p = 0; p < ne; ++p) {
    L += ez[p] * ez[p];
    ez[p] *= h2;
  }
  L *= 0.5 * h2;
  memset(hx, 0, sizeof(double) * nx_);
  memset(hy, 0, sizeof(double) * ny_);
  if (grad) {
    for (int n = 0; n < K; ++n) or2d_step_T(g, ez, hx, hy);
    or2d_taylor_h_T(g, hx, hy, grad);
    for (int p = 0; p < ne; ++p) grad[p] += ez[p];
    zero_boundary(g, F_EZ, grad);
  }
  free(ez);
  free(hx);
  free(hy);
  return L;
}

/* ------------------------------------------------------------------ */
/* Non-compact fourth-order comparator NC (Sec. 5.2): the leapfrog updating rules of the Yee
 * scheme with the stencil K4 of Eq. "eq:K4" at a = 0, i.e. the first derivative on a staggered
 * line
 *   D u_i = (9/8 (u_{i+1/2} - u_{i-1/2}) - 1/24 (u_{i+3/2} - u_{i-3/2})) / h,
 * and, where that stencil would leave the line, the standard fourth-order one-sided staggered
 * difference: at the first output, from the first four inputs at offsets -1/2, 1/2, 3/2, 5/2,
 *   D u = (-23 u_0 + 21 u_1 + 3 u_2 - u_3) / (24 h),
 * and its mirror image at the last output.  The weights are the unique ones exact for cubics
 * (Taylor expansion), which a test checks. */

/* Derivative of one staggered line of nin values: out[k] (k = 0 .. nin-2) sits between inputs k
 * and k+1 (N half-node values give the N-1 interior nodes; N+1 node values give the N half-nodes). */
void or_nc_line(int nin, double h, const double* f, double* out) {
  int nout = nin - 1; /* both kinds: one output between each pair of neighbouring inputs */
  for (int k = 0; k < nout; ++k) {
    /* inputs straddling output k: f[k] (left, offset -1/2) and f[k+1] (right, +1/2) */
    double v;
    if (k >= 1 && k + 2 < nin) {
      v = (9.0 / 8.0) * (f[k + 1] - f[k]) - (1.0 / 24.0) * (f[k + 2] - f[k - 1]);
    } else if (k == 0) {
      v = (-23.0 * f[0] + 21.0 * f[1] + 3.0 * f[2] - f[3]) / 24.0;
    } else {
      int m = nin - 1; /* last input, offset +1/2 of the last output */
      v = (23.0 * f[m] - 21.0 * f[m - 1] - 3.0 * f[m - 2] + f[m - 3]) / 24.0;
    }
    out[k] = v / h;
  }
}

/* One NC step in place (leapfrog as or2d_yee_step, derivatives by or_nc_line):
 *   E_z += h_tau Z (D_x H_y - D_y H_x);  H_x -= (h_tau/Z) D_y E_z;  H_y += (h_tau/Z) D_x E_z. */
void or2d_nc_step(const or_grid2d* g, double* ez, double* hx, double* hy) {
  int N = g->N;
  double* f = (double*)malloc(sizeof(double) * (N + 1));
  double* d = (double*)malloc(sizeof(double) * (N + 1));
  double ce = g->ht * g->Z, ch = g->ht / g->Z;
  /* E_z: rows j = 1..N-1, D_x H_y (H_y row j has N half-node values) */
  for (int j = 1; j < N; ++j) {
    for (int i = 0; i < N; ++i) f[i] = hy[(size_t)j * N + i];
    or_nc_line(N, g->h, f, d);
    for (int i = 1; i < N; ++i) ez[(size_t)j * (N + 1) + i] += ce * d[i - 1];
  }
  /* columns i = 1..N-1, D_y H_x (H_x column i has N half-node values) */
  for (int i = 1; i < N; ++i) {
    for (int j = 0; j < N; ++j) f[j] = hx[(size_t)j * (N + 1) + i];
    or_nc_line(N, g->h, f, d);
    for (int j = 1; j < N; ++j) ez[(size_t)j * (N + 1) + i] -= ce * d[j - 1];
  }
  /* H_x: columns i = 1..N-1, D_y E_z (N+1 node values) -> N half-nodes */
  for (int i = 1; i < N; ++i) {
    for (int j = 0; j <= N; ++j) f[j] = ez[(size_t)j * (N + 1) + i];
    or_nc_line(N + 1, g->h, f, d);
    for (int j = 0; j < N; ++j) hx[(size_t)j * (N + 1) + i] -= ch * d[j];
  }
  /* H_y: rows j = 1..N-1, D_x E_z */
  for (int j = 1; j < N; ++j) {
    for (int i = 0; i <= N; ++i) f[i] = ez[(size_t)j * (N + 1) + i];
    or_nc_line(N + 1, g->h, f, d);
    for (int i = 0; i < N; ++i) hy[(size_t)j * N + i] += ch * d[i];
  }
  free(f);
  free(d);
}

/* ------------------------------------------------------------------ */
/* Tracked-Delta-E variant: the literal Step 1 / Step 2 of Sec. 3.4.  Besides E and H it carries
 * DE, a fourth-order approximation of Delta E_z on the E grid.  After Step 1 it is advanced
 * with the modified Helmholtz equation of Eq. "eq:mhe" (with J = 0),
 *   DE^{n+1} = DE^n + kappa^2 (E^{n+1} - E^n) - Z (24/h_tau) curl_h H^{n+1/2},
 * curl_h H = delta_x H_y - delta_y H_x the unfiltered Pade curl (App. A.1), and Step 2 filters E
 * with it in the form of Eq. "eq:helm2": G_E = (1 + kappa^2 h^2/12) E + (h^2/12) DE.  DE is 0 on
 * the PEC nodes (Delta E_z = d_tt E_z = 0 there, Table "tab:bc_terms"). */
void or2d_step_tracked(or_grid2d* g, double* ez, double* hx, double* hy, double* de) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* Gx = (double*)malloc(sizeof(double) * nx_);
  double* Gy = (double*)malloc(sizeof(double) * ny_);
  double* R = (double*)malloc(sizeof(double) * ne);
  double* C = (double*)malloc(sizeof(double) * ne);
  double* Es = (double*)malloc(sizeof(double) * ne);
  double* GE = (double*)malloc(sizeof(double) * ne);
  double* Rx = (double*)malloc(sizeof(double) * nx_);
  double* Ry = (double*)malloc(sizeof(double) * ny_);
  double* Hs = (double*)malloc(sizeof(double) * (nx_ > ny_ ? nx_ : ny_));
  /* Step 1, as in or2d_step */
  or2d_filter(g, F_HX, hx, Gx);
  or2d_filter(g, F_HY, hy, Gy);
  or2d_curl_h_to_e(g, Gx, Gy, R);
  or2d_p1_solve_cg(g, F_EZ, R, Es);
  for (int p = 0; p < ne; ++p) ez[p] += g->ht * Es[p];
  /* DE += kappa^2 h_tau E* - Z (24/h_tau) curl_h H; or2d_curl_h_to_e gives kappa^2 Z curl_h H */
  or2d_curl_h_to_e(g, hx, hy, C);
  for (int p = 0; p < ne; ++p) de[p] += g->kappa2 * g->ht * Es[p] - (24.0 / g->ht) * C[p] / g->kappa2;
  zero_boundary(g, F_EZ, de);
  /* Step 2 with G_E = beta E + (h^2/12) DE */
  double h2_12 = g->h * g->h / 12.0;
  for (int p = 0; p < ne; ++p) GE[p] = g->beta * ez[p] + h2_12 * de[p];
  zero_boundary(g, F_EZ, GE);
  or2d_curl_e_to_h(g, GE, Rx, Ry);
  or2d_p1_solve_cg(g, F_HX, Rx, Hs);
  for (int p = 0; p < nx_; ++p) hx[p] += g->ht * Hs[p];
  or2d_p1_solve_cg(g, F_HY, Ry, Hs);
  for (int p = 0; p < ny_; ++p) hy[p] += g->ht * Hs[p];
  free(Gx);
  free(Gy);
  free(R);
  free(C);
  free(Es);
  free(GE);
  free(Rx);
  free(Ry);
  free(Hs);
}

/* ------------------------------------------------------------------ */
/* Current sources J = J_z z (2D TM_z, so div J = 0), a superposition of driven sine modes
 *   J_z = a sin(m pi x) sin(n pi y) sin(w t),  src rows (m, n, a, w),
 * which vanish on the walls with all the derivatives the Neumann data of Sec. 3.3 involve, so the
 * even ghosts of Cor. "cor:ghost_cor" stay exact.  The modified Helmholtz equations of Eq. "eq:mh"
 * gain, from the Taylor expansion of Sec. 3.1 written out with Faraday's and Ampere's laws,
 *   E:  P(J) = Z (-kappa^2 J + grad div J - d_tt J) = -Z (kappa^2 - w^2) J   at t^{n+1/2},
 *   H:  + curl d_t J = (d_y d_t J_z, -d_x d_t J_z)                            at t^{n+1},
 * each passed through the right-hand-side filter of Eq. "eq:ell" with the exact Laplacian of
 * the source (the form of Eq. "eq:helm2"): factor beta - (h^2/12) pi^2 (m^2 + n^2). */
static void add_sources_e(const or_grid2d* g, const double* src, int nsrc, double t, double* R) {
  int N = g->N;
  double pi = M_PI, h = g->h;
  for (int q = 0; q < nsrc; ++q) {
    double m = src[4 * q], n = src[4 * q + 1], a = src[4 * q + 2], w = src[4 * q + 3];
    double filt = g->beta - (h * h / 12.0) * pi * pi * (m * m + n * n);
    double amp = -g->Z * (g->kappa2 - w * w) * filt * a * sin(w * t);
    for (int j = 1; j < N; ++j)
      for (int i = 1; i < N; ++i) R[(size_t)j * (N + 1) + i] += amp * sin(pi * m * i * h) * sin(pi * n * j * h);
  }
}

static void add_sources_h(const or_grid2d* g, const double* src, int nsrc, double t, double* Rx, double* Ry) {
  int N = g->N;
  double pi = M_PI, h = g->h;
  for (int q = 0; q < nsrc; ++q) {
    double m = src[4 * q], n = src[4 * q + 1], a = src[4 * q + 2], w = src[4 * q + 3];
    double filt = g->beta - (h * h / 12.0) * pi * pi * (m * m + n * n);
    double c = filt * a * w * cos(w * t);
    for (int j = 0; j < N; ++j) /* H_x at (x_i, y_{j+1/2}): d_y d_t J_z */
      for (int i = 1; i < N; ++i)
        Rx[(size_t)j * (N + 1) + i] += c * pi * n * sin(pi * m * i * h) * cos(pi * n * (j + 0.5) * h);
    for (int j = 1; j < N; ++j) /* H_y at (x_{i+1/2}, y_j): -d_x d_t J_z */
      for (int i = 0; i < N; ++i)
        Ry[(size_t)j * N + i] -= c * pi * m * cos(pi * m * (i + 0.5) * h) * sin(pi * n * j * h);
  }
}

/* One full step with sources: or2d_step with P(J)^{n+1/2} added to the E right-hand side and
 * curl d_t J^{n+1} to the H right-hand sides; n is the index of the step (E^n -> E^{n+1}). */
void or2d_step_src(or_grid2d* g, double* ez, double* hx, double* hy, const double* src, int nsrc, long n) {
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* Gx = (double*)malloc(sizeof(double) * nx_);
  double* Gy = (double*)malloc(sizeof(double) * ny_);
  double* R = (double*)malloc(sizeof(double) * ne);
  double* Es = (double*)malloc(sizeof(double) * ne);
  double* GE = (double*)malloc(sizeof(double) * ne);
  double* Rx = (double*)malloc(sizeof(double) * nx_);
  double* Ry = (double*)malloc(sizeof(double) * ny_);
  double* Hs = (double*)malloc(sizeof(double) * (nx_ > ny_ ? nx_ : ny_));
  or2d_filter(g, F_HX, hx, Gx);
  or2d_filter(g, F_HY, hy, Gy);
  or2d_curl_h_to_e(g, Gx, Gy, R);
  add_sources_e(g, src, nsrc, (n + 0.5) * g->ht, R);
  or2d_p1_solve_cg(g, F_EZ, R, Es);
  for (int p = 0; p < ne; ++p) ez[p] += g->ht * Es[p];
  or2d_filter(g, F_EZ, ez, GE);
  or2d_curl_e_to_h(g, GE, Rx, Ry);
  add_sources_h(g, src, nsrc, (n + 1.0) * g->ht, Rx, Ry);
  or2d_p1_solve_cg(g, F_HX, Rx, Hs);
  for (int p = 0; p < nx_; ++p) hx[p] += g->ht * Hs[p];
  or2d_p1_solve_cg(g, F_HY, Ry, Hs);
  for (int p = 0; p < ny_; ++p) hy[p] += g->ht * Hs[p];
  free(Gx);
  free(Gy);
  free(R);
  free(Es);
  free(GE);
  free(Rx);
  free(Ry);
  free(Hs);
}

/* Exact driven solution for the sources above (particular solution, w^2 != pi^2 (m^2 + n^2)):
 *   E_z = A cos(w t) sin(m pi x) sin(n pi y),  A = Z a w / (w^2 - pi^2 (m^2 + n^2)),
 *   H_x = -(A n pi / (Z w)) sin(w t) sin(m pi x) cos(n pi y),  H_y = (A m pi / (Z w)) sin(w t) cos(m pi x) sin(n pi y),
 * from Faraday's law and d_tt E_z = Delta E_z - Z d_t J_z. */
void or2d_exact_driven(const or_grid2d* g, const double* src, int nsrc, double tE, double tH, double* ez, double* hx,
                       double* hy) {
  int N = g->N;
  double h = g->h, pi = M_PI;
  memset(ez, 0, sizeof(double) * (N + 1) * (N + 1));
  memset(hx, 0, sizeof(double) * N * (N + 1));
  memset(hy, 0, sizeof(double) * N * (N + 1));
  for (int q = 0; q < nsrc; ++q) {
    double m = src[4 * q], n = src[4 * q + 1], a = src[4 * q + 2], w = src[4 * q + 3];
    double A = g->Z * a * w / (w * w - pi * pi * (m * m + n * n));
    double ce = A * cos(w * tE), sh = A * sin(w * tH) / (g->Z * w);
    for (int j = 1; j < N; ++j)
      for (int i = 1; i < N; ++i) ez[(size_t)j * (N + 1) + i] += ce * sin(pi * m * i * h) * sin(pi * n * j * h);
    for (int j = 0; j < N; ++j)
      for (int i = 1; i < N; ++i)
        hx[(size_t)j * (N + 1) + i] += -sh * pi * n * sin(pi * m * i * h) * cos(pi * n * (j + 0.5) * h);
    for (int j = 1; j < N; ++j)
      for (int i = 0; i < N; ++i)
        hy[(size_t)j * N + i] += sh * pi * m * cos(pi * m * (i + 0.5) * h) * sin(pi * n * j * h);
  }
}

/* ------------------------------------------------------------------ */
/* Sources that do not vanish on the walls: inhomogeneous Neumann data (Sec. 3.3, Method 2).
 * Source rows (m, n, a, w, px, py):
 *   J_z = a X(m pi x) Y(n pi y) sin(w t),   X = sin if px = 0, cos if px = 1 (Y likewise by py),
 * m, n >= 0 (a sine index >= 1).  The right-hand-side terms P(J) and curl d_t J are those of
 * add_sources_e / add_sources_h with these profiles; every profile satisfies X'' = -(m pi)^2 X, so
 * the filter factor is the same.  With J_z nonzero on a wall three boundary data change, each
 * derived from Faraday's and Ampere's laws (d_t E = Z (curl H - J), d_t H = -curl E / Z) and the
 * PEC conditions E_z = 0, H.n = 0 on the wall, the way Sec. 3.3 derives the Neumann data:
 *   - on x = 0, 1 (H_y Neumann in x):  d_x H_y = J_z,   d_xxx H_y = d_tt J_z + d_xx J_z - d_yy J_z;
 *     on y = 0, 1 (H_x Neumann in y):  d_y H_x = -J_z,  d_yyy H_x = -(d_tt J_z + d_yy J_z - d_xx J_z).
 *     (Ampere's law on the wall gives the first derivative; differentiating it twice across the wall,
 *     with div H = 0 and Delta E_z = d_tt E_z + Z d_t J_z = Z d_t J_z on the wall, the third.)
 *     The ghost half a cell outside follows from the Taylor relation of Eq. "eq:gst2",
 *     phi(h/2) - phi(-h/2) = h phi' + (h^3/24) phi''' + O(h^5) at the wall:
 *       u(-1) = u(0) - g_lo,  u(n) = u(n-1) + g_hi,  g = h phi' + (h^3/24) phi''' on that wall.
 *     The H filter of Step 1 takes the data of H at t^{n+1/2}; the H solves of Step 2 take the data
 *     of their unknown H* = (H^{n+3/2} - H^{n+1/2}) / h_tau, i.e. the difference of the data at
 *     t^{n+3/2} and t^{n+1/2} over h_tau.
 *   - G_E on the boundary nodes is (h^2/12) Delta E_z = (h^2/12) Z d_t J_z at t^{n+1} (E_z = 0
 *     there; with J = 0 this is the zero of Sec. 3.4).
 * Ghost values at the Dirichlet end points of a wall (the corners) are not used: the second
 * differences there are zero, as for every Dirichlet point.  The one-sided Pade rows of the PAPER
 * closure need no ghost; the REFLECT rows assume even data at the walls and are not meant for
 * these sources. */
static double prof(int p, double k, double x) { return p ? cos(M_PI * k * x) : sin(M_PI * k * x); }
static double dprof(int p, double k, double x) { return p ? -M_PI * k * sin(M_PI * k * x) : M_PI * k * cos(M_PI * k * x); }
/* exact profile value on a wall: side 0 is x = 0, side 1 is x = 1 */
static double prof_wall(int p, int k, int side) {
  if (!p) return 0.0;
  return (side && (k & 1)) ? -1.0 : 1.0;
}
/* profile at node i of n cells (exact at the two walls) */
static double prof_node(int p, int k, int i, int n) {
  if (i == 0) return prof_wall(p, k, 0);
  if (i == n) return prof_wall(p, k, 1);
  return prof(p, k, (double)i / n);
}

/* Second differences along one axis with ghost data on the Neumann ends of that axis
 * (d2_axis with u(-1) = u(0) - glo[line], u(n) = u(n-1) + ghi[line]; line = the other index). */
static void d2_axis_g(const or_grid2d* g, int f, int axis, const double* u, double* out, const double* glo,
                      const double* ghi) {
  int nx, ny, bx, by;
  field_dims(g, f, &nx, &ny, &bx, &by);
  double ih2 = 1.0 / (g->h * g->h);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t p = (size_t)j * nx + i;
      if (!axis_interior(bx, i, nx) || !axis_interior(by, j, ny)) { out[p] = 0.0; continue; }
      double um, up;
      if (axis == 0) {
        um = (i - 1 >= 0) ? u[p - 1] : u[p] - glo[j];
        up = (i + 1 < nx) ? u[p + 1] : u[p] + ghi[j];
      } else {
        um = (j - 1 >= 0) ? u[p - nx] : u[p] - glo[i];
        up = (j + 1 < ny) ? u[p + nx] : u[p] + ghi[i];
      }
      out[p] = (um - 2.0 * u[p] + up) * ih2;
    }
}

/* Ghost data of H_x (indexed by column i, walls y = 0, 1) and H_y (indexed by row j, walls
 * x = 0, 1).  diff = 0: the data of H at t1; diff = 1: of (H(t1) - H(t0)) / h_tau. */
void or2d_wall_ghosts(const or_grid2d* g, const double* src, int nsrc, double t0, double t1, int diff, double* gx_lo,
                      double* gx_hi, double* gy_lo, double* gy_hi) {
  int N = g->N;
  double h = g->h, pi2 = M_PI * M_PI;
  for (int k = 0; k <= N; ++k) gx_lo[k] = gx_hi[k] = gy_lo[k] = gy_hi[k] = 0.0;
  for (int q = 0; q < nsrc; ++q) {
    const double* s = src + 6 * q;
    int m = (int)s[0], n = (int)s[1], px = (int)s[4], py = (int)s[5];
    double a = s[2], w = s[3];
    double T = diff ? (sin(w * t1) - sin(w * t0)) / g->ht : sin(w * t1);
    /* x walls, H_y: g = h J + (h^3/24)(d_tt + d_xx - d_yy) J = J (h + (h^3/24)(pi^2 n^2 - pi^2 m^2 - w^2)) */
    double cx = h + h * h * h / 24.0 * (pi2 * n * n - pi2 * m * m - w * w);
    /* y walls, H_x: g = -h J - (h^3/24)(d_tt + d_yy - d_xx) J = -J (h + (h^3/24)(pi^2 m^2 - pi^2 n^2 - w^2)) */
    double cy = -(h + h * h * h / 24.0 * (pi2 * m * m - pi2 * n * n - w * w));
    for (int j = 1; j < N; ++j) {
      double Yj = prof_node(py, n, j, N);
      gy_lo[j] += cx * a * prof_wall(px, m, 0) * Yj * T;
      gy_hi[j] += cx * a * prof_wall(px, m, 1) * Yj * T;
    }
    for (int i = 1; i < N; ++i) {
      double Xi = prof_node(px, m, i, N);
      gx_lo[i] += cy * a * Xi * prof_wall(py, n, 0) * T;
      gx_hi[i] += cy * a * Xi * prof_wall(py, n, 1) * T;
    }
  }
}

/* Right-hand-side filter of Eq. "eq:ell" for H_x or H_y with the ghost data on its Neumann axis. */
static void filter_ghost(const or_grid2d* g, int f, const double* u, double* G, const double* glo, const double* ghi) {
  int nx, ny, bx, by;
  field_dims(g, f, &nx, &ny, &bx, &by);
  int n = nx * ny;
  double* t = (double*)malloc(sizeof(double) * n);
  int neu_axis = (f == F_HX) ? 1 : 0;
  d2_axis_g(g, f, neu_axis, u, G, glo, ghi);
  d2_axis(g, f, 1 - neu_axis, u, t);
  double h2_12 = g->h * g->h / 12.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t p = (size_t)j * nx + i;
      if (!axis_interior(bx, i, nx) || !axis_interior(by, j, ny)) G[p] = 0.0;
      else G[p] = g->beta * u[p] + h2_12 * (G[p] + t[p]);
    }
  free(t);
}

/* P1 of H_x or H_y applied to the zero field with the ghost data: the affine part of P1 with
 * inhomogeneous ghosts, P1_g x = P1 x + P1_g 0.  The 9-point stencil with the ghost nodes,
 * written as the Kronecker composition with the Neumann-axis difference first. */
void or2d_p1_ghost_shift(const or_grid2d* g, int f, const double* glo, const double* ghi, double* c) {
  int nx, ny, bx, by;
  field_dims(g, f, &nx, &ny, &bx, &by);
  int n = nx * ny;
  double* z = (double*)calloc(n, sizeof(double));
  double* dn = (double*)malloc(sizeof(double) * n);
  double* dnd = (double*)malloc(sizeof(double) * n);
  int neu_axis = (f == F_HX) ? 1 : 0;
  d2_axis_g(g, f, neu_axis, z, dn, glo, ghi);
  d2_axis(g, f, 1 - neu_axis, dn, dnd);
  double h2_6 = g->h * g->h / 6.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t p = (size_t)j * nx + i;
      if (!axis_interior(bx, i, nx) || !axis_interior(by, j, ny)) c[p] = 0.0;
      else c[p] = -(dn[p] + h2_6 * dnd[p]);
    }
  free(z);
  free(dn);
  free(dnd);
}

/* G_E on the boundary nodes: (h^2/12) Z d_t J_z at time t (interior entries untouched). */
void or2d_ge_wall(const or_grid2d* g, const double* src, int nsrc, double t, double* GE) {
  int N = g->N;
  double c = g->h * g->h / 12.0 * g->Z;
  for (int j = 0; j <= N; ++j)
    for (int i = 0; i <= N; ++i) {
      if (i > 0 && i < N && j > 0 && j < N) continue;
      double v = 0.0;
      for (int q = 0; q < nsrc; ++q) {
        const double* s = src + 6 * q;
        int m = (int)s[0], n = (int)s[1], px = (int)s[4], py = (int)s[5];
        v += s[2] * s[3] * cos(s[3] * t) * prof_node(px, m, i, N) * prof_node(py, n, j, N);
      }
      GE[(size_t)j * (N + 1) + i] = c * v;
    }
}

/* P(J) (E side, t) and curl d_t J (H side, t) through the filter, for the profiled sources. */
static void add_sources_e_xy(const or_grid2d* g, const double* src, int nsrc, double t, double* R) {
  int N = g->N;
  double h = g->h;
  for (int q = 0; q < nsrc; ++q) {
    const double* s = src + 6 * q;
    int m = (int)s[0], n = (int)s[1], px = (int)s[4], py = (int)s[5];
    double a = s[2], w = s[3];
    double filt = g->beta - (h * h / 12.0) * M_PI * M_PI * ((double)m * m + (double)n * n);
    double amp = -g->Z * (g->kappa2 - w * w) * filt * a * sin(w * t);
    for (int j = 1; j < N; ++j)
      for (int i = 1; i < N; ++i) R[(size_t)j * (N + 1) + i] += amp * prof(px, m, i * h) * prof(py, n, j * h);
  }
}

static void add_sources_h_xy(const or_grid2d* g, const double* src, int nsrc, double t, double* Rx, double* Ry) {
  int N = g->N;
  double h = g->h;
  for (int q = 0; q < nsrc; ++q) {
    const double* s = src + 6 * q;
    int m = (int)s[0], n = (int)s[1], px = (int)s[4], py = (int)s[5];
    double a = s[2], w = s[3];
    double filt = g->beta - (h * h / 12.0) * M_PI * M_PI * ((double)m * m + (double)n * n);
    double c = filt * a * w * cos(w * t);
    for (int j = 0; j < N; ++j) /* H_x at (x_i, y_{j+1/2}): d_y d_t J_z */
      for (int i = 1; i < N; ++i) Rx[(size_t)j * (N + 1) + i] += c * prof(px, m, i * h) * dprof(py, n, (j + 0.5) * h);
    for (int j = 1; j < N; ++j) /* H_y at (x_{i+1/2}, y_j): -d_x d_t J_z */
      for (int i = 0; i < N; ++i) Ry[(size_t)j * N + i] -= c * dprof(px, m, (i + 0.5) * h) * prof(py, n, j * h);
  }
}

/* One full step with profiled sources (PAPER closure): or2d_step_src with the ghost data above in
 * the H filter of Step 1 and the H solves of Step 2, and G_E on the walls from d_t J. */
void or2d_step_src_xy(or_grid2d* g, double* ez, double* hx, double* hy, const double* src, int nsrc, long n) {
  int N = g->N;
  int ne = or2d_field_size(g, F_EZ), nx_ = or2d_field_size(g, F_HX), ny_ = or2d_field_size(g, F_HY);
  double* Gx = (double*)malloc(sizeof(double) * nx_);
  double* Gy = (double*)malloc(sizeof(double) * ny_);
  double* R = (double*)malloc(sizeof(double) * ne);
  double* Es = (double*)malloc(sizeof(double) * ne);
  double* GE = (double*)malloc(sizeof(double) * ne);
  double* Rx = (double*)malloc(sizeof(double) * nx_);
  double* Ry = (double*)malloc(sizeof(double) * ny_);
  double* Hs = (double*)malloc(sizeof(double) * (nx_ > ny_ ? nx_ : ny_));
  double* c = (double*)malloc(sizeof(double) * (nx_ > ny_ ? nx_ : ny_));
  double* gd = (double*)malloc(sizeof(double) * 4 * (N + 1));
  double *gxl = gd, *gxh = gd + (N + 1), *gyl = gd + 2 * (N + 1), *gyh = gd + 3 * (N + 1);
  double th = (n + 0.5) * g->ht, t1 = (n + 1.0) * g->ht, t32 = (n + 1.5) * g->ht;
  /* Step 1 */
  or2d_wall_ghosts(g, src, nsrc, th, th, 0, gxl, gxh, gyl, gyh);
  filter_ghost(g, F_HX, hx, Gx, gxl, gxh);
  filter_ghost(g, F_HY, hy, Gy, gyl, gyh);
  or2d_curl_h_to_e(g, Gx, Gy, R);
  add_sources_e_xy(g, src, nsrc, th, R);
  or2d_p1_solve_cg(g, F_EZ, R, Es);
  for (int p = 0; p < ne; ++p) ez[p] += g->ht * Es[p];
  /* Step 2 */
  or2d_filter(g, F_EZ, ez, GE);
  or2d_ge_wall(g, src, nsrc, t1, GE);
  or2d_curl_e_to_h(g, GE, Rx, Ry);
  add_sources_h_xy(g, src, nsrc, t1, Rx, Ry);
  or2d_wall_ghosts(g, src, nsrc, th, t32, 1, gxl, gxh, gyl, gyh);
  or2d_p1_ghost_shift(g, F_HX, gxl, gxh, c);
  for (int p = 0; p < nx_; ++p) Rx[p] -= c[p];
  or2d_p1_ghost_shift(g, F_HY, gyl, gyh, c);
  for (int p = 0; p < ny_; ++p) Ry[p] -= c[p];
  or2d_p1_solve_cg(g, F_HX, Rx, Hs);
  for (int p = 0; p < nx_; ++p) hx[p] += g->ht * Hs[p];
  or2d_p1_solve_cg(g, F_HY, Ry, Hs);
  for (int p = 0; p < ny_; ++p) hy[p] += g->ht * Hs[p];
  free(Gx);
  free(Gy);
  free(R);
  free(Es);
  free(GE);
  free(Rx);
  free(Ry);
  free(Hs);
  free(c);
  free(gd);
}
