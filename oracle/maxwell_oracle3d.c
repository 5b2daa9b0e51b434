/*
 * Plain FP64 CPU oracle of the three-dimensional compact scheme (six components)
 * of Versano, Turkel & Tsynkov (arXiv 2306.17263).
 *
 * TEST INFRASTRUCTURE ONLY, like maxwell_oracle.c (which provides the Pade line
 * solver or_pade_line used here).  The CUDA library never calls or includes this.
 *
 * Written from the paper's definitions:
 *   - meshes of the six components: Sec. 2, Eq. "eq:meshes";
 *   - Dirichlet / Neumann type of every component along every axis: Table "tab:bc"
 *     (a component is Dirichlet, with stored zeros at the walls, along the axes on
 *     which it sits on nodes, and Neumann, with even ghosts, along the axes on which
 *     it sits on half-nodes);
 *   - Delta_h = D_xx + D_yy + D_zz and Upsilon_h = D_zz D_xx + D_yy D_zz + D_xx D_yy:
 *     Sec. 3.2, Eq. "eq:ell";
 *   - P1 = -(Delta_h + (h^2/6) Upsilon_h) + kappa^2 (1 + 2/r^2): Def. "def:operatorsP";
 *   - curl_h = [[0, -d_z, d_y], [d_z, 0, -d_x], [-d_y, d_x, 0]] with the Pade
 *     derivatives of App. A.1: Sec. 3.4;
 *   - Step 1 / Step 2 with J = rho = 0: Sec. 3.4 (third rows read as E_z, H_z), and with
 *     divergence-free current sources (or3d_step_src, end of this file);
 *   - conjugate-gradient solves: Sec. 3.2.
 * The exact cavity mode used for checks is not in the paper (it treats 2D only in its
 * experiments): E = A (cos ax sin by sin cz, sin ax cos by sin cz, sin ax sin by cos cz)
 * cos(omega t) with (a, b, c) = pi (m, n, p), A . (a, b, c) = 0, omega = |(a, b, c)|, and
 * H = -(1/(Z omega)) curl(E / cos(omega t)) sin(omega t), derived from Maxwell's equations
 * (Sec. 2, Eq. "eq:maxwellv").
 *
 * Array layout: [z][y][x], x fastest, boundary points stored.  Component c:
 *   0 E_x (N, N+1, N+1)   1 E_y (N+1, N, N+1)   2 E_z (N+1, N+1, N)
 *   3 H_x (N+1, N, N)     4 H_y (N, N+1, N)     5 H_z (N, N, N+1)       (nx, ny, nz)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { BC_DIR3 = 0, BC_NEU3 = 1 };
enum { P_HALF_TO_NODE = 0, P_NODE_TO_HALF = 1 };

void or_pade_line(int M, int closure, int kind, double h, const double* f, double* fp);

typedef struct {
  int N;
  double r, Z, h, ht, kappa2, beta, c1;
  int closure;
  double cg_tol;
  int cg_maxit;
  long cg_iters_total;
  long cg_solves;
} or_grid3d;

int or3d_sizeof(void) { return (int)sizeof(or_grid3d); }

void or3d_setup(or_grid3d* g, int N, double r, double Z, int closure) {
  g->N = N;
  g->r = r;
  g->Z = Z;
  g->h = 1.0 / N;
  g->ht = r * g->h;
  g->kappa2 = 24.0 / (g->ht * g->ht);
  g->beta = 1.0 + g->kappa2 * g->h * g->h / 12.0; /* = 1 + 2/r^2 */
  g->c1 = g->kappa2 * g->beta;
  g->closure = closure;
  g->cg_tol = 1e-14;
  g->cg_maxit = 200;
  g->cg_iters_total = 0;
  g->cg_solves = 0;
}

void or3d_set_cg(or_grid3d* g, double tol, int maxit) {
  g->cg_tol = tol;
  g->cg_maxit = maxit;
}

/* Table "tab:bc": E_s is Neumann along s and Dirichlet along the other axes; H_s is
 * Dirichlet along s and Neumann along the other axes. */
int or3d_bc(int c, int axis) {
  int s = c % 3;
  if (c < 3) return axis == s ? BC_NEU3 : BC_DIR3;
  return axis == s ? BC_DIR3 : BC_NEU3;
}

void or3d_dims(const or_grid3d* g, int c, int* d) {
  for (int a = 0; a < 3; ++a) d[a] = or3d_bc(c, a) == BC_DIR3 ? g->N + 1 : g->N;
}

long or3d_field_size(const or_grid3d* g, int c) {
  int d[3];
  or3d_dims(g, c, d);
  return (long)d[0] * d[1] * d[2];
}

/* Is point (i, j, k) an unknown of component c (not a Dirichlet wall point)? */
static int unknown3(const or_grid3d* g, int c, const int* d, int i, int j, int k) {
  int idx[3] = {i, j, k};
  for (int a = 0; a < 3; ++a)
    if (or3d_bc(c, a) == BC_DIR3 && (idx[a] == 0 || idx[a] == d[a] - 1)) return 0;
  (void)g;
  return 1;
}

static void zero_walls3(const or_grid3d* g, int c, double* u) {
  int d[3];
  or3d_dims(g, c, d);
  for (int k = 0; k < d[2]; ++k)
    for (int j = 0; j < d[1]; ++j)
      for (int i = 0; i < d[0]; ++i)
        if (!unknown3(g, c, d, i, j, k)) u[((size_t)k * d[1] + j) * d[0] + i] = 0.0;
}

/* D_2 along one axis (App. A.1): Dirichlet axes read the stored wall zeros, Neumann axes the
 * even ghosts u(-1) = u(0), u(n) = u(n-1) (Cor. "cor:ghost_cor").  0 at wall points. */
static void d2_axis3(const or_grid3d* g, int c, int axis, const double* u, double* out) {
  int d[3];
  or3d_dims(g, c, d);
  const double ih2 = 1.0 / (g->h * g->h);
  const size_t stride[3] = {1, (size_t)d[0], (size_t)d[0] * d[1]};
  for (int k = 0; k < d[2]; ++k)
    for (int j = 0; j < d[1]; ++j)
      for (int i = 0; i < d[0]; ++i) {
        size_t p = ((size_t)k * d[1] + j) * d[0] + i;
        if (!unknown3(g, c, d, i, j, k)) {
          out[p] = 0.0;
          continue;
        }
        int idx[3] = {i, j, k};
        int q = idx[axis];
        double um = (q - 1 >= 0) ? u[p - stride[axis]] : u[p];
        double up = (q + 1 < d[axis]) ? u[p + stride[axis]] : u[p];
        out[p] = (um - 2.0 * u[p] + up) * ih2;
      }
}

/* Delta_h = D_xx + D_yy + D_zz (Sec. 3.2). */
void or3d_laplacian(const or_grid3d* g, int c, const double* u, double* out) {
  long n = or3d_field_size(g, c);
  double* t = (double*)malloc(sizeof(double) * n);
  d2_axis3(g, c, 0, u, out);
  for (int a = 1; a < 3; ++a) {
    d2_axis3(g, c, a, u, t);
    for (long p = 0; p < n; ++p) out[p] += t[p];
  }
  free(t);
}

/* Right-hand-side filter of Eq. "eq:ell": G = (1 + kappa^2 h^2/12) u + (h^2/12) Delta_h u. */
void or3d_filter(const or_grid3d* g, int c, const double* u, double* G) {
  long n = or3d_field_size(g, c);
  or3d_laplacian(g, c, u, G);
  const double h2_12 = g->h * g->h / 12.0;
  for (long p = 0; p < n; ++p) G[p] = g->beta * u[p] + h2_12 * G[p];
  zero_walls3(g, c, G);
}

/* P1 = -(Delta_h + (h^2/6) Upsilon_h) + c1, Upsilon_h = D_zz D_xx + D_yy D_zz + D_xx D_yy
 * (Def. "def:operatorsP"), as compositions of the one-axis D_2 operators. */
void or3d_p1_apply(const or_grid3d* g, int c, const double* x, double* y) {
  long n = or3d_field_size(g, c);
  double* dd[3];
  double* t = (double*)malloc(sizeof(double) * n);
  for (int a = 0; a < 3; ++a) {
    dd[a] = (double*)malloc(sizeof(double) * n);
    d2_axis3(g, c, a, x, dd[a]);
  }
  const double h2_6 = g->h * g->h / 6.0;
  for (long p = 0; p < n; ++p) y[p] = g->c1 * x[p] - (dd[0][p] + dd[1][p] + dd[2][p]);
  /* Upsilon_h: D_zz D_xx + D_yy D_zz + D_xx D_yy */
  const int pairs[3][2] = {{2, 0}, {1, 2}, {0, 1}};
  for (int q = 0; q < 3; ++q) {
    d2_axis3(g, c, pairs[q][0], dd[pairs[q][1]], t);
    for (long p = 0; p < n; ++p) y[p] -= h2_6 * t[p];
  }
  zero_walls3(g, c, y);
  for (int a = 0; a < 3; ++a) free(dd[a]);
  free(t);
}

static double dot3(long n, const double* a, const double* b) {
  double s = 0.0;
  for (long p = 0; p < n; ++p) s += a[p] * b[p];
  return s;
}

/* Conjugate gradients for P1 x = b from x = 0 to ||r|| <= tol ||b|| (Sec. 3.2). */
int or3d_p1_solve_cg(or_grid3d* g, int c, const double* b, double* x) {
  long n = or3d_field_size(g, c);
  double* r = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  double* Ap = (double*)malloc(sizeof(double) * n);
  for (long i = 0; i < n; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
    p[i] = b[i];
  }
  zero_walls3(g, c, r);
  zero_walls3(g, c, p);
  double bb = dot3(n, r, r), rr = bb;
  int it = 0;
  while (rr > g->cg_tol * g->cg_tol * bb && it < g->cg_maxit && bb > 0.0) {
    or3d_p1_apply(g, c, p, Ap);
    double alpha = rr / dot3(n, p, Ap);
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    double rr_new = dot3(n, r, r);
    for (long i = 0; i < n; ++i) p[i] = r[i] + (rr_new / rr) * p[i];
    rr = rr_new;
    ++it;
  }
  g->cg_iters_total += it;
  g->cg_solves += 1;
  free(r);
  free(p);
  free(Ap);
  return it;
}

/* Pade derivative along `axis` from component cs to component cd (App. A.1): for every line
 * along the axis, HALF_TO_NODE maps the N half-node values to the N-1 interior nodes, and
 * NODE_TO_HALF maps the N+1 node values (wall zeros included) to the N half-nodes.  The
 * other two coordinates are of the same type in cs and cd.  dst is zero elsewhere. */
static void pade_field3(const or_grid3d* g, int cs, int cd, int axis, int kind, const double* src, double* dst) {
  int ds[3], dd[3];
  or3d_dims(g, cs, ds);
  or3d_dims(g, cd, dd);
  const int N = g->N;
  const int M = (kind == P_HALF_TO_NODE) ? N - 1 : N;
  const size_t ss[3] = {1, (size_t)ds[0], (size_t)ds[0] * ds[1]};
  const size_t sd[3] = {1, (size_t)dd[0], (size_t)dd[0] * dd[1]};
  const int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
  double* f = (double*)malloc(sizeof(double) * (M + 1));
  double* fp = (double*)malloc(sizeof(double) * M);
  memset(dst, 0, sizeof(double) * (size_t)dd[0] * dd[1] * dd[2]);
  for (int u = 0; u < ds[a1]; ++u)
    for (int v = 0; v < ds[a2]; ++v) {
      size_t bs = u * ss[a1] + v * ss[a2], bd = u * sd[a1] + v * sd[a2];
      for (int q = 0; q <= M; ++q) f[q] = src[bs + q * ss[axis]];
      or_pade_line(M, g->closure, kind, g->h, f, fp);
      for (int q = 0; q < M; ++q) {
        int o = (kind == P_HALF_TO_NODE) ? q + 1 : q;
        dst[bd + o * sd[axis]] = fp[q];
      }
    }
  free(f);
  free(fp);
}

/* Step 1 right-hand side: R_E = kappa^2 Z curl_h G_H (Sec. 3.4):
 *   R_x = kappa^2 Z (-d_z G_y + d_y G_z), R_y = kappa^2 Z (d_z G_x - d_x G_z),
 *   R_z = kappa^2 Z (-d_y G_x + d_x G_y). */
void or3d_curl_h_to_e(const or_grid3d* g, const double* const* G, double* const* R) {
  const double s = g->kappa2 * g->Z;
  for (int e = 0; e < 3; ++e) {
    long n = or3d_field_size(g, e);
    double* a = (double*)malloc(sizeof(double) * n);
    double* b = (double*)malloc(sizeof(double) * n);
    /* R_e = s (d_{e+1} G_{e+2} - d_{e+2} G_{e+1}) (cyclic indices) */
    int p1 = (e + 1) % 3, p2 = (e + 2) % 3;
    pade_field3(g, 3 + p2, e, p1, P_HALF_TO_NODE, G[p2], a);
    pade_field3(g, 3 + p1, e, p2, P_HALF_TO_NODE, G[p1], b);
    for (long p = 0; p < n; ++p) R[e][p] = s * (a[p] - b[p]);
    zero_walls3(g, e, R[e]);
    free(a);
    free(b);
  }
}

/* Step 2 right-hand side: R_H = -(kappa^2/Z) curl_h G_E (Sec. 3.4). */
void or3d_curl_e_to_h(const or_grid3d* g, const double* const* G, double* const* R) {
  const double s = -g->kappa2 / g->Z;
  for (int hc = 0; hc < 3; ++hc) {
    long n = or3d_field_size(g, 3 + hc);
    double* a = (double*)malloc(sizeof(double) * n);
    double* b = (double*)malloc(sizeof(double) * n);
    int p1 = (hc + 1) % 3, p2 = (hc + 2) % 3;
    pade_field3(g, p2, 3 + hc, p1, P_NODE_TO_HALF, G[p2], a);
    pade_field3(g, p1, 3 + hc, p2, P_NODE_TO_HALF, G[p1], b);
    for (long p = 0; p < n; ++p) R[hc][p] = s * (a[p] - b[p]);
    zero_walls3(g, 3 + hc, R[hc]);
    free(a);
    free(b);
  }
}

/* One full step (Sec. 3.4, Step 1 then Step 2) on f[0..5] = E_x, E_y, E_z, H_x, H_y, H_z. */
void or3d_step(or_grid3d* g, double* const* f) {
  double* G[3];
  double* R[3];
  double* X[3];
  for (int q = 0; q < 3; ++q) {
    long n = or3d_field_size(g, 3 + q) > or3d_field_size(g, q) ? or3d_field_size(g, 3 + q) : or3d_field_size(g, q);
    G[q] = (double*)malloc(sizeof(double) * n);
    R[q] = (double*)malloc(sizeof(double) * n);
    X[q] = (double*)malloc(sizeof(double) * n);
  }
  /* Step 1 */
  for (int q = 0; q < 3; ++q) or3d_filter(g, 3 + q, f[3 + q], G[q]);
  or3d_curl_h_to_e(g, (const double* const*)G, R);
  for (int q = 0; q < 3; ++q) {
    or3d_p1_solve_cg(g, q, R[q], X[q]);
    long n = or3d_field_size(g, q);
    for (long p = 0; p < n; ++p) f[q][p] += g->ht * X[q][p];
  }
  /* Step 2 */
  for (int q = 0; q < 3; ++q) or3d_filter(g, q, f[q], G[q]);
  or3d_curl_e_to_h(g, (const double* const*)G, R);
  for (int q = 0; q < 3; ++q) {
    or3d_p1_solve_cg(g, 3 + q, R[q], X[q]);
    long n = or3d_field_size(g, 3 + q);
    for (long p = 0; p < n; ++p) f[3 + q][p] += g->ht * X[q][p];
  }
  for (int q = 0; q < 3; ++q) {
    free(G[q]);
    free(R[q]);
    free(X[q]);
  }
}

/* Exact cavity modes (header comment), superposed.  modes[6m..6m+5] = (m, n, p, A_x, A_y, A_z)
 * with A . (m, n, p) = 0.  E at time tE, H at time tH; wall points are zero. */
void or3d_exact(const or_grid3d* g, const double* modes, int nmodes, double tE, double tH, double* const* f) {
  const int N = g->N;
  const double h = g->h, pi = M_PI;
  for (int c = 0; c < 6; ++c) memset(f[c], 0, sizeof(double) * or3d_field_size(g, c));
  for (int q = 0; q < nmodes; ++q) {
    const double* md = modes + 6 * q;
    const double a = pi * md[0], b = pi * md[1], cc = pi * md[2];
    const double Ax = md[3], Ay = md[4], Az = md[5];
    const double w = sqrt(a * a + b * b + cc * cc);
    const double ce = cos(w * tE), sh = -sin(w * tH) / (g->Z * w);
    /* amplitude and (sin = 0 / cos = 1) pattern per component and axis */
    const double amp[6] = {Ax * ce, Ay * ce, Az * ce, sh * (Az * b - Ay * cc), sh * (Ax * cc - Az * a),
                           sh * (Ay * a - Ax * b)};
    const double k3[3] = {a, b, cc};
    for (int c = 0; c < 6; ++c) {
      int d[3];
      or3d_dims(g, c, d);
      for (int k = 0; k < d[2]; ++k)
        for (int j = 0; j < d[1]; ++j)
          for (int i = 0; i < d[0]; ++i) {
            if (!unknown3(g, c, d, i, j, k)) continue;
            int idx[3] = {i, j, k};
            double v = amp[c];
            for (int ax = 0; ax < 3; ++ax) {
              /* node axes (Dirichlet) carry sin at x = idx h; half axes carry cos at (idx + 1/2) h */
              if (or3d_bc(c, ax) == BC_DIR3) v *= sin(k3[ax] * idx[ax] * h);
              else v *= cos(k3[ax] * (idx[ax] + 0.5) * h);
            }
            f[c][((size_t)k * d[1] + j) * d[0] + i] += v;
          }
    }
  }
  (void)N;
}

/* Error against the exact modes: out[0] = sqrt(h^3 sum (u - u_ex)^2) over the six components,
 * out[1] = out[0] / sqrt(h^3 sum u_ex^2), out[2] = max |u - u_ex|, out[3] = sum |u - u_ex|. */
void or3d_error(const or_grid3d* g, const double* modes, int nmodes, double tE, double tH, const double* const* f,
                double* out) {
  double* ex[6];
  for (int c = 0; c < 6; ++c) ex[c] = (double*)malloc(sizeof(double) * or3d_field_size(g, c));
  or3d_exact(g, modes, nmodes, tE, tH, ex);
  double s2 = 0.0, r2 = 0.0, mx = 0.0, s1 = 0.0;
  for (int c = 0; c < 6; ++c) {
    long n = or3d_field_size(g, c);
    for (long p = 0; p < n; ++p) {
      double e = f[c][p] - ex[c][p];
      s2 += e * e;
      r2 += ex[c][p] * ex[c][p];
      s1 += fabs(e);
      if (fabs(e) > mx) mx = fabs(e);
    }
    free(ex[c]);
  }
  double h3 = g->h * g->h * g->h;
  out[0] = sqrt(h3 * s2);
  out[1] = r2 > 0.0 ? sqrt(s2 / r2) : 0.0;
  out[2] = mx;
  out[3] = s1;
}

/* Discrete energy W^n = Z^{-1} ||E^n||^2 + Z <H^{n-1/2}, H^{n+1/2}> with h^3-weighted sums over
 * the stored points (wall values are zero): the 3D form of the leapfrog invariant of the 2D
 * diagnostic (the paper is silent on a discrete energy; Sec. 4 writes the scheme as a leapfrog).
 * f holds E^n and H^{n+1/2}; H^{n-1/2} = H^{n+1/2} - h_tau H*, with H* = P1^{-1} R_H(E^n) the
 * Step 2 increment (Sec. 3.4). */
double or3d_energy(or_grid3d* g, const double* const* f) {
  double* G[3];
  double* R[3];
  double* X[3];
  for (int q = 0; q < 3; ++q) {
    long n = or3d_field_size(g, 3 + q) > or3d_field_size(g, q) ? or3d_field_size(g, 3 + q) : or3d_field_size(g, q);
    G[q] = (double*)malloc(sizeof(double) * n);
    R[q] = (double*)malloc(sizeof(double) * n);
    X[q] = (double*)malloc(sizeof(double) * n);
  }
  for (int q = 0; q < 3; ++q) or3d_filter(g, q, f[q], G[q]);
  or3d_curl_e_to_h(g, (const double* const*)G, R);
  for (int q = 0; q < 3; ++q) or3d_p1_solve_cg(g, 3 + q, R[q], X[q]);
  double se = 0.0, sh = 0.0;
  for (int q = 0; q < 3; ++q) {
    long n = or3d_field_size(g, q);
    for (long p = 0; p < n; ++p) se += f[q][p] * f[q][p];
    n = or3d_field_size(g, 3 + q);
    for (long p = 0; p < n; ++p) sh += (f[3 + q][p] - g->ht * X[q][p]) * f[3 + q][p];
  }
  for (int q = 0; q < 3; ++q) {
    free(G[q]);
    free(R[q]);
    free(X[q]);
  }
  return g->h * g->h * g->h * (se / g->Z + g->Z * sh);
}

/* Pade divergence of H on the N^3 cell centres: div_h H = d_x H_x + d_y H_y + d_z H_z, each a
 * node -> half-node derivative of App. A.1 along its own axis (the 3D form of the 2D
 * diagnostic).  Returns sqrt(h^3 sum div^2); div_out (N^3, [z][y][x]) may be NULL. */
double or3d_divergence(const or_grid3d* g, const double* const* f, double* div_out) {
  const int N = g->N;
  const long nc = (long)N * N * N;
  double* div = div_out ? div_out : (double*)malloc(sizeof(double) * nc);
  double* line = (double*)malloc(sizeof(double) * (N + 1));
  double* dl = (double*)malloc(sizeof(double) * N);
  for (long p = 0; p < nc; ++p) div[p] = 0.0;
  for (int a = 0; a < 3; ++a) {
    int d[3];
    or3d_dims(g, 3 + a, d); /* d[a] = N + 1 nodes along a, N half points across */
    const double* u = f[3 + a];
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j) {
        /* the line along axis a through centre indices (j, k) of the two other axes */
        for (int t = 0; t <= N; ++t) {
          int c[3];
          c[a] = t;
          c[(a + 1) % 3] = j;
          c[(a + 2) % 3] = k;
          line[t] = u[((long)c[2] * d[1] + c[1]) * d[0] + c[0]];
        }
        or_pade_line(N, g->closure, P_NODE_TO_HALF, g->h, line, dl);
        for (int t = 0; t < N; ++t) {
          int c[3];
          c[a] = t;
          c[(a + 1) % 3] = j;
          c[(a + 2) % 3] = k;
          div[((long)c[2] * N + c[1]) * N + c[0]] += dl[t];
        }
      }
  }
  double s = 0.0;
  for (long p = 0; p < nc; ++p) s += div[p] * div[p];
  free(line);
  free(dl);
  if (!div_out) free(div);
  return sqrt(g->h * g->h * g->h * s);
}

long or3d_cg_iters_total(const or_grid3d* g) { return g->cg_iters_total; }
long or3d_cg_solves(const or_grid3d* g) { return g->cg_solves; }

/* ------------------------------------------------------------------ */
/* Current sources on 3D grids: divergence-free driven modes shaped like a cavity mode's E,
 *   J = (a_x cos ax sin by sin cz, a_y sin ax cos by sin cz, a_z sin ax sin by cos cz) sin(w t),
 *   (a, b, c) = pi (m, n, p),  (a_x, a_y, a_z) . (m, n, p) = 0,
 * rows (m, n, p, a_x, a_y, a_z, w).  div J = 0, so rho = 0 and the normal data of E stay
 * homogeneous (d_n E_n = rho = 0); the tangential components of J vanish on every wall with all
 * the derivatives the Neumann data of H involve (Sec. 3.3), so the even ghosts of Cor.
 * "cor:ghost_cor" stay exact.  The source terms are those of the 2D oracle's add_sources_e /
 * add_sources_h written for the vector current (Sec. 3.1: the Taylor expansion with Faraday's and
 * Ampere's laws):
 *   E:  P(J) = Z (-kappa^2 J + grad div J - d_tt J) = -Z (kappa^2 - w^2) J     at t^{n+1/2},
 *   H:  + curl d_t J = w cos(w t) (a_z b - a_y c, a_x c - a_z a, a_y a - a_x b) (H-mode shapes)  at t^{n+1},
 * each through the right-hand-side filter of Eq. "eq:ell" with the exact Laplacian of the source
 * (factor beta - (h^2/12)(a^2 + b^2 + c^2)).  A source with p = 0 is J = a_z sin ax sin by z^, the
 * 2D TM_z source extended in z (likewise m = 0, n = 0 in the other orientations). */

/* R[q] += amp[q] * shape of component (side == 0 ? q : 3 + q) with the wavenumbers k3. */
static void add_shaped3(const or_grid3d* g, int side, const double* k3, const double* amp, double* const* R) {
  const double h = g->h;
  for (int q = 0; q < 3; ++q) {
    const int c = side == 0 ? q : 3 + q;
    int d[3];
    or3d_dims(g, c, d);
    for (int k = 0; k < d[2]; ++k)
      for (int j = 0; j < d[1]; ++j)
        for (int i = 0; i < d[0]; ++i) {
          if (!unknown3(g, c, d, i, j, k)) continue;
          int idx[3] = {i, j, k};
          double v = amp[q];
          for (int ax = 0; ax < 3; ++ax) {
            if (or3d_bc(c, ax) == BC_DIR3) v *= sin(k3[ax] * idx[ax] * h);
            else v *= cos(k3[ax] * (idx[ax] + 0.5) * h);
          }
          R[q][((size_t)k * d[1] + j) * d[0] + i] += v;
        }
  }
}

static void add_sources3(const or_grid3d* g, const double* src, int nsrc, double t, int side, double* const* R) {
  for (int q = 0; q < nsrc; ++q) {
    const double* s = src + 7 * q;
    const double k3[3] = {M_PI * s[0], M_PI * s[1], M_PI * s[2]};
    const double ax = s[3], ay = s[4], az = s[5], w = s[6];
    const double filt = g->beta - (g->h * g->h / 12.0) * (k3[0] * k3[0] + k3[1] * k3[1] + k3[2] * k3[2]);
    double amp[3];
    if (side == 0) {
      const double f = -g->Z * (g->kappa2 - w * w) * filt * sin(w * t);
      amp[0] = f * ax;
      amp[1] = f * ay;
      amp[2] = f * az;
    } else {
      const double f = filt * w * cos(w * t);
      amp[0] = f * (az * k3[1] - ay * k3[2]);
      amp[1] = f * (ax * k3[2] - az * k3[0]);
      amp[2] = f * (ay * k3[0] - ax * k3[1]);
    }
    add_shaped3(g, side, k3, amp, R);
  }
}

/* One full step with sources: or3d_step with P(J)^{n+1/2} added to the E right-hand sides and
 * curl d_t J^{n+1} to the H right-hand sides; n is the index of the step (E^n -> E^{n+1}). */
void or3d_step_src(or_grid3d* g, double* const* f, const double* src, int nsrc, long n) {
  double* G[3];
  double* R[3];
  double* X[3];
  for (int q = 0; q < 3; ++q) {
    long m = or3d_field_size(g, 3 + q) > or3d_field_size(g, q) ? or3d_field_size(g, 3 + q) : or3d_field_size(g, q);
    G[q] = (double*)malloc(sizeof(double) * m);
    R[q] = (double*)malloc(sizeof(double) * m);
    X[q] = (double*)malloc(sizeof(double) * m);
  }
  for (int q = 0; q < 3; ++q) or3d_filter(g, 3 + q, f[3 + q], G[q]);
  or3d_curl_h_to_e(g, (const double* const*)G, R);
  add_sources3(g, src, nsrc, (n + 0.5) * g->ht, 0, R);
  for (int q = 0; q < 3; ++q) {
    or3d_p1_solve_cg(g, q, R[q], X[q]);
    long m = or3d_field_size(g, q);
    for (long p = 0; p < m; ++p) f[q][p] += g->ht * X[q][p];
  }
  for (int q = 0; q < 3; ++q) or3d_filter(g, q, f[q], G[q]);
  or3d_curl_e_to_h(g, (const double* const*)G, R);
  add_sources3(g, src, nsrc, (n + 1.0) * g->ht, 1, R);
  for (int q = 0; q < 3; ++q) {
    or3d_p1_solve_cg(g, 3 + q, R[q], X[q]);
    long m = or3d_field_size(g, 3 + q);
    for (long p = 0; p < m; ++p) f[3 + q][p] += g->ht * X[q][p];
  }
  for (int q = 0; q < 3; ++q) {
    free(G[q]);
    free(R[q]);
    free(X[q]);
  }
}

/* Exact driven solution for these sources (particular solution, w^2 != a^2 + b^2 + c^2), from
 * d_tt E = Delta E - Z d_t J (div E = 0) and Faraday's law:
 *   E = A cos(w t) (a_x, a_y, a_z) (E-mode shapes),  A = Z w / (w^2 - (a^2 + b^2 + c^2)),
 *   H = -(A sin(w t) / (Z w)) (a_z b - a_y c, a_x c - a_z a, a_y a - a_x b) (H-mode shapes),
 * at times tE, tH; wall points zero. */
void or3d_exact_driven(const or_grid3d* g, const double* src, int nsrc, double tE, double tH, double* const* f) {
  for (int c = 0; c < 6; ++c) memset(f[c], 0, sizeof(double) * or3d_field_size(g, c));
  for (int q = 0; q < nsrc; ++q) {
    const double* s = src + 7 * q;
    const double k3[3] = {M_PI * s[0], M_PI * s[1], M_PI * s[2]};
    const double ax = s[3], ay = s[4], az = s[5], w = s[6];
    const double A = g->Z * w / (w * w - (k3[0] * k3[0] + k3[1] * k3[1] + k3[2] * k3[2]));
    const double ce = A * cos(w * tE), sh = -A * sin(w * tH) / (g->Z * w);
    const double ae[3] = {ce * ax, ce * ay, ce * az};
    const double ah[3] = {sh * (az * k3[1] - ay * k3[2]), sh * (ax * k3[2] - az * k3[0]), sh * (ay * k3[0] - ax * k3[1])};
    add_shaped3(g, 0, k3, ae, f);
    add_shaped3(g, 1, k3, ah, f + 3);
  }
}
