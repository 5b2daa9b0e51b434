// Host-side set-up: Pade operator tables and the stability limit.
//
// The Pade first derivative of App. A.1 (Eq. "eq:lhs") is  A f' = D1 f / h  with A the
// M x M matrix [1,22,1]/24 in the interior and one-sided end rows.  Its inverse decays like
// |rho|^|i-j|, rho = -11 + sqrt(120) ~ -0.0455, so W = A^{-1} D1~ (D1~ the plain difference)
// is banded to any working precision.  The GPU applies W as an explicit stencil: one
// Toeplitz row for the interior and explicit rows near both ends, found here by solving
// A^T z = e_i for the rows of A^{-1}.
#include <cmath>
#include <cstring>

#include "k_fp64.cuh"

namespace ms {

Shape field_shape(int N, int f) {
  if (f == EZ) return Shape{N + 1, N + 1, DIR, DIR};
  if (f == HX) return Shape{N + 1, N, DIR, NEU};
  return Shape{N, N + 1, NEU, DIR};
}

// Entries of 24*A: returns the number of (col, val) pairs of row i.
static int row24(int M, int closure, int kind, int i, int* col, double* val) {
  if (i == 0 || i == M - 1) {
    const bool first = (i == 0);
    if (closure == MS_CLOSURE_PAPER) {
      const double c[4] = {26.0, -5.0, 4.0, -1.0};
      for (int k = 0; k < 4; ++k) {
        col[k] = first ? k : M - 1 - k;
        val[k] = c[k];
      }
      return 4;
    }
    // REFLECT: the derivative on half-nodes of a field vanishing at the wall is even about it
    // (diagonal 23); the derivative at nodes of a field even about the wall vanishes there (22).
    col[0] = i;
    val[0] = (kind == NODE_TO_HALF) ? 23.0 : 22.0;
    col[1] = first ? i + 1 : i - 1;
    val[1] = 1.0;
    return 2;
  }
  col[0] = i - 1; val[0] = 1.0;
  col[1] = i;     val[1] = 22.0;
  col[2] = i + 1; val[2] = 1.0;
  return 3;
}

// Row i of (24 A)^{-1}: solve (24 A)^T z = e_i by banded elimination (A^T is column
// diagonally dominant, so no pivoting is needed).  Bandwidth 3 on both sides.
static void inverse_row24(int M, int closure, int kind, int i, std::vector<double>* z) {
  const int P = 3, W = 2 * P + 1;
  std::vector<double> band((size_t)M * W, 0.0);  // band[r*W + (c - r + P)] = (24A)^T (r, c)
  for (int r = 0; r < M; ++r) {
    int col[4];
    double val[4];
    int n = row24(M, closure, kind, r, col, val);
    for (int k = 0; k < n; ++k) {
      // entry (r, col) of 24A is entry (col, r) of its transpose
      band[(size_t)col[k] * W + (r - col[k] + P)] += val[k];
    }
  }
  std::vector<double>& x = *z;
  x.assign(M, 0.0);
  x[i] = 1.0;
  for (int k = 0; k < M; ++k) {
    const double piv = band[(size_t)k * W + P];
    for (int r = k + 1; r <= k + P && r < M; ++r) {
      double a = band[(size_t)r * W + (k - r + P)];
      if (a == 0.0) continue;
      const double l = a / piv;
      for (int c = k; c <= k + P && c < M; ++c) band[(size_t)r * W + (c - r + P)] -= l * band[(size_t)k * W + (c - k + P)];
      x[r] -= l * x[k];
    }
  }
  for (int r = M - 1; r >= 0; --r) {
    double s = x[r];
    for (int c = r + 1; c <= r + P && c < M; ++c) s -= band[(size_t)r * W + (c - r + P)] * x[c];
    x[r] = s / band[(size_t)r * W + P];
  }
}

void pade_dense_row(int M, int closure, int kind, int i, std::vector<double>* row) {
  std::vector<double> z;
  inverse_row24(M, closure, kind, i, &z);
  row->assign(M + 1, 0.0);
  // W = (24A)^{-1} * 24 * D1~, (D1~ f)_m = f_{m+1} - f_m  =>  W_{i,k} = 24 (z_{k-1} - z_k)
  for (int k = 0; k <= M; ++k) {
    double zm1 = (k >= 1) ? z[k - 1] : 0.0;
    double zk = (k < M) ? z[k] : 0.0;
    (*row)[k] = 24.0 * (zm1 - zk);
  }
}

static double tail_outside(const std::vector<double>& row, int i, int K) {
  double s = 0.0;
  for (int k = 0; k < (int)row.size(); ++k)
    if (k < i - K || k > i + K + 1) s += std::fabs(row[k]);
  return s;
}

static double abs_sum(const std::vector<double>& row) {
  double s = 0.0;
  for (double v : row) s += std::fabs(v);
  return s;
}

// Row i of A^{-1} itself (length M): the operator applied to first differences.
static void inverse_row(int M, int closure, int kind, int i, std::vector<double>* row) {
  inverse_row24(M, closure, kind, i, row);
  for (double& v : *row) v *= 24.0;
}

int build_pade_table(int M, int closure, int kind, double tol, PadeTable* t, std::string* err, bool of_differences) {
  if (M < 4) {
    *err = "Pade line too short (need at least 4 outputs)";
    return -1;
  }
  auto dense_row = [&](int i, std::vector<double>* r) {
    if (of_differences) inverse_row(M, closure, kind, i, r);
    else pade_dense_row(M, closure, kind, i, r);
  };
  // Band half-width K from the middle row, then widened until every end row also fits.
  const int mid = M / 2;
  std::vector<double> row;
  dense_row(mid, &row);
  int K = 1;
  while (K < M && tail_outside(row, mid, K) > tol * abs_sum(row)) ++K;
  const int probe = std::min(M, 40);
  for (int i = 0; i < probe; ++i) {
    for (int side = 0; side < 2; ++side) {
      int ii = side ? M - 1 - i : i;
      dense_row(ii, &row);
      while (K < M && tail_outside(row, ii, K) > tol * abs_sum(row)) ++K;
    }
  }
  // B: first row index from which the rows equal the interior row (within tol) up to M-1-B.
  std::vector<double> mrow;
  dense_row(mid, &mrow);
  const double ref = abs_sum(mrow);
  int B = K + 1;
  for (;; ++B) {
    if (2 * B >= M) break;
    bool same = true;
    for (int side = 0; side < 2 && same; ++side) {
      int ii = side ? M - 1 - B : B;
      dense_row(ii, &row);
      for (int d = -K; d <= K + 1; ++d) {
        double a = row[ii + d], b = mrow[mid + d];
        if (std::fabs(a - b) > tol * ref) { same = false; break; }
      }
    }
    if (same) break;
  }
  t->M = M;
  t->K = K;
  t->rows = M;
  t->n_in = M + 1;
  t->left = K;
  t->all_explicit = (2 * B >= M);
  if (t->all_explicit) B = M;
  t->B = B;
  const int rs = t->row_stride();
  // Layout: B head rows, then (unless all explicit) B tail rows, then the interior row.
  const int nrows = t->all_explicit ? M + 1 : 2 * B + 1;
  t->w.assign((size_t)nrows * rs, 0.0);
  auto put = [&](int slot, int i) {
    dense_row(i, &row);
    for (int d = -K; d <= K + 1; ++d) {
      int k = i + d;
      if (k >= 0 && k < (int)row.size()) t->w[(size_t)slot * rs + (d + K)] = row[k];
    }
  };
  if (t->all_explicit) {
    for (int i = 0; i < M; ++i) put(i, i);
    put(M, mid);
  } else {
    for (int i = 0; i < B; ++i) put(i, i);
    for (int i = 0; i < B; ++i) put(B + i, M - B + i);
    put(2 * B, mid);
  }
  return 0;
}

void build_pade_table_T(const PadeTable& f, PadeTable* t) {
  const int M = f.M, K = f.K, rs = f.row_stride();
  // entry (i, k) of the forward band: output i, input k
  auto W = [&](int i, int k) {
    if (i < 0 || i >= M) return 0.0;
    const int d = k - i + K;
    if (d < 0 || d > 2 * K + 1) return 0.0;
    return pade_row_ptr(f.w.data(), i, M, K, f.B, f.all_explicit)[d];
  };
  // W^T row k reads W column k at rows k - K - 1 .. k + K; it is the reversed interior row as
  // soon as all of those rows are interior rows of W, i.e. away from B + K + 1 rows of each end.
  const int R = M + 1;
  int B = f.B + K + 1;
  t->M = M;
  t->K = K;
  t->rows = R;
  t->n_in = M;
  t->left = K + 1;
  t->all_explicit = f.all_explicit || 2 * B >= R;
  if (t->all_explicit) B = R;
  t->B = B;
  const int nrows = t->all_explicit ? R + 1 : 2 * B + 1;
  t->w.assign((size_t)nrows * rs, 0.0);
  auto put = [&](int slot, int k) {
    for (int s = 0; s < rs; ++s) t->w[(size_t)slot * rs + s] = W(k - (K + 1) + s, k);
  };
  if (t->all_explicit) {
    for (int k = 0; k < R; ++k) put(k, k);
    put(R, R / 2);
  } else {
    for (int k = 0; k < B; ++k) put(k, k);
    for (int k = 0; k < B; ++k) put(B + k, R - B + k);
    put(2 * B, R / 2);
  }
}

// Fourier symbol of one full step (Sec. 4): a mode is neutrally stable iff
// (h_tau lambda)^2 = r^2 g^2 (d_x^2 + d_y^2) <= 4 in units h = 1, with d the Pade symbol and
// g = kappa^2 (beta - (mu_x + mu_y)/12) / (kappa^2 beta + mu_x + mu_y - mu_x mu_y / 6).
static double max_amp2_2d(double r) {
  const double k2 = 24.0 / (r * r), beta = 1.0 + 2.0 / (r * r);
  double worst = 0.0;
  const int n = 256;
  for (int a = 1; a <= n; ++a) {
    double tx = M_PI * a / n;
    double mx = 4.0 * std::sin(tx / 2) * std::sin(tx / 2);
    double dx = 2.0 * std::sin(tx / 2) * 12.0 / (11.0 + std::cos(tx));
    for (int b = 1; b <= n; ++b) {
      double ty = M_PI * b / n;
      double my = 4.0 * std::sin(ty / 2) * std::sin(ty / 2);
      double dy = 2.0 * std::sin(ty / 2) * 12.0 / (11.0 + std::cos(ty));
      double g = k2 * (beta - (mx + my) / 12.0) / (k2 * beta + mx + my - mx * my / 6.0);
      double v = r * r * g * g * (dx * dx + dy * dy);
      if (v > worst) worst = v;
    }
  }
  return worst;
}

double stability_limit_2d() {
  static double cached = 0.0;
  if (cached > 0.0) return cached;
  double lo = 0.3, hi = 1.0;
  for (int it = 0; it < 60; ++it) {
    double mid = 0.5 * (lo + hi);
    if (max_amp2_2d(mid) <= 4.0) lo = mid;
    else hi = mid;
  }
  cached = lo;
  return cached;
}

}  // namespace ms
