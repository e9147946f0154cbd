// Small dense symmetric linear algebra for the LOBPCG Rayleigh-Ritz step
// (host, FP64): Cholesky factorization, the symmetric eigenproblem
// (Householder tridiagonalization and implicit shifted QR), and the
// generalized symmetric-definite eigenproblem by Cholesky reduction.
#include <algorithm>
#include <cmath>
#include <vector>

#include "qcad_dense.h"

namespace qcad {

#define A_(i, j) A[(size_t)(j) * n + (i)]

bool dense_cholesky(int n, double* A) {
  // left-looking by columns: column j less its earlier columns scaled by row j (the same
  // subtractions, in the same order, as the row-wise dot products), then scaled by 1 / L(j, j)
  for (int j = 0; j < n; ++j) {
    double* cj = A + (size_t)j * n;
    for (int k = 0; k < j; ++k) {
      const double* ck = A + (size_t)k * n;
      const double f = ck[j];
      for (int i = j; i < n; ++i) cj[i] -= ck[i] * f;
    }
    const double d = cj[j];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double l = std::sqrt(d);
    cj[j] = l;
    for (int i = j + 1; i < n; ++i) cj[i] /= l;
    for (int i = 0; i < j; ++i) cj[i] = 0.0;
  }
  return true;
}

// Symmetric eigenproblem in two stages: Householder reduction to tridiagonal form
// T = Q^T A Q (Q accumulated), then the implicit symmetric QR iteration with Wilkinson
// shifts on T, each step a chase of the bulge by Givens rotations that are accumulated
// into Q. O(n^3) with a small constant; eigenvalues ascending on return.
void dense_sym_eig(int n, double* A, double* w, double* V) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) V[(size_t)j * n + i] = (i == j) ? 1.0 : 0.0;
  std::vector<double> v(n), p(n), wv(n), t(n);
  // Householder: column k below the subdiagonal is annihilated by H = I - 2 u u^T acting on
  // rows/columns k+1..n-1 (A22 <- A22 - 2 u w^T - 2 w u^T, w = A22 u - (u^T A22 u) u).
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double xn2 = 0.0;
    for (int i = 0; i < m; ++i) {
      v[i] = A_(k + 1 + i, k);
      xn2 += v[i] * v[i];
    }
    const double xn = std::sqrt(xn2);
    if (xn == 0.0) continue;
    const double alpha = v[0] > 0.0 ? -xn : xn;
    v[0] -= alpha;
    double vn2 = 0.0;
    for (int i = 0; i < m; ++i) vn2 += v[i] * v[i];
    if (vn2 == 0.0) continue;
    const double inv = 1.0 / std::sqrt(vn2);
    for (int i = 0; i < m; ++i) v[i] *= inv;
    // p = A22 v, row i taken as column i (A22 is symmetric), so that the inner loops run down columns
    double up = 0.0;
    for (int i = 0; i < m; ++i) {
      const double* col = A + (size_t)(k + 1 + i) * n + (k + 1);
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += col[j] * v[j];
      p[i] = s;
      up += v[i] * s;
    }
    for (int i = 0; i < m; ++i) wv[i] = p[i] - up * v[i];
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) A_(k + 1 + i, k + 1 + j) -= 2.0 * (v[i] * wv[j] + wv[i] * v[j]);
    A_(k + 1, k) = alpha;
    A_(k, k + 1) = alpha;
    for (int i = 1; i < m; ++i) {
      A_(k + 1 + i, k) = 0.0;
      A_(k, k + 1 + i) = 0.0;
    }
    // V <- V H on columns k+1..n-1: t = V[:, k+1:] v, then V[:, k+1+i] -= 2 v_i t (column sweeps)
    std::fill(t.begin(), t.end(), 0.0);
    for (int i = 0; i < m; ++i) {
      const double* col = V + (size_t)(k + 1 + i) * n;
      const double vi = v[i];
      for (int r = 0; r < n; ++r) t[r] += col[r] * vi;
    }
    for (int i = 0; i < m; ++i) {
      double* col = V + (size_t)(k + 1 + i) * n;
      const double f = 2.0 * v[i];
      for (int r = 0; r < n; ++r) col[r] -= f * t[r];
    }
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = A_(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = A_(i + 1, i);
  // implicit QR on the tridiagonal (d, e): deflate from the bottom, chase one bulge per step
  const double eps = 2.220446049250313e-16;
  int m = n - 1, guard = 0;
  while (m > 0 && guard < 60 * n) {
    if (std::fabs(e[m - 1]) <= eps * (std::fabs(d[m - 1]) + std::fabs(d[m]))) {
      e[m - 1] = 0.0;
      --m;
      continue;
    }
    int l = m - 1;
    while (l > 0 && std::fabs(e[l - 1]) > eps * (std::fabs(d[l - 1]) + std::fabs(d[l]))) --l;
    ++guard;
    // Wilkinson shift: eigenvalue of the trailing 2x2 block nearer to d[m]
    const double delta = 0.5 * (d[m - 1] - d[m]);
    const double b2 = e[m - 1] * e[m - 1];
    const double den = delta + (delta >= 0.0 ? 1.0 : -1.0) * std::sqrt(delta * delta + b2);
    const double mu = den != 0.0 ? d[m] - b2 / den : d[m];
    double x = d[l] - mu, y = e[l], bulge = 0.0;
    for (int k = l; k < m; ++k) {
      if (k > l) {
        x = e[k - 1];
        y = bulge;
      }
      // the projected matrices' entries are far from the overflow and underflow thresholds
      const double r = std::sqrt(x * x + y * y);
      const double c = r != 0.0 ? x / r : 1.0, s = r != 0.0 ? y / r : 0.0;
      if (k > l) e[k - 1] = r;
      const double a = d[k], b = e[k], cc = d[k + 1];
      d[k] = c * c * a + 2.0 * c * s * b + s * s * cc;
      e[k] = c * s * (cc - a) + (c * c - s * s) * b;
      d[k + 1] = s * s * a - 2.0 * c * s * b + c * c * cc;
      if (k + 1 < m) {
        bulge = s * e[k + 1];
        e[k + 1] *= c;
      }
      double* vk = V + (size_t)k * n;
      double* vk1 = V + (size_t)(k + 1) * n;
      for (int r2 = 0; r2 < n; ++r2) {
        const double a0 = vk[r2], a1 = vk1[r2];
        vk[r2] = c * a0 + s * a1;
        vk1[r2] = -s * a0 + c * a1;
      }
    }
  }
  // sort ascending
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] < d[b]; });
  std::vector<double> Vs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = d[idx[j]];
    for (int i = 0; i < n; ++i) Vs[(size_t)j * n + i] = V[(size_t)idx[j] * n + i];
  }
  std::copy(Vs.begin(), Vs.end(), V);
}

void dense_inv_lt(int n, const double* L, double* R) {
  // Solve L^T R = I column by column (R upper triangular: rows below j of column j are zero).
  for (int j = 0; j < n; ++j) {
    double* rj = R + (size_t)j * n;
    for (int i = j + 1; i < n; ++i) rj[i] = 0.0;
    for (int i = j; i >= 0; --i) {
      const double* li = L + (size_t)i * n;  // column i of L: L(k, i) for k > i
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = i + 1; k <= j; ++k) s -= li[k] * rj[k];
      rj[i] = s / li[i];
    }
  }
}

bool dense_gen_eig(int n, const double* A, const double* B, double* w, double* X) {
  std::vector<double> L(B, B + (size_t)n * n);
  if (!dense_cholesky(n, L.data())) return false;
  std::vector<double> R((size_t)n * n);
  dense_inv_lt(n, L.data(), R.data());  // R = L^-T
  // C = R^T A R
  std::vector<double> AR((size_t)n * n, 0.0), C((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) {
      const double r = R[(size_t)j * n + k];
      if (r == 0.0) continue;
      for (int i = 0; i < n; ++i) AR[(size_t)j * n + i] += A[(size_t)k * n + i] * r;
    }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int k = 0; k <= i; ++k) s += R[(size_t)i * n + k] * AR[(size_t)j * n + k];  // R upper triangular
      C[(size_t)j * n + i] = s;
    }
  // symmetrize against rounding
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < j; ++i) {
      const double s = 0.5 * (C[(size_t)j * n + i] + C[(size_t)i * n + j]);
      C[(size_t)j * n + i] = s;
      C[(size_t)i * n + j] = s;
    }
  std::vector<double> V((size_t)n * n);
  dense_sym_eig(n, C.data(), w, V.data());
  // X = R V (column j of X as a sum of columns of R)
  for (int j = 0; j < n; ++j) {
    double* xj = X + (size_t)j * n;
    std::fill(xj, xj + n, 0.0);
    for (int k = 0; k < n; ++k) {
      const double f = V[(size_t)j * n + k];
      const double* rk = R.data() + (size_t)k * n;
      for (int i = 0; i < n; ++i) xj[i] += rk[i] * f;
    }
  }
  return true;
}

#undef A_

}  // namespace qcad
