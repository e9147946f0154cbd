// Small dense symmetric linear algebra for the LOBPCG Rayleigh-Ritz step
// (host, FP64): Cholesky factorization, cyclic Jacobi eigenvalue iteration,
// and the generalized symmetric-definite eigenproblem by Cholesky reduction.
#include <algorithm>
#include <cmath>
#include <vector>

#include "qcad_dense.h"

namespace qcad {

#define A_(i, j) A[(size_t)(j) * n + (i)]

bool dense_cholesky(int n, double* A) {
  for (int j = 0; j < n; ++j) {
    double d = A_(j, j);
    for (int k = 0; k < j; ++k) d -= A_(j, k) * A_(j, k);
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double l = std::sqrt(d);
    A_(j, j) = l;
    for (int i = j + 1; i < n; ++i) {
      double s = A_(i, j);
      for (int k = 0; k < j; ++k) s -= A_(i, k) * A_(j, k);
      A_(i, j) = s / l;
    }
    for (int i = 0; i < j; ++i) A_(i, j) = 0.0;
  }
  return true;
}

void dense_sym_eig(int n, double* A, double* w, double* V) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) V[(size_t)j * n + i] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int j = 0; j < n; ++j) {
      diag += A_(j, j) * A_(j, j);
      for (int i = 0; i < j; ++i) off += A_(i, j) * A_(i, j);
    }
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = A_(p, q);
        if (apq == 0.0) continue;
        const double app = A_(p, p), aqq = A_(q, q);
        // rotation angle that annihilates A(p,q)
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A_(k, p), akq = A_(k, q);
          A_(k, p) = c * akp - s * akq;
          A_(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A_(p, k), aqk = A_(q, k);
          A_(p, k) = c * apk - s * aqk;
          A_(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)p * n + k], vkq = V[(size_t)q * n + k];
          V[(size_t)p * n + k] = c * vkp - s * vkq;
          V[(size_t)q * n + k] = s * vkp + c * vkq;
        }
      }
    }
  }
  // sort ascending
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A_(a, a) < A_(b, b); });
  std::vector<double> Vs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = A_(idx[j], idx[j]);
    for (int i = 0; i < n; ++i) Vs[(size_t)j * n + i] = V[(size_t)idx[j] * n + i];
  }
  std::copy(Vs.begin(), Vs.end(), V);
}

void dense_inv_lt(int n, const double* L, double* R) {
  // Solve L^T R = I column by column (R upper triangular).
  for (int j = 0; j < n; ++j) {
    for (int i = n - 1; i >= 0; --i) {
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)i * n + k] * R[(size_t)j * n + k];
      R[(size_t)j * n + i] = s / L[(size_t)i * n + i];
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
      for (int k = 0; k < n; ++k) s += R[(size_t)i * n + k] * AR[(size_t)j * n + k];
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
  // X = R V
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += R[(size_t)k * n + i] * V[(size_t)j * n + k];
      X[(size_t)j * n + i] = s;
    }
  return true;
}

#undef A_

}  // namespace qcad
