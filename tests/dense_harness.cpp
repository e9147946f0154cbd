// C entry points to the host dense routines of the LOBPCG Rayleigh-Ritz step, compiled by
// tests/test_dense_host.py together with the library's dense.cpp (CPU only).
#include "qcad_dense.h"

extern "C" {
void h_sym_eig(int n, double* A, double* w, double* V) { qcad::dense_sym_eig(n, A, w, V); }
int h_gen_eig(int n, const double* A, const double* B, double* w, double* X) {
  return qcad::dense_gen_eig(n, A, B, w, X) ? 1 : 0;
}
int h_cholesky(int n, double* A) { return qcad::dense_cholesky(n, A) ? 1 : 0; }
void h_inv_lt(int n, const double* L, double* R) { qcad::dense_inv_lt(n, L, R); }
}
