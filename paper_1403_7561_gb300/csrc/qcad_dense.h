// Schrodinger subdomain map, dense block kernels of LOBPCG and the small
// host-side dense linear algebra of its Rayleigh-Ritz step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define QCAD_DENSE_MAXP 128

namespace qcad {

// Element block [i0, i0+nxs) x [j0, j0+nys) x [k0, k0+nzs) of a mesh with
// nxn x nyn nodes per plane.
struct SubdomainMap {
  int i0, j0, k0;
  int nxs, nys, nzs;   // subdomain elements per axis
  long long nxn, nyn;  // global mesh nodes per axis (x, y)
};

template <class T>
void launch_potential(const SubdomainMap& sm, const double* phi, double V0, const double* hx, const double* hy,
                      const double* hz, const double* vxq /* extra potential at the Gauss points or null */, T* cV,
                      double* vmin, cudaStream_t s);
void launch_pack(const SubdomainMap& sm, int nvec, double* full, long long ldf, double* dof, long long ldd,
                 int unpack, cudaStream_t s);
// G1 = A^T B1 and, if B2 is not null, G2 = A^T B2 (p x p each, row-major, FP64, overwritten;
// q must equal p). part: device scratch of gram_part_doubles(p, p) doubles. p <= 64. upper: the
// double-float kernel may form only the entries a <= b (the others are then unspecified).
template <class T>
void launch_gram(long long n, int p, int q, const T* A, long long lda, const T* B1, const T* B2, long long ldb,
                 double* G1, double* G2, double* part, cudaStream_t s, bool upper = false);
size_t gram_part_doubles(int p, int q);
// p <= 64. nbase > 1: the same C applied to nbase block sets, set b at A, Y1, Y2 + b * bstride.
// LOBPCG update of [X | W | P] (nb columns each at stride ld; nbase block sets bstride elements
// apart): P' = [W P] Cz, X' = X Cx + P' in place, with C = [Cx; Cz] the (nb + nz) x nb coefficients
// of the first nb Ritz vectors (column-major); nz <= 2 nb (the W and P columns in use); nb <= 20.
template <class T>
void launch_lobpcg_update(long long n, int nb, int nz, T* S, long long ld, const T* C, cudaStream_t s, int nbase,
                          long long bstride);
// Column moves within column-major blocks: column src[t] to column dst[t] for t < n (n <= 40),
// each row's sources read before any of its destinations is written, so sources and
// destinations may overlap; nbase block sets bstride elements apart, as launch_lobpcg_update.
struct ColMoves {
  int n;
  short src[40], dst[40];
};
template <class T>
void launch_move_cols(long long n, T* S, long long ld, const ColMoves& mv, cudaStream_t s, int nbase,
                      long long bstride);
template <class T>
void launch_combine(long long n, int p, int q, int q1, const T* A, long long lda, const T* C, T* Y1, T* Y2,
                    long long ldy, cudaStream_t s, int nbase = 1, long long bstride = 0);
template <class T>
void launch_residual_block(long long n, int m, const T* HX, const T* MX, long long ld, const double* lam,
                           const T* dinv, T* W, double* norms, cudaStream_t s);
template <class T>
void launch_cheb_block_init(long long n, int m, long long ld, const T* R, const T* dinv, double inv_theta, T* W,
                            T* D, T* Z, cudaStream_t s);
template <class T>
void launch_cheb_block_step(long long n, int m, long long ld, const T* HD, const T* dinv, double c1, double c2,
                            T* W, T* D, T* Z, cudaStream_t s);
template <class T>
void launch_power_sub(long long n, const T* v, const T* Hv, const T* dinv, T* vn, double* acc, cudaStream_t s);
// Box modes (a, b, c) >= 1 of the columns of a smooth starting block (at most 32 columns).
struct BoxModes {
  int a[32], b[32], c[32];
};
template <class T>
void launch_box_mode_block(long long n, int m, long long ld, int nx, int ny, int nz, const BoxModes& modes, double eps,
                           const unsigned char* interior, uint64_t seed, T* X, cudaStream_t s);
template <class T>
void launch_random_block(long long n, int m, long long ld, const unsigned char* interior, uint64_t seed, T* X,
                         cudaStream_t s);

// Host dense routines on column-major n x n matrices (n <= QCAD_DENSE_MAXP).
// Cholesky A = L L^T in place (lower); returns false if A is not numerically SPD.
bool dense_cholesky(int n, double* A);
// Symmetric eigen-decomposition (Householder tridiagonalization, implicit QR): A is destroyed,
// w ascending eigenvalues, V column eigenvectors.
void dense_sym_eig(int n, double* A, double* w, double* V);
// Generalized symmetric-definite problem A x = lam B x via Cholesky of B:
// returns false if B is not SPD. X is B-orthonormal.
bool dense_gen_eig(int n, const double* A, const double* B, double* w, double* X);
// Inverse of the lower Cholesky factor's transpose applied from the right:
// returns Rinv (n x n, column-major) with B = L L^T and Rinv = L^-T.
void dense_inv_lt(int n, const double* L, double* Rinv);

}  // namespace qcad
