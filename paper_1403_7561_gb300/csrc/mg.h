// Geometric multigrid V-cycle preconditioner for the Jacobian J = K + M_c of the Newton-Krylov
// solve, in FP32 (mixed precision) or FP64 (plain FP64) (a preconditioner choice: the paper
// leaves the linear solver's preconditioner open).
//
// Levels: level 0 is the mesh; each coarser level keeps every other node plane along each axis
// that has at least two elements (plus the last plane when the element count is odd), so a
// coarse interval holds one or two fine elements. Transfers are the Q1 interpolation P (exact
// for the tensor-product node coordinates) with Dirichlet rows and columns removed; coarse
// operators are Galerkin products P^T J P, stored per coarse element as an 8 x 8 matrix
// (row-major, corner index ix + 2 iy + 4 iz). Smoothing is one damped-Jacobi step before and
// after each coarse correction, weight 1/theta with theta the centre of [hi/8, hi] and hi the
// Gershgorin bound of D^-1 J on that level; the coarsest level (at most 512 nodes) is solved
// by a degree-16 Chebyshev iteration inside one thread block. Pre- and post-smoothing use the
// same polynomial, so the V-cycle is a symmetric positive definite preconditioner for CG.
#pragma once
#include <cuda_runtime.h>

#include "qcad_host.h"
#include "qcad_internal.cuh"

struct qcad_mesh_s;

namespace qcad {

constexpr int MG_MAX_LEVELS = 16;
constexpr int MG_COARSE_NODES = 512;   // the coarsest level has at most this many nodes
constexpr int MG_COARSE_DEGREE = 16;   // Chebyshev degree of the coarsest solve
constexpr float MG_ALPHA = 8.0f;       // smoothing interval [hi / MG_ALPHA, hi]

// Transfer tables along one axis, from a level to the next coarser one.
struct MgElemMap {   // per fine element: its coarse element and the 1D P[f][C], f, C in {0, 1}
  int E;
  float p00, p01, p10, p11;
};
struct MgProl {      // per fine node: the two coarse nodes it interpolates from
  int c0, c1;
  float w0, w1;
};
struct MgRestr {     // per coarse node: its coincident fine node f0 and the fine nodes on each side
  int f0, f1, f2;
  float w0, w1, w2;  // w0 = 1; an absent neighbour has weight 0 and index f0
};
struct MgChild {     // per coarse element: its first fine element and how many (1 or 2)
  int first, count;
};

// One level as the kernels see it, in the precision T of its operator and vectors (the
// transfer weights are FP32 in both precisions: the same P serves restriction and
// prolongation, so the V-cycle stays symmetric whatever their rounding).
template <class T>
struct MgLevelDev {
  int nx, ny, nz, nxn, nyn, nzn;
  const T* A;                 // 64 per element (levels >= 1)
  T* dinv;                    // 0 on Dirichlet rows (levels >= 1)
  const unsigned char* mask;  // 1 on Dirichlet nodes
  T *b, *x, *w;
  // to the next coarser level (absent on the coarsest)
  const MgElemMap* em[3];
  const MgProl* pr[3];
  const MgRestr* rs[3];
  const MgChild* ch[3];
};

// Damping weight of level l: 1 / theta, theta = (hi + hi / MG_ALPHA) / 2.
// (0 on a level whose bound is 0: every node of it is a Dirichlet node.)
template <class T>
__device__ __forceinline__ T mg_omega(const T* par, int l) {
  const T hi = par[l];
  return hi > T(0) ? T(2) / (hi * (T(1) + T(1) / T(MG_ALPHA))) : T(0);
}

// Host side (mg.cu). The hierarchy (levels, transfers, masks) is built once per mesh and serves
// both precisions; the Galerkin operators and the level vectors exist per precision T (float:
// the mixed-precision solve, double: the plain FP64 solve), allocated on first use.
bool mg_prepare(qcad_mesh_s* m);                    // builds the hierarchy once; false if unusable
// Operators and vectors of precision T (allocated once; idempotent). Must run before a V-cycle of
// that precision is enqueued or captured: the kernels take the level pointers by value.
template <class T>
void mg_reserve(qcad_mesh_s* m);
// Galerkin operators of the current linearization in precision T (nothing to do when they are
// current; force = rebuild anyway).
template <class T>
void mg_setup(qcad_mesh_s* m, cudaStream_t s, bool force = false);
void mg_invalidate(qcad_mesh_s* m);                  // the next mg_setup rebuilds (both precisions)
// PCG start: x = 0, r = b and z = V-cycle(r), ending with the phase-0 bookkeeping.
template <class T>
void mg_enqueue_init(qcad_mesh_s* m, const PcgVecs<T>& v, PcgScalars* sc, cudaStream_t s);
// One PCG iteration after its apply kernel: update of x and r, then z = V-cycle(r).
template <class T>
void mg_enqueue_update(qcad_mesh_s* m, const PcgVecs<T>& v, PcgScalars* sc, cudaStream_t s);
int mg_launches_per_iteration(qcad_mesh_s* m);      // kernels of one PCG iteration, apply included
int mg_levels(qcad_mesh_s* m);

// Level-0 V-cycle kernels on the plane-factorized z-march (kernels_lin.cu).
template <class T>
void launch_mg_resid0(const Grid<T>& g, PcgVecs<T> v, PcgScalars* sc, LaunchCfg cfg, cudaStream_t s);
template <class T>
void launch_mg_post0(const Grid<T>& g, PcgVecs<T> v, PcgScalars* sc, const T* par, LaunchCfg cfg, cudaStream_t s);

}  // namespace qcad
