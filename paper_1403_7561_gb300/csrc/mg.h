// Geometric multigrid V-cycle preconditioner for the FP32 Jacobian J = K + M_c of the
// mixed-precision Newton-Krylov solve (a preconditioner choice: the paper leaves the linear
// solver's preconditioner open).
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

// One level as the kernels see it.
struct MgLevelDev {
  int nx, ny, nz, nxn, nyn, nzn;
  const float* A;             // 64 per element (levels >= 1)
  float* dinv;                // 0 on Dirichlet rows (levels >= 1)
  const unsigned char* mask;  // 1 on Dirichlet nodes
  float *b, *x, *w;
  // to the next coarser level (absent on the coarsest)
  const MgElemMap* em[3];
  const MgProl* pr[3];
  const MgRestr* rs[3];
  const MgChild* ch[3];
};

// Damping weight of level l: 1 / theta, theta = (hi + hi / MG_ALPHA) / 2.
// (0 on a level whose bound is 0: every node of it is a Dirichlet node.)
__device__ __forceinline__ float mg_omega(const float* par, int l) {
  const float hi = par[l];
  return hi > 0.0f ? 2.0f / (hi * (1.0f + 1.0f / MG_ALPHA)) : 0.0f;
}

// Host side (mg.cu).
bool mg_prepare(qcad_mesh_s* m);                    // builds the hierarchy once; false if unusable
// Galerkin operators of the current FP32 linearization (nothing to do when they are current;
// force = rebuild anyway).
void mg_setup(qcad_mesh_s* m, cudaStream_t s, bool force = false);
void mg_invalidate(qcad_mesh_s* m);                  // the next mg_setup rebuilds
// PCG start: x = 0, r = b and z = V-cycle(r), ending with the phase-0 bookkeeping.
void mg_enqueue_init(qcad_mesh_s* m, const PcgVecs<float>& v, PcgScalars* sc, cudaStream_t s);
// One PCG iteration after its apply kernel: update of x and r, then z = V-cycle(r).
void mg_enqueue_update(qcad_mesh_s* m, const PcgVecs<float>& v, PcgScalars* sc, cudaStream_t s);
int mg_launches_per_iteration(qcad_mesh_s* m);      // kernels of one PCG iteration, apply included
int mg_levels(qcad_mesh_s* m);

// Level-0 V-cycle kernels on the plane-factorized z-march (kernels_lin.cu).
void launch_mg_resid0(const Grid<float>& g, PcgVecs<float> v, PcgScalars* sc, LaunchCfg cfg, cudaStream_t s);
void launch_mg_post0(const Grid<float>& g, PcgVecs<float> v, PcgScalars* sc, const float* par, LaunchCfg cfg,
                     cudaStream_t s);

}  // namespace qcad
