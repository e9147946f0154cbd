/*
 * qcad.h - C ABI of libqcad, a GB300 (sm_103a) finite-element solver for the
 * semiclassical nonlinear Poisson equation and the effective-mass Schrodinger
 * equation of silicon quantum-dot devices, after Gao et al., "QCAD Simulation
 * and Optimization of Semiconductor Quantum Dots" (arXiv:1403.7561).
 *
 * Units everywhere: length nm, potential V, energy eV, density nm^-3,
 * temperature K, permittivity relative to eps0, effective masses in m0.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Device pointers must be CUDA device memory of the device the mesh was
 *   created on. Host pointers are ordinary host memory. The caller owns every
 *   pointer it passes; the library owns everything inside a qcad_mesh_t.
 * - All GPU work of a mesh runs on the stream given at creation. For NULL the
 *   mesh creates its own blocking stream (ordered with the legacy default
 *   stream, and capturable into CUDA graphs). Every call returns after that
 *   stream has been synchronized, because several calls return host outputs.
 * - Node index n = i + (nx+1)*(j + (ny+1)*k); element index
 *   e = i + nx*(j + ny*k) (x fastest, k counts element layers upward from z=0).
 * - On QCAD_ERR_INVALID_ARG no output is touched. On any error a message is
 *   available from qcad_last_error() (thread-local, valid until the next call
 *   on the same thread). No C++ exception crosses this boundary.
 */
#ifndef QCAD_H
#define QCAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QCAD_OK = 0,
  QCAD_ERR_INVALID_ARG = 1,   /* bad size, pointer or option; outputs untouched */
  QCAD_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  QCAD_ERR_OOM = 3,           /* device allocation failed */
  QCAD_ERR_NOT_CONVERGED = 4, /* iteration limit reached; outputs hold the last iterate */
  QCAD_ERR_NONFINITE = 5,     /* a NaN/Inf appeared; outputs undefined */
  QCAD_ERR_TIMEOUT = 6        /* a bounded device wait gave up */
} qcad_status;

/* Material parameters (Sec. II.A: eps_s, chi, E_g of Eq. EcEv_phi; the DOS
 * masses of Eq. EffectiveMass; dopants and ionization energies/degeneracies of
 * Eq. FinalIonization). A device holds at most one semiconductor material. */
typedef struct {
  double eps_r;        /* relative static permittivity */
  double chi;          /* electron affinity, eV */
  double Eg;           /* band gap, eV */
  int semiconductor;   /* 1: carries n, p and dopant charge; 0: insulator (rho = 0) */
  double m_l, m_t;     /* electron longitudinal / transverse masses, m0 */
  double m_hh, m_lh;   /* heavy / light hole masses, m0 */
  double N_A, N_D;     /* acceptor / donor concentrations, nm^-3 */
  double E_a, E_d;     /* acceptor / donor ionization energies, eV */
  double g_A, g_D;     /* ground-state degeneracies (paper: 4 and 2) */
} qcad_material;

typedef struct { double x0, x1, y0, y1; } qcad_rect;          /* closed rectangle on the top face */
typedef struct { double x0, x1, y0, y1, z0, z1; } qcad_box;   /* element-centroid box */

/* Charged gate (Sec. II.A.4, the Robin condition): gate `gate` is pinned to its
 * potential phi_0 (Eq. ContOnIns) a distance d outside the top surface, with a
 * sheet charge q sigma on the surface, so that the outward flux is
 * eps_s dphi/dn = eps_s (phi_0 - phi)/d + q sigma. Its surface is the top-plane
 * faces with all four corners in the gate's rectangle; its nodes are unknowns,
 * not Dirichlet nodes; eps_s is the permittivity of the top element layer.
 * sigma > 0 is positive charge. */
typedef struct {
  int gate;       /* index into gates */
  double sigma;   /* nm^-2 */
  double d;       /* nm, > 0 (the paper uses 10) */
} qcad_charged_gate;

/* Surface charge on an explicit surface (Sec. II.A.4, Eq. NeuBC4fc): the jump of
 * the normal displacement across the node plane at height z is q sigma over the
 * faces of that plane with all four corners in the rectangle (on an outer face,
 * an applied flux). z must be a node plane of the mesh. sigma > 0 is positive
 * charge, nm^-2. */
typedef struct { double z, x0, x1, y0, y1, sigma; } qcad_surface_charge;

/* Layered box device on a structured Q1 hexahedral mesh: uniform spacing in x
 * and y, uniform within each z layer group (bottom to top). Gates are
 * Dirichlet patches on the top face z = Lz (charged gates carry the Robin
 * condition instead, see qcad_charged_gate); the bottom face is an Ohmic
 * contact when bottom_ohmic is set; every other boundary is natural Neumann
 * (Sec. II.A.4). Dots are the semiconductor elements whose centroid lies in a
 * box (the paper's quantum region, Sec. III). The Schrodinger subdomain is the
 * element block [sub[0],sub[1]) x [sub[2],sub[3]) x [sub[4],sub[5]) with
 * psi = 0 on its boundary (Sec. II.B). All arrays are host memory, read only
 * during qcad_mesh_create. */
typedef struct {
  double Lx, Ly;
  int nx, ny;
  int n_layers;
  const int* layer_n;              /* [n_layers] element layers per group */
  const double* layer_thickness;   /* [n_layers] nm */
  const int* layer_material;       /* [n_layers] index into materials */
  int n_materials;
  const qcad_material* materials;  /* [n_materials] */
  int n_gates;
  const qcad_rect* gates;          /* [n_gates]; a node in several gates belongs to the first */
  int gate_work_function_set;      /* 0: Phi_m = q phi_ref, so phi_ins = V_g (Eq. ContOnIns) */
  double gate_work_function;       /* Phi_m in eV when gate_work_function_set */
  int bottom_ohmic;
  int n_dots;                      /* at most QCAD_MAX_DOTS */
  const qcad_box* dots;
  int has_subdomain;
  int sub[6];
  /* surface terms of the weak form (both lists may be empty). A device with either
   * runs the element-gather Jacobian kernels and Jacobi or Chebyshev-Jacobi PCG: the
   * multigrid preconditioner falls back to Jacobi, and the batched solve, the
   * self-consistent Schrodinger-Poisson loop and the allocation-free residual reject
   * it (INVALID_ARG). */
  int n_charged_gates;                       /* at most n_gates, each gate at most once */
  const qcad_charged_gate* charged_gates;
  int n_surface_charges;
  const qcad_surface_charge* surface_charges;
} qcad_device;

#define QCAD_MAX_DOTS 8
#define QCAD_MAX_GATES 32

typedef struct qcad_mesh_s* qcad_mesh_t;

/* Bias point (Sec. II.A.2, II.A.4): E_F = -q V_sub in the semiconductor; gate
 * Dirichlet values by Eq. ContOnIns; the Ohmic value by the contact formulas
 * of Sec. II.A.4 for the chosen statistics (0 MB, Eq. MBstatistics; 1 FD,
 * Eq. FDstatistics with Eq. FDIntApprox) and ionization model. */
typedef struct {
  double T;
  int n_gates;
  const double* V_gate;            /* host [n_gates], V */
  double V_sub;
  int statistics;                  /* 0 MB, 1 FD */
  int incomplete_ionization;       /* 0 complete, 1 Eq. FinalIonization */
} qcad_bias;

typedef struct {
  int precision;          /* 0: FP64 throughout; 1: mixed (FP32 Krylov operator, vectors and
                             preconditioner; FP64 residual, reductions and Newton update) */
  double newton_tol_R;    /* stop when max |R_i| over free nodes < this (V*nm) ... */
  double newton_tol_dphi; /* ... and the last max |alpha delta| < this (V) */
  int max_newton;
  int max_krylov;         /* per linear solve */
  int cheb_degree;        /* preconditioner: k >= 1 Chebyshev-Jacobi of degree k (1 = Jacobi);
                             -1 geometric multigrid V-cycle (in the solve's precision: FP32 for
                             precision 1, FP64 for precision 0); 0 = autotuned per mesh and
                             precision among Jacobi, odd Chebyshev degrees and the V-cycle */
  int warm_start;         /* 1: phi holds the initial guess; 0: Laplace solve with the contact values */
  int linear;             /* 1: rho = 0 (dielectric-only solve) */
} qcad_solver_opts;

typedef struct {
  int newton_iters;
  int krylov_iters_total;
  int applies_total;      /* operator applies issued (Krylov + preconditioner + power steps) */
  double final_res_inf;
  double final_dphi_inf;
  double seconds;         /* host wall clock of the call */
  int status_detail;
} qcad_solve_report;

/* Builds the mesh, its per-axis geometry tables, contact masks and region
 * tables on the current CUDA device (Sec. I: FE mesh with material blocks).
 * cuda_stream: cudaStream_t or NULL. On success *out owns device memory
 * until qcad_mesh_destroy. Errors: INVALID_ARG (sizes, layers, pointers),
 * OOM, CUDA. */
qcad_status qcad_mesh_create(const qcad_device* dev, void* cuda_stream, qcad_mesh_t* out);
void qcad_mesh_destroy(qcad_mesh_t m);
qcad_status qcad_mesh_info(qcad_mesh_t m, int64_t* n_nodes, int64_t* n_elems, int* n_gates,
                           int* n_dots, int64_t* n_sub_dof);

/* Contact values (Sec. II.A.4): writes the Dirichlet value of every Dirichlet
 * node into phi (device, n_nodes FP64) and leaves free nodes untouched.
 * Returns the gate (Eq. ContOnIns) and Ohmic (Eqs. PotBC4MBCompIon,
 * PotBC4MBIncompIon with Eq. Yval4MBIncompIon or Eq. ApproxLogTerms below
 * 50 K, PotBC4FDCompIon with Eq. FDintInverse) values in host arrays
 * phi_gate [n_gates] and *phi_ohmic (either may be NULL). */
qcad_status qcad_contact_values(qcad_mesh_t m, const qcad_bias* b, double* phi,
                                double* phi_gate, double* phi_ohmic);

/* Nonlinear Poisson residual (Sec. II.A.3, Eq. PoissonWeakForm, scaled by
 * 1/eps0): R_i = sum_e int eps_r grad phi.grad N_i - (q/eps0) int rho(phi) N_i
 * on free nodes, 0 on Dirichlet nodes; rho = p - n + ND+ - NA- (+ fixed charge)
 * at the 2x2x2 Gauss points. phi: device [n_nodes] (Dirichlet entries are used
 * as given). R: device [n_nodes]. diag: device [n_nodes] diagonal of the
 * Jacobian (1 on Dirichlet rows) or NULL. fixed_charge_elem: device [n_elems]
 * nm^-3 or NULL. stats: host [2] = {max |R_i|, sum R_i^2} or NULL. */
qcad_status qcad_poisson_residual(qcad_mesh_t m, const qcad_bias* b, const double* fixed_charge_elem,
                                  const double* phi, double* R, double* diag, double* stats);

/* Jacobian-vector product of the residual above (the Newton Jacobian of
 * Sec. II.C.2, differentiated by hand): y = J(phi) v on free rows with J =
 * K - (q/eps0) int rho'(phi) N_a N_b, and y_i = v_i on Dirichlet rows (v is
 * read as zero at Dirichlet nodes). precision 0: FP64 apply; 1: the FP32
 * apply used by the mixed solver (inputs and outputs still FP64 here).
 * phi, v, y: device [n_nodes]. */
qcad_status qcad_poisson_jv(qcad_mesh_t m, const qcad_bias* b, const double* phi, const double* v,
                            double* y, int precision);

/* Newton solve of the nonlinear Poisson equation (Sec. II.A; solved by a
 * Newton solver in the paper, Sec. II.A.3) with a PCG linear solver whose
 * preconditioner o->cheb_degree selects (autotuned by default: on meshes that
 * coarsen, the geometric multigrid V-cycle wins in both precisions), to the
 * tolerances in o. phi: device [n_nodes]; input guess when
 * o->warm_start, output solution (Dirichlet entries set to contact values).
 * fixed_charge_elem: device [n_elems] or NULL. rep: host or NULL.
 * Errors: NOT_CONVERGED (phi holds the last iterate, rep filled),
 * NONFINITE, INVALID_ARG, CUDA. */
qcad_status qcad_poisson_solve(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o,
                               const double* fixed_charge_elem, double* phi, qcad_solve_report* rep);

/* Integrated electron count N_d = int_dot n dOmega of every dot (Sec. III,
 * capacitance equation), 2x2x2 Gauss quadrature. phi: device; N: host [n_dots]. */
qcad_status qcad_electron_counts(qcad_mesh_t m, const qcad_bias* b, const double* fixed_charge_elem,
                                 const double* phi, double* N);

/* Dot-to-gate capacitances by the paper's finite difference (Sec. III):
 * C_d = q (N_d(V_g + dV) - N_d(V_g)) / dV for gate `gate`, in aF. Two Newton
 * solves; the second is warm-started from the first. phi: device [n_nodes]
 * scratch/output (the solution at V_g + dV on return) or NULL (library
 * scratch). C_aF: host [n_dots]. */
qcad_status qcad_capacitance(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, int gate,
                             double dV, const double* fixed_charge_elem, double* phi, double* C_aF);

/* Adjoint sensitivities of the dot electron counts at a converged phi:
 * J lambda_d = dN_d/dphi on free rows (J symmetric), then
 * dN_d/dV_g = dN_d/dphi_D . e_g - lambda_d . (J_fD e_g) and
 * dN_d/dtheta_e = (q/eps0) sum_{a in e, free} lambda_{d,a} int_e N_a.
 * q dN_d/dV_g is the capacitance of Sec. III in the limit dV -> 0.
 * phi: device [n_nodes] converged solution. dN_dV: host [n_dots * n_gates]
 * (row-major, 1/V). dN_dq: device [n_dots * n_elems] (electrons per nm^-3)
 * or NULL. o->precision selects the linear solver precision. */
qcad_status qcad_adjoint(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, const double* phi,
                         const double* fixed_charge_elem, double* dN_dV, double* dN_dq);

/* Effective-mass Schrodinger operators on the subdomain (Sec. II.B, Eq.
 * SchrodEqnWeakForm; diagonal mass tensor of Eq. Schrodinger3D; potential of
 * Eq. SchrodPotEnergy without V_xc): for the nvec columns of X (device,
 * n_sub_dof x nvec, column-major, interior subdomain nodes in node order),
 * HX = H X and MX = M X (either may be NULL). phi: device [n_nodes].
 * m_eff: host [3] (m_x, m_y, m_z) in m0. precision 0 FP64, 1 FP32 apply. */
qcad_status qcad_schrodinger_apply(qcad_mesh_t m, const qcad_bias* b, const double* phi, const double* m_eff,
                                   int nvec, const double* X, double* HX, double* MX, int precision);

/* Lowest nev eigenpairs of H psi = E M psi on the subdomain by LOBPCG with a
 * degree-5 Chebyshev-Jacobi preconditioner and FP64 Rayleigh-Ritz (the paper uses an Anasazi
 * eigensolver, Sec. II.B), started from the subdomain box's lowest sine modes; an FP32 phase,
 * then FP64 vectors with double-float H/M applies, Gram products and block updates, where
 * columns already at tol get no new search directions (soft locking; QCAD_LOBPCG_LOCK=0 turns
 * it off). phi: device [n_nodes]. evals: host [nev], eV,
 * ascending. evecs: device [n_sub_dof x nev] column-major, M-orthonormal, or
 * NULL. tol: relative residual ||H x - E M x|| / (|E| ||M x||) per pair.
 * Errors: NOT_CONVERGED (best pairs returned), INVALID_ARG (no subdomain,
 * nev < 1 or nev > 16). */
qcad_status qcad_schrodinger_eigs(qcad_mesh_t m, const qcad_bias* b, const double* phi, int nev,
                                  const double* m_eff, double tol, double* evals, double* evecs,
                                  qcad_solve_report* rep);

/* Interface-charge calibration (Sec. III: the effective interface charge Q_it is the tuning
 * parameter chosen so that the dot holds the wanted number of electrons). The fixed charge is
 * theta = sigma * pattern (pattern: device, n_elems, the per-element density of a unit sheet,
 * nm^-3 per nm^-2); sigma (nm^-2) is found by Newton on N_dot(sigma) = target_N with the adjoint
 * slope dN/dsigma = (dN/dtheta) . pattern, safeguarded by bisection inside the bracket the
 * iterates establish, each step a semiclassical Newton solve (warm-started after the first) and
 * the dot counts. Stops when |N_dot - target_N| <= tol_N; at most max_iter (<= 32) solves. phi
 * (device, n_nodes) and theta (device, n_elems) receive the last solve's potential and charge;
 * sigma (host) the last sigma. NOT_CONVERGED when tol_N is not reached. */
#define QCAD_CALIB_HIST 32
typedef struct {
  int iters;                        /* Poisson solves run */
  int converged;
  double N;                         /* dot electrons at the last solve */
  double dN_dsigma;                 /* last adjoint slope, electrons per nm^-2 */
  double seconds;
  double sigma_hist[QCAD_CALIB_HIST];
  double N_hist[QCAD_CALIB_HIST];
} qcad_calib_report;
qcad_status qcad_calibrate_sheet_charge(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, int dot,
                                        double target_N, const double* pattern, double sigma0, double tol_N,
                                        int max_iter, double* phi, double* theta, double* sigma,
                                        qcad_calib_report* rep);

/* Self-consistent Schrodinger-Poisson solve by the predictor-corrector scheme (Sec. II.C) for
 * electrons confined in three dimensions. The quantum region is the Schrodinger subdomain; there
 * the electron density of the Poisson equation is the predictor density of
 * Eq. ApproxEDens3DConfined, n~(phi) = sum_i 4 |psi_i|^2 / (1 + exp((E_i - E_F - q(phi - phi_prev))
 * / kT)) (exp(-a) for arguments a > 100), built from the nev lowest eigenpairs computed at phi_prev;
 * elsewhere it stays semiclassical. The Schrodinger potential is V = q phi_ref - chi - q phi + V_xc(n)
 * (Eq. SchrodPotEnergy) with the Hedin-Lundqvist V_xc of Eq. Vxc and the mass of Eq. mxc when
 * use_vxc != 0. Steps: (1) semiclassical Newton solve; (2) eigenpairs (LOBPCG, relative residual
 * eig_tol of the spectrum shifted so that the potential's minimum sits at 0.1 eV); (3) Newton solve
 * with n~, warm-started at the previous potential, then n~ and V_xc at the new potential; (4) stop
 * when k >= 2 and max |phi^(k) - phi^(k-1)| < tol_dphi (V), else repeat, at most max_iter times.
 * tol_dphi <= 0 runs exactly max_iter iterations. phi: device, n_nodes, output. evals: host, nev
 * (eV, from the last step (2)). nev must include every occupied level. NOT_CONVERGED when the
 * tolerance is not reached; the report holds the per-iteration history. The mesh's residual uses the
 * quantum density only inside this call. */
#define QCAD_SP_HIST 64
typedef struct {
  int sp_iters;                  /* outer iterations run */
  int converged;
  double dphi_inf;               /* max |phi^(k) - phi^(k-1)| of the last iteration, V */
  double n_quantum;              /* electrons in the quantum region (integral of n~ at the final phi) */
  double seconds;                /* host wall clock of the call */
  double dphi_hist[QCAD_SP_HIST];  /* max |phi^(k) - phi^(k-1)| per iteration */
  double e1_hist[QCAD_SP_HIST];    /* lowest eigenvalue per iteration, eV */
} qcad_sp_report;
qcad_status qcad_sp_solve(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, int nev,
                          const double* m_eff, double eig_tol, double tol_dphi, int max_iter, int use_vxc,
                          double* phi, double* evals, qcad_sp_report* rep);

/* The adjoint capacitance (as qcad_adjoint) and the Schrodinger eigenpairs (as
 * qcad_schrodinger_eigs) at one converged potential phi, computed concurrently:
 * the eigensolve runs on a second stream of the mesh from a second host thread
 * while the adjoint runs on the mesh stream (the paper computes the two one
 * after the other; they share only read-only data). Arguments as in the two
 * calls; eig_rep is the eigensolve's report (may be NULL). Returns the
 * adjoint's status if it is not OK, else the eigensolve's. */
qcad_status qcad_adjoint_eigs(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, const double* phi,
                              const double* fixed_charge_elem, double* dN_dV, double* dN_dq, int nev,
                              const double* m_eff, double tol, double* evals, double* evecs,
                              qcad_solve_report* eig_rep);

/* Batched form (no counterpart in the paper, which solves one device at a
 * time; the operator of every instance is the one of qcad_poisson_solve):
 * n independent meshes of any sizes, each with its own bias, solved by a
 * lockstep Newton iteration: one residual launch for all instances (a work
 * table maps blocks to (instance, tile)), and the linear solves either as
 * FP32 Jacobi-PCG iterations advancing all unconverged instances with one
 * apply launch and one update launch (o->cheb_degree 1; chunks of 8 iterations
 * replayed from a captured CUDA graph), or (o->cheb_degree 0 or -1, every mesh
 * large enough for a coarse level) as each instance's multigrid-preconditioned
 * PCG, its captured 4-iteration graph replayed together with the others' on a
 * pool of streams (instances run side by side) and one status read per round. Instances drop out on their own
 * device-resident convergence flags. ms, bs, phis: host arrays of n entries
 * (phis[i] device [n_nodes of ms[i]], FP64, also the warm start). reps: host
 * [n] or NULL. o->precision must be 1 (mixed). All meshes must be distinct and
 * on one device; the call uses the stream of ms[0] and synchronizes the
 * others. Returns the first non-OK instance status (NOT_CONVERGED or
 * NONFINITE; the per-instance reports say which); INVALID_ARG otherwise. */
qcad_status qcad_poisson_solve_batch(int n, const qcad_mesh_t* ms, const qcad_bias* bs,
                                     const qcad_solver_opts* o, double* const* phis, qcad_solve_report* reps);

/* Batched adjoint sensitivities (Sec. III's capacitance C = q dN/dV by the adjoint) of several
 * meshes at once, e.g. the bias points of a gate sweep solved by qcad_poisson_solve_batch: for
 * every mesh i and dot d, J_i lam = dN_d/dphi on the free rows, with all (mesh, dot) systems in
 * one batched FP32 Jacobi-PCG (one apply launch and one update launch per iteration over a work
 * table of the systems, iteration chunks replayed from a captured CUDA graph), each round
 * followed by every system's FP64 residual, until each is below 1e-13 of its right-hand side;
 * then dN_d/dV_g as qcad_adjoint forms it. ms, bs, phis: host arrays of n entries (phis[i]:
 * device [n_nodes of ms[i]], a converged potential at bs[i]). dN_dV: host, the meshes' blocks
 * one after the other, block i = n_dots(i) x n_gates(i) row-major (1/V). o->precision must be
 * 1; no fixed charge; meshes distinct, on one device, without charged gates or surface charges.
 * Uses the stream of ms[0]. */
qcad_status qcad_adjoint_batch(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                               const double* const* phis, double* dN_dV);

/* Kernel timing: with profiling enabled, every launch of the timed kernel
 * classes on the mesh stream (including those inside captured CUDA graphs) is
 * bracketed by CUDA events and its duration accumulated. Classes: 0 FP32
 * Jacobian apply (PCG), 1 FP64 Jacobian apply (PCG), 2 FP32 PCG update,
 * 3 FP64 PCG update, 4 FP64 residual, 5 Schrodinger H/M apply, 6 multigrid
 * PCG iteration tail (update and V-cycle, timed as one span).
 * qcad_profile_read returns the launch count and total milliseconds of one
 * class; qcad_profile_reset clears the counters. Profiling is off by default. */
qcad_status qcad_profile_enable(qcad_mesh_t m, int enable);
qcad_status qcad_profile_reset(qcad_mesh_t m);
qcad_status qcad_profile_read(qcad_mesh_t m, int kernel_class, int64_t* launches, double* total_ms);

/* Launch configuration of the z-marching kernels, per kernel family: 0 FP64
 * residual, 1 FP64 linear operators (Jacobian apply, PCG apply, Chebyshev
 * step), 2 FP32 linear operators. tile_rows: warps per block, 4, 8, 16 or 32;
 * z_chunk: node planes per block, 1..4096. variant (families 1 and 2; ignored
 * for 0): 0 element-gather kernel, 1 element-gather with two nodes per thread
 * and packed f32x2 arithmetic (FP32 only; FP64 runs variant 0), 2
 * plane-factorized kernel with one node row per thread, 3 plane-factorized
 * with two node rows per thread. Shapes a variant does not support are
 * clamped to the nearest supported one (FP64 plane-factorized: at most 8
 * warps). Defaults: variant 3, 8 warps, z chunk 16.
 * qcad_autotune times the Jacobian apply of the given precision (0 FP64,
 * 1 FP32) over variants, tile rows and z chunks on the mesh, keeps the
 * fastest for that family and returns it (outputs may be NULL); best_ms is
 * its time per apply. */
qcad_status qcad_set_launch(qcad_mesh_t m, int family, int variant, int tile_rows, int z_chunk);
/* The current launch shape of a family (as qcad_set_launch) and, for families 1 (FP64) and
 * 2 (FP32), the preconditioner the mesh's autotuner chose, coded as cheb_degree in
 * qcad_solver_opts (0: not tuned yet). Outputs may be NULL. */
qcad_status qcad_launch_info(qcad_mesh_t m, int family, int* variant, int* tile_rows, int* z_chunk,
                             int* cheb_degree);
qcad_status qcad_autotune(qcad_mesh_t m, const qcad_bias* b, int precision, int* variant, int* tile_rows,
                          int* z_chunk, float* best_ms);

/* Allocation-free residual, for callers that cannot allocate device memory
 * (code inside another framework's allocator or memory pool, or in a loop
 * where cudaMalloc/cudaFree are not allowed). The paper has no counterpart;
 * this is a packaging of the residual above. Computes the same R (and stats)
 * as qcad_poisson_residual, but from the device description directly: no mesh
 * object, no cudaMalloc/cudaFree, no host heap on success. The description is
 * checked as qcad_mesh_create checks it (sizes, layers, one semiconductor
 * material, permittivities > 0, the 32-bit index limits); charged gates and
 * surface charges are rejected. Its scratch (geometry tables, contact masks,
 * reduction accumulators) is one static device array of 2 MiB that every GPU
 * loading this library holds until process exit; meshes whose tables do not
 * fit (roughly (nx+1)*(ny+1) + 60*(nx+ny+nz) bytes) are rejected with
 * QCAD_ERR_INVALID_ARG before the device is touched. All calls share that
 * array and leave the last call's contents in it; the accumulators are
 * cleared at the start of every call. Calls whose GPU work overlaps (on
 * different streams or host threads) race on the array. The first call on a
 * device looks up the array's device address with that device current.
 * dev, b: host; cuda_stream: cudaStream_t or NULL (legacy default stream);
 * fixed_charge_elem (device [n_elems] or NULL), phi, R: device; stats: host
 * [2] {max |R_i|, sum R_i^2} or NULL. Returns after the stream has been
 * synchronized. */
qcad_status qcad_poisson_residual_noalloc(const qcad_device* dev, const qcad_bias* b, void* cuda_stream,
                                          const double* fixed_charge_elem, const double* phi, double* R,
                                          double* stats);

/* Arithmetic peaks of the current CUDA device, measured by microbenchmarks (no
 * counterpart in the paper): the denominators of the roofline of a kernel bound
 * by arithmetic rather than memory, such as the FP64 Newton residual, whose
 * carrier statistics (Sec. II.A.1-3) evaluate FP64 exponentials at every Gauss
 * point. fp64_tflops and fp32_tflops: fused multiply-add throughput in TFLOP/s
 * (2 flops per FMA); fp64_exp_per_s: FP64 exp() evaluations per second. Each
 * kernel runs eight independent dependency chains per thread on 8 blocks of
 * 256 threads per SM, once untimed and then three times timed with CUDA events
 * on a private stream; the best run is reported (about 0.15 s in all). Host
 * outputs, each may be NULL. Errors: CUDA. */
qcad_status qcad_alu_peaks(double* fp64_tflops, double* fp32_tflops, double* fp64_exp_per_s);

/* Number of CUDA kernels this library has launched in the process (kernels
 * inside replayed CUDA graphs included). Host output *count. */
qcad_status qcad_launch_count(int64_t* count);

const char* qcad_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QCAD_H */
