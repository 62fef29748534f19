/*
 * richards.h - C ABI of the GB300 backward-Euler Richards solver.
 *
 * The library advances the mixed-form Richards equation
 *     rho*phi ds(p)/dt - div(K(p) grad p) - dK(p)/dz = 0
 * (Sec. 2 of Bertaccini, D'Ambra, Durastante, Filippone, "Why
 * diffusion-based preconditioning of Richards equation works", arXiv
 * 2112.05051) by fully implicit backward-Euler steps on a cell-centred
 * 7-point grid (eq. (dynamic_of_the_problem), Sec. 2.1).  Each step runs an
 * inexact Newton iteration with an Armijo line search (Sec. 3) whose
 * corrections J d = -Phi are solved by flexible CG or flexible GMRES,
 * right-preconditioned (eq. (precsystem)) by a smoothed-aggregation AMG
 * V-cycle (eq. (Vcycle), Sec. 5.2) built on the diffusion-only matrix of
 * Sec. 4 (the Jacobian with the gravity and dK/dp terms dropped).
 *
 * Conventions shared by every call
 *   - Cell (i,j,k), 0-based, is unknown c = i + nx*(j + ny*k); z (k) points up.
 *     The grid has nx*ny*nz unknown cells; spacing h_d = l_d/(n_d + 1): the
 *     paper's N = n + 2 nodes per direction with the outermost on the boundary.
 *   - Faces are numbered -x, +x, -y, +y, -z (bottom), +z (top).
 *   - Every pointer named *_dev is a device pointer on the context's device;
 *     it is borrowed for the duration of the call and never freed by the
 *     library.  Pointers named *_host are host memory.
 *   - Work is enqueued on the CUDA stream given to rich_create.  Calls that
 *     return scalars or statistics synchronise that stream before returning.
 *   - Every call returns RICH_OK (0) or a negative error code; rich_strerror
 *     gives its text.  On error no output is guaranteed except as stated.
 *   - Stencil arrays ("7n") hold 7 blocks of n doubles: the diagonal, then the
 *     coefficients of the -x, +x, -y, +y, -z, +z neighbours (0 where the
 *     neighbour lies outside the grid).
 */
#ifndef RICHARDS_GB300_H
#define RICHARDS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RICH_OK                0
#define RICH_EINVAL           -1  /* bad size, null pointer, non-positive dt, bad option */
#define RICH_ENOMEM           -2  /* device allocation failed */
#define RICH_ECUDA            -3  /* a CUDA call failed (see rich_last_cuda_error) */
#define RICH_ENOTCONV_LIN     -4  /* Krylov solve reached maxit without meeting eta */
#define RICH_ENOTCONV_NEWTON  -5  /* Newton reached max_newton without meeting rtol */
#define RICH_ELINESEARCH      -6  /* line search step fell below lambda_min or no descent */
#define RICH_ENONFINITE       -7  /* NaN or Inf in a residual or Krylov scalar */
#define RICH_ESTATE           -8  /* call made before its prerequisite (e.g. no Jacobian yet) */
#define RICH_ELIMIT           -9  /* a size limit of the implementation was exceeded */
#define RICH_EBUSY           -10  /* request server: the request has not finished yet */

#define RICH_AGG_MIS2          0
#define RICH_AGG_MATCHING      1

/* V-cycle smoother (Sec. 5.2).  L1JACOBI: x <- x + D_l1^-1 (b - A x), D_l1 the row
 * l1 norms.  HYBRID_GS: the paper's hybrid backward/forward Gauss-Seidel (Sec. 6:
 * backward sweeps before, forward sweeps after the coarse correction) -- Gauss-Seidel
 * inside the block of unknowns one GPU thread (or lane group) owns, Jacobi between
 * blocks, scaled by a_ii + sum of |a_ij| over couplings to other blocks (the l1 form,
 * convergent for any blocks); blocks are vertical column segments on the finest grid
 * and runs of consecutive rows on coarser levels. */
#define RICH_SMOOTH_L1JACOBI   0
#define RICH_SMOOTH_HYBRID_GS  1

/* Preconditioner of the Krylov solves.  AMG: the V-cycle above.  AS: the paper's
 * one-level additive Schwarz preconditioner (Sec. 5.2, eq. (AS); Sec. 6 overlaps the
 * subdomains by one layer and applies ILU(0) to each), M^-1 = sum_t R_t^T M_t^-1 R_t
 * over subdomains that are boxes of as_block cells per side grown by as_overlap
 * layers; M_t is the principal submatrix of the diffusion matrix A_aux and M_t^-1
 * its ILU(0) solve in the box's lexicographic order (for the 7-point matrix:
 * L = I + L_A D^-1, U = D + U_A, D_c = m_cc - sum over lower neighbours of
 * m_ck^2 / D_k); the contributions covering a cell are summed in a fixed order. */
#define RICH_PRECOND_AMG       0
#define RICH_PRECOND_AS        1

/* Storage of the coarse-level matrices for the V-cycle's row operations */
#define RICH_LAYOUT_AUTO       0
#define RICH_LAYOUT_CSR        1
#define RICH_LAYOUT_SELL       2   /* SELL kernel: four gathers in flight per row */
#define RICH_LAYOUT_SELL8      3   /* eight gathers in flight per row */
#define RICH_LAYOUT_SELL2      4   /* two lanes per row */
#define RICH_LAYOUT_SELLP      5   /* slot loads of the next four columns in flight during the gathers */

/* ---- enumerations ------------------------------------------------------- */
/* Face conductivity K_av (Sec. 2.1): arithmetic (K_L+K_U)/2; upstream
 * (eq. (upstream_mean)) K_U if p_U - p_L >= 0 else K_L with U the +d cell;
 * harmonic 2 K_L K_U / (K_L + K_U); geometric sqrt(K_L K_U). */
#define RICH_KMEAN_ARITH      0
#define RICH_KMEAN_UPSTREAM   1
#define RICH_KMEAN_HARMONIC   2
#define RICH_KMEAN_GEOMETRIC  3
/* Sec. 2.1 also allows two different means, one for the horizontal and one for
 * the vertical direction: RICH_KMEAN_SPLIT(h, v) applies mean h on the x and y
 * faces and mean v on the z faces (h, v among the four above).  Every entry point
 * that takes a kmean accepts these codes. */
#define RICH_KMEAN_SPLIT_FLAG 0x100
#define RICH_KMEAN_SPLIT(h, v) (RICH_KMEAN_SPLIT_FLAG | ((h) << 4) | (v))

#define RICH_BC_NOFLUX     0  /* the whole face flux (diffusion + gravity) is zero */
#define RICH_BC_DIRICHLET  1  /* ghost node at p = value, K from the adjacent cell's K_s */
#define RICH_BC_INTERFACE  2  /* the face between two subdomains of a split grid (Sec. 5.1): the ghost is
                                 the neighbouring subdomain's cell, its pressure per cell in
                                 value_field_dev[f] (required; refreshed by rich_set_face_values) and its
                                 K_s in ghost_ks_dev[f] (NULL: the soil's ks_const).  The residual and the
                                 Jacobian rows of the face cells are those of the unsplit grid: J and
                                 A_aux keep the coupling to the ghost in their plane of face f */

/* Precision of the AMG preconditioner.  The Newton residual, the Jacobian,
 * line-search norms and the outer Krylov vectors and dot products are FP64
 * in both modes; MIXED stores and applies the hierarchy (matrices,
 * transfer operators, l1 diagonals, coarsest inverse, V-cycle vectors) in
 * FP32 with FP32 accumulation. */
#define RICH_PREC_FP64   0
#define RICH_PREC_MIXED  1

#define RICH_KRYLOV_FCG     0  /* Notay's flexible CG, truncation 1 */
#define RICH_KRYLOV_FGMRES  1  /* Saad's flexible GMRES(m), CGS2, Givens */

/* AMG reuse across Newton iterations.
 *  REFRESH      aggregates, P and R from the first setup of the run are kept;
 *               each new diffusion matrix refreshes every coarse matrix
 *               A_{l+1} = R A_l P numerically (same sparsity patterns).
 *  SETUP_ONCE   the paper's scheme (Sec. 6): the hierarchy of the first
 *               Jacobian is kept and only the finest matrix and its smoother
 *               are replaced.
 *  REBUILD_STEP a full setup at the first Newton iteration of each step,
 *               REFRESH at the following ones. */
#define RICH_AMG_REFRESH       0
#define RICH_AMG_SETUP_ONCE    1
#define RICH_AMG_REBUILD_STEP  2

/* ---- parameter structs -------------------------------------------------- */
typedef struct {
  int nx, ny, nz;          /* unknown cells per direction, each >= 1 */
  double lx, ly, lz;       /* box size (cm) */
  double h[3];             /* cell spacing per axis (cm); 0 (the usual): l / (n + 1).  A block of a split
                              grid gives its whole grid's spacing here, which l / (n + 1) of its own box
                              cannot always reproduce to the last bit */
} rich_grid;

/* Celia/Haverkamp laws, eqs. (s(p)) and (K(p)) of Sec. 2:
 *   s(p) = alpha (theta_s - theta_r)/(alpha + |p|^beta) + theta_r,
 *   K(p) = K_s a / (a + |p|^gamma)            for p < 0;
 *   s = theta_s, K = K_s, s' = K' = 0        for p >= 0 (saturated). */
typedef struct {
  double alpha, beta, theta_s, theta_r, a, gamma;
  double ks_const;         /* K_s when ks_field_dev is NULL */
  double rho_phi;          /* factor of the storage term (1 in the paper's 1D forms) */
  const double* ks_field_dev; /* per-cell K_s (n doubles, device) or NULL; copied at create */
} rich_soil;

typedef struct {
  int kind[6];             /* RICH_BC_* per face */
  double value[6];         /* Dirichlet pressure head (cm) per face */
  /* Optional per-cell Dirichlet values (device, NULL = the constant value[f]),
   * one per boundary cell of the face, indexed i + nx*j on the z faces,
   * i + nx*k on the y faces and j + ny*k on the x faces.  rich_create copies
   * them; rich_residual_noalloc reads them in place.  Used for the paper's
   * infiltration problem (Sec. 6): p = 0 on a centred square of the top face,
   * h_r elsewhere. */
  const double* value_field_dev[6];
  /* RICH_BC_INTERFACE faces: per-cell K_s of the ghost cells (device, same indexing), or
   * NULL for the soil's ks_const; copied at create.  Ignored on other faces. */
  const double* ghost_ks_dev[6];
} rich_bc;

typedef struct {
  double theta;            /* strength threshold (0.08): a_ij^2 >= theta_l^2 |a_ii a_jj|, theta_l = theta 2^-l */
  uint64_t seed;           /* MIS-2 priority seed: key(i) = top30(splitmix64(seed^i))<<32 | i */
  int coarse_max;          /* stop coarsening below this many unknowns (2000) */
  int max_levels;          /* at most this many levels (10) */
  int nu1, nu2;            /* l1-Jacobi pre/post sweeps (1, 1) */
  int smooth_levels;       /* levels 0..smooth_levels-1 smooth P; deeper ones use P = P_tent (10 = all) */
  int product_lists;       /* 1 (default): the first Galerkin refresh records, per entry of A P and of
                              R (A P), the list of (A entry, B entry) pairs summed into it, and every
                              refresh sums those lists (about 8 bytes per scalar product of device
                              memory; used only while it fits in half the free device memory).
                              0: every refresh searches
                              each product's output position instead (no extra memory). */
  int aggregation;         /* RICH_AGG_MIS2 (default): strength graph + MIS-2 roots.  RICH_AGG_MATCHING:
                              the paper's SMATCH-style coupled aggregation (Sec. 5.2): compatible weights
                              w_ij = 1 - (a_ij + a_ji)/(a_ii + a_jj) of the negative couplings (FP32),
                              locally dominant matching, log2(max_agg_size) pairing passes on the
                              successive pair graphs */
  int max_agg_size;        /* largest aggregate of the matching (8, as in the paper's runs) */
  int smoother;            /* RICH_SMOOTH_L1JACOBI (default) or RICH_SMOOTH_HYBRID_GS */
  int hgs_seg;             /* hybrid Gauss-Seidel blocks on the finest grid: segments of this many cells of
                              one vertical column (16) */
  int hgs_block;           /* hybrid Gauss-Seidel blocks on coarser levels: this many consecutive rows (16) */
  int precond;             /* RICH_PRECOND_AMG (default) or RICH_PRECOND_AS */
  int as_block;            /* AS subdomain box: cells per side (8) */
  int as_overlap;          /* AS overlap in layers (1, as in the paper's runs); as_block + 2 as_overlap <= 24 */
  int autotune;            /* 1 (default): the first time a CSR row operation of the V-cycle (sweep,
                              residual, restriction, prolongation) meets a shape class (rows in
                              quarter-octave bins, mean row length), every lane-group width (1..32 lanes
                              per row, and 1..8 with four-way unrolled rows) is timed on it and the
                              fastest is kept for the process
                              (rich_autotune_table lists the choices); 0: a fixed rule by the mean row
                              length */
  int isolated_join;       /* MIS-2 pass 3 (1, default): a node without strong neighbours whose row is not
                              diagonally dominant (a_ii < 2 sum_{j!=i} |a_ij|) joins the aggregate of its
                              aggregated neighbour j with the largest (fp32 |a_ij|, key(j)); dominant rows
                              (e.g. under a Dirichlet face) stay out.  0: every such node stays out */
  int csr_layout;          /* the V-cycle's sparse row operations below the finest level (sweep, residual,
                              restriction, prolongation).  RICH_LAYOUT_AUTO (default): a coarse A, P or R
                              with >= 2048 rows may get a SELL-C-sigma copy (slices of 32 rows sorted by
                              length within windows of 1024 rows, one thread per row): the autotuner
                              times it beside the CSR variants when it first meets the matrix's shape
                              class, and keeps it only if it wins; a matrix whose class chose it gets
                              its copy on first use.  RICH_LAYOUT_CSR: CSR only, no copy.
                              RICH_LAYOUT_SELL / _SELL8 / _SELL2 / _SELLP: the SELL copy for every such
                              matrix, with that SELL kernel (no timing) */
  int graph;               /* 1 (default): with the l1-Jacobi AMG preconditioner, the V-cycle's second
                              application is captured as one CUDA graph (on a stream of its own) and the
                              later ones replay it, and so are FCG's iterations from the second on (one
                              graph per parity of the iteration, while the solve writes the same x): the
                              same kernels on the same buffers, so the same results, with fewer launch
                              gaps; a hierarchy whose capture fails, and any application while a kernel
                              is being profiled, launches directly.  0: direct launches always */
} rich_amg_opts;

typedef struct {
  int kind;                /* RICH_KRYLOV_* */
  int restart;             /* m of FGMRES(m), <= 63 */
  double eta;              /* stop when ||b - J x||_2 <= eta ||b||_2 */
  int maxit;               /* iteration limit */
  double stall;            /* give up (RICH_ENOTCONV_LIN) after an FGMRES restart cycle, or a window of 30
                              FCG iterations, that reduced ||b - J x||_2 by less than this fraction of
                              its value at the cycle's (window's) start; 0 (default): off.  In [0, 1) */
} rich_krylov_opts;

typedef struct {
  int iterations;          /* Krylov iterations done */
  int converged;           /* 1 if eta was met */
  double res0, res;        /* ||b||_2 and the final ||b - J x||_2 */
} rich_krylov_stats;

typedef struct {
  rich_krylov_opts krylov;
  rich_amg_opts amg;
  int amg_policy;          /* RICH_AMG_* */
  double rtol, atol;       /* converged when ||Phi||_2 <= max(rtol ||Phi_0||_2, atol, eps ||m||_2),
                              m_c = sum of the magnitudes of the products summed into Phi_c
                              (the accuracy to which Phi can be evaluated) */
  int max_newton;          /* Newton iteration limit (50) */
  double armijo_c;         /* sufficient-decrease constant (1e-4) */
  double lambda_min;       /* smallest line-search step (1e-10) */
  int fcg_fallback_restart;/* FGMRES(m) retry after an FCG failure (30) */
  int max_dt_halvings;     /* time-step control (0 = off, default).  H > 0: rich_step covers dt with
                              backward-Euler steps of length dt / 2^k: an attempt that fails with
                              RICH_ENOTCONV_NEWTON, RICH_ELINESEARCH or, when FCG met (p, J p) <= 0,
                              RICH_ENOTCONV_LIN is discarded (p restored) and retried with half its
                              length, down to dt / 2^H (a Krylov solve that only ran out of iterations
                              ends the step: a shorter step does not mend the preconditioner); after an
                              accepted substep the length doubles back whenever the time reached is a
                              multiple of the doubled length, so the substeps end exactly at dt.  Under
                              control an FCG solve that meets (p, J p) <= 0 fails the attempt at once
                              instead of falling back to FGMRES.  The paper fixes dt per step (Sec. 6);
                              this is host-side control for steep wetting fronts */
} rich_newton_opts;

typedef struct {
  int newton_its;          /* Newton corrections applied */
  int linear_its;          /* Krylov iterations over all corrections (incl. fallbacks) */
  int line_search_evals;   /* residual evaluations inside line searches */
  int fallbacks;           /* FCG solves retried with FGMRES */
  int amg_setups;          /* full hierarchy builds during the step */
  int amg_refreshes;       /* numeric refreshes / fine-level updates during the step */
  int converged;           /* 1 if rtol/atol was met */
  double res0, res;        /* ||Phi||_2 at the start and at the end of the step */
  double min_lambda;       /* smallest accepted step length */
  /* device time per phase (ms), the phases of the paper's time breakdown
   * (Sec. 6): residual evaluations (Feval), Jacobian + diffusion-matrix
   * assembly (Jacobian/Auxiliary), AMG setup or refresh (Setup), Krylov
   * solves (LinSol); the rest of the step is Overhead (no Halo on one GPU). */
  double ms_feval, ms_jacobian, ms_setup, ms_linsol, ms_total;
  int substeps;            /* backward-Euler steps that covered dt (1 without time-step control) */
  int dt_failures;         /* attempts discarded and retried with half the step */
  double dt_min;           /* shortest accepted substep */
} rich_step_stats;

typedef struct {
  int levels;              /* number of levels incl. the finest */
  int n[16];               /* unknowns per level */
  long long nnz[16];       /* nonzeros of A per level */
  int mis_rounds[16];      /* MIS-2 rounds used to coarsen level l */
  double omega[16];        /* prolongator damping 4/(3 rho) of level l */
  double operator_complexity; /* sum nnz(A_l) / nnz(A_0) */
} rich_amg_info;               /* all zero with the AS preconditioner (one level, no hierarchy) */

typedef struct rich_ctx rich_ctx;

/* ---- lifetime ---------------------------------------------------------- */
/* Create a context on the current device.  stream is a cudaStream_t (NULL =
 * legacy default stream).  Copies the K_s field.  Allocates the per-grid
 * buffers (constitutive values, Jacobian and diffusion stencils, CSR pattern
 * of the finest AMG level, Krylov work vectors are allocated lazily). */
int rich_create(const rich_grid* grid, const rich_soil* soil, int kmean, const rich_bc* bc,
                int precision, void* stream, rich_ctx** out);
int rich_destroy(rich_ctx* ctx);
const char* rich_strerror(int status);
const char* rich_last_cuda_error(void);
int rich_num_cells(const rich_ctx* ctx, long long* n_out);

/* ---- Sec. 5.1: the split grid (x-y blocks with whole columns, a one-cell
 * halo exchanged before each residual, Jacobian and SpMV, dot products summed
 * over the blocks) ------------------------------------------------------- */
/* Replaces the per-cell values of face f (Dirichlet pressures, or the ghost
 * pressures of a RICH_BC_INTERFACE face after a halo exchange) with values_dev
 * (device, the face's cell count, indexing of rich_bc.value_field_dev), copied on
 * the context's stream.  RICH_ESTATE if the face was created without a per-cell
 * field, RICH_EINVAL on a bad face or pointer. */
int rich_set_face_values(rich_ctx* ctx, int face, const double* values_dev);
/* out_dev[t] = field_dev[the cell next to face f with face index t]: packs the cells
 * a neighbouring subdomain needs as its ghosts (the send side of a halo exchange),
 * in the layout of the per-cell face arrays.  Device pointers; the context's
 * stream; out_dev holds the face's cell count. */
int rich_pack_face(rich_ctx* ctx, int face, const double* field_dev, double* out_dev);
/* y_dev[c] += M[c, ghost t] ghost_dev[t] over the cells c next to interface face f:
 * the coupling to the neighbouring subdomain's cells that the context's current J
 * (which = 0) or A_aux (which = 1) keeps in the plane of face f.  After
 * rich_jacobian_apply on the subdomain's own cells, one call per interface face
 * with the neighbour's x (a halo exchange of x) gives the split grid's J x.
 * RICH_EINVAL unless face is an interface face; RICH_ESTATE before rich_jacobian. */
int rich_face_apply(rich_ctx* ctx, int face, int which, const double* ghost_dev, double* y_dev);
/* Vector operations on the context's cells, for drivers above the library (the
 * split grid's Krylov method): *out_host = x . y (device vectors of n doubles,
 * the library's fixed-order reduction; synchronises), and y = a x + b y (y = a x
 * when b == 0).  On the context's stream. */
int rich_vec_dot(rich_ctx* ctx, const double* x_dev, const double* y_dev, double* out_host);
int rich_vec_axpby(rich_ctx* ctx, double a, const double* x_dev, double b, double* y_dev);

/* ---- Sec. 2: constitutive law and residual ----------------------------- */
/* s_dev[c] = s(p_dev[c]) (eq. (s(p))).  Used for s(p^{l-1}) of a step. */
int rich_saturation(rich_ctx* ctx, const double* p_dev, double* s_dev);

/* Phi(p) of eq. (dynamic_of_the_problem) with s(p^{l-1}) = s_old_dev and time
 * step dt > 0, written to F_dev (n doubles).  If norms_host is not NULL it
 * receives {||Phi||_2, ||Phi||_inf} (and the call synchronises); a
 * non-finite Phi returns RICH_ENONFINITE after writing F_dev. */
int rich_residual(rich_ctx* ctx, const double* p_dev, const double* s_old_dev, double dt,
                  double* F_dev, double* norms_host);
/* rich_residual with the scale of Phi's rounding error beside the norms:
 * norms3_host (3 doubles, required) receives {||Phi||_2, ||Phi||_inf, ||m||_2},
 * m_c the sum of the magnitudes of the products added into Phi_c before they
 * cancel (storage terms |s|/dt, face terms K_av (|p_c| + |p_nb|)/h^2 and the
 * gravity terms), so that eps ||m||_2 is the accuracy to which Phi can be
 * evaluated: the round-off floor of the Newton convergence test (Sec. 3) that
 * rich_step applies.  On the split grid the blocks' ||m||_2^2 add up to the
 * whole grid's.  Synchronises; RICH_ENONFINITE as rich_residual. */
int rich_residual3(rich_ctx* ctx, const double* p_dev, const double* s_old_dev, double dt,
                   double* F_dev, double* norms3_host);

/* The residual of rich_residual without a context and without any device
 * allocation.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory where they need a residual (a fixed,
 * pre-reserved memory budget, an allocator that owns all device memory, or a
 * loop that must not risk the synchronisation a cudaMalloc can cause).
 * Inputs as for rich_create/rich_residual (soil->ks_field_dev is read in place,
 * not copied); F_dev receives Phi; norms_host, if not NULL, receives
 * {||Phi||_2, ||Phi||_inf} and the call then synchronises the stream.
 * The only scratch is a file-scope device array of about 1 MB shared by all
 * calls; grids above 134,217,728 cells (512^3) return RICH_ELIMIT.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress),
 * so make that first call before any stream capture.  Calls that overlap on the
 * GPU race on the shared array and must be serialised by the caller. */
int rich_residual_noalloc(const rich_grid* grid, const rich_soil* soil, int kmean, const rich_bc* bc,
                          const double* p_dev, const double* s_old_dev, double dt, double* F_dev,
                          double* norms_host, void* stream);

/* ---- Sec. 3-4: Jacobian and diffusion-only preconditioner matrix ------- */
/* Assemble J(p) = dPhi/dp (exact derivative of the residual; in the interior
 * the printed entries of Supplementary A (arithmetic) and C (upstream)) and
 * the diffusion-only SPD matrix A_aux = diag(rho_phi s'/dt) + sum over faces
 * of (K_av/h^2)(e_c - e_nb)(e_c - e_nb)^T (Dirichlet faces on the diagonal),
 * the frozen-coefficient matrix of q_prec = -K(p) grad p (Sec. 4).  Both are
 * kept in the context for amg_setup / krylov_solve.  J7_dev and A7_dev, if
 * not NULL, receive copies in the 7n stencil layout. */
int rich_jacobian(rich_ctx* ctx, const double* p_dev, double dt, double* J7_dev, double* A7_dev);

/* y_dev = J x_dev with the context's current Jacobian (stencil SpMV). */
int rich_jacobian_apply(rich_ctx* ctx, const double* x_dev, double* y_dev);

/* ---- Sec. 5.2: AMG ----------------------------------------------------- */
/* Build the smoothed-aggregation hierarchy from the context's current A_aux
 * (strength, MIS-2 aggregation, P = (I - omega D^-1 A) P_tent, R = P^T,
 * A_{l+1} = R A_l P, dense inverse of the coarsest matrix).  opts NULL =
 * defaults.  info_host, if not NULL, receives the level sizes. */
int amg_setup(rich_ctx* ctx, const rich_amg_opts* opts, rich_amg_info* info_host);
/* Refresh the hierarchy from the context's current A_aux (policy
 * RICH_AMG_REFRESH or RICH_AMG_SETUP_ONCE semantics). */
int amg_update(rich_ctx* ctx, int policy);
/* z_dev = B r_dev: one V-cycle with zero initial guess (FP64 in and out; in
 * MIXED mode the cycle itself runs in FP32). */
int amg_vcycle(rich_ctx* ctx, const double* r_dev, double* z_dev);
/* Export level l for inspection (host buffers sized from rich_amg_info;
 * RICH_EINVAL for a level the hierarchy does not have, e.g. any with AS):
 * aggregate index per node of level l (n[l] ints, level < levels-1), and the
 * CSR of A_l (rowptr n[l]+1, col nnz, val nnz).  Any pointer may be NULL.
 * In MIXED precision, levels below the finest return the FP32 values the
 * V-cycle uses (the Galerkin refresh runs in FP32 there), widened to double. */
int amg_export_level(rich_ctx* ctx, int level, int* agg_host, int* rowptr_host, int* col_host,
                     double* val_host);
/* Export P_l (n[l] x n[l+1]) as CSR to host buffers; nnz via nnz_out. */
int amg_export_prolongator(rich_ctx* ctx, int level, long long* nnz_out, int* rowptr_host, int* col_host,
                           double* val_host);

/* ---- Sec. 3: Newton correction solve ------------------------------------ */
/* Solve J x = b (current Jacobian, current hierarchy) with x0 = 0. */
int krylov_solve(rich_ctx* ctx, const double* b_dev, double* x_dev, const rich_krylov_opts* opts,
                 rich_krylov_stats* stats_host);

/* ---- Sec. 3: one backward-Euler step ------------------------------------ */
/* p_dev holds p^{l-1} on entry and p^l on return (or the last accepted
 * Newton iterate on error; under time-step control, the pressure at the start
 * of the substep that failed).  opts NULL = defaults.
 * The first call of a context builds the AMG hierarchy.  Counts in stats_host
 * cover every attempt, discarded ones included. */
int rich_step(rich_ctx* ctx, double* p_dev, double dt, const rich_newton_opts* opts,
              rich_step_stats* stats_host);
/* The same step on a host array: copies p_host to the device, steps, and
 * copies the result back (both copies on the context's stream). */
int rich_step_host(rich_ctx* ctx, double* p_host, double dt, const rich_newton_opts* opts,
                   rich_step_stats* stats_host);

/* ---- batched steps (several small problems, one launch per operation) ----- */
/* A context holding nbatch (1..32) independent problems of one grid shape,
 * stacked along z: problem b owns cells [b n, (b+1) n) (n = nx ny nz of `grid`),
 * the stacked grid keeps the problems' spacing, and the faces between two stacked
 * problems are their own bottom and top faces (bc applies to each).  soil->ks_field_dev,
 * if not NULL, holds nbatch * n values; per-cell Dirichlet values are accepted on the
 * z faces only (the same for every problem).  The paper has no batched form; this is
 * how the request server packs small requests: every kernel launch (constitutive
 * law, residual, Jacobian, stencil SpMV, each V-cycle level operation) covers all
 * problems, while the Newton iteration, its line search and FCG keep their scalars,
 * convergence tests and statistics per problem. */
int rich_create_batch(const rich_grid* grid, int nbatch, const rich_soil* soil, int kmean, const rich_bc* bc,
                      int precision, void* stream, rich_ctx** out);
/* One backward-Euler step (Sec. 3) of every problem of a batch context: p_dev holds
 * nbatch * n values; stats_host and status_host receive one entry per problem
 * (status as rich_step's; a problem that fails is left at its last accepted Newton
 * iterate and does not hold the others back).  opts must use FCG without time-step
 * control (RICH_EINVAL otherwise); RICH_ELIMIT where 3 x nbatch x the per-problem
 * reduction grid exceeds the context's partial-sum buffer (only above 21 problems); there is no FGMRES fallback in a batch, so a
 * problem whose FCG fails reports RICH_ENOTCONV_LIN.  The AMG hierarchy is built on
 * the block-diagonal diffusion matrix of all problems (aggregates never cross
 * problems) at the first call and refreshed afterwards.  Returns RICH_OK when the
 * batch ran (whatever the per-problem statuses), an error code otherwise. */
int rich_step_batch(rich_ctx* ctx, double* p_dev, double dt, const rich_newton_opts* opts,
                    rich_step_stats* stats_host, int* status_host);

/* ---- instrumentation ----------------------------------------------------- */
/* Measured arithmetic peak of the current device in TFLOP/s (2 flops per fused
 * multiply-add): FP64 (fp64 != 0) or FP32 FMA pipes, non-tensor, timed with CUDA
 * events over launches that keep every SM busy with independent FMA chains (the
 * best of three after a warm-up launch; about 0.1 s).  Allocates a small buffer
 * and synchronises the device's legacy default stream.  Used to place FP64
 * kernels on their roofline. */
int rich_measure_fma_peak(int fp64, double* tflops);

/* The autotuner's choices so far, one line "mode value_bytes rows_bin mean_row_length
 * sell_offered variant best_us best_csr_variant" each (mode 0 y = A x, 1 y += A x,
 * 2 l1-Jacobi sweep, 3 residual; rows_bin = floor(4 log2 rows); sell_offered 1 where a
 * SELL copy was a candidate; variant = lanes per row, + 256 for four-way unrolled rows,
 * 512 / 513 for the SELL copy with 4 / 8 gathers in flight per row, 514 for the SELL
 * copy with two lanes per row, 515 for the software-pipelined one; best_csr_variant
 * the fastest CSR candidate), written into buf (at most cap bytes, NUL-terminated). */
int rich_autotune_table(char* buf, int cap);
/* Adds the entries of a saved table (rich_autotune_table's text) to the process's
 * autotuner, so that a later process runs the same variants without timing them
 * (e.g. under a profiler, whose serialised launches would skew the timings).
 * Classes already tuned keep their choice.  RICH_EINVAL (nothing added) on a
 * malformed line or an unknown variant. */
int rich_autotune_load(const char* text);
/* The SELL-C-sigma layout (csr_layout) the library gives a CSR matrix of n rows
 * (the coarse operators, restrictions and prolongators of the Sec. 5.2 hierarchy),
 * computed on the host from its row pointer (rowptr_host, n + 1 entries,
 * non-decreasing): rows sorted by decreasing length (ties in row order) within
 * each window of 1024 rows, cut into slices of 32.  perm_host receives
 * 32 * ceil(n / 32) row indices (-1 past n), sptr_host the ceil(n / 32) + 1 slot
 * offsets of the slices (slice s spans 32 x its first row's length slots), and
 * *slots their total.  Host memory only; RICH_EINVAL on a bad argument or a
 * decreasing row pointer, RICH_ELIMIT when the slots exceed 32-bit offsets. */
int rich_sell_layout(const int* rowptr_host, int n, int* perm_host, int* sptr_host,
                     long long* slots);

/* Number of kernels this library has launched since it was loaded. */
int rich_kernel_launches(long long* out);
/* Time every launch of the kernel called name (NULL disables) with CUDA events
 * on its launching stream, from now until the next call.  Names: "residual",
 * "assemble", "stencil_spmv", "l1jacobi_l0", "l1jacobi", "csr_resid",
 * "restrict", "prolong", "coarse_gemv", "multidot", "multiaxpy", "fcg_update",
 * "spgemm_numeric". */
int rich_profile_kernel(const char* name);
/* Time only every stride-th launch of the profiling target (1 = every launch,
 * the default); the events around each timed launch cost a few microseconds of
 * host and device time, so a stride keeps a long run's timing close to an
 * unprofiled one.  A stride coprime with the period of the launch pattern
 * (e.g. 7 for the V-cycle's six sweeps) samples every position of it.
 * RICH_EINVAL for stride < 1. */
int rich_profile_stride(int stride);
/* Sum of the recorded launch durations (ms), number of recorded launches, the
 * algorithmic bytes those launches must move and (flops_total may be NULL) their
 * algorithmic floating-point operations (synchronises the events). */
int rich_profile_result(double* ms_total, long long* launches, double* bytes_total, double* flops_total);
/* With the target "*": per-kernel totals, one line "name launches ms bytes flops"
 * each (algorithmic bytes and flops), written into buf (at most cap bytes,
 * NUL-terminated). */
int rich_profile_table(char* buf, int cap);

/* Peak device memory of the library on the current device: every allocation it
 * makes comes from that device's stream-ordered pool, whose high-water marks of
 * bytes in use and bytes reserved are returned (either pointer may be NULL).
 * reset != 0 restarts both marks from the current usage. */
int rich_memory_peak(long long* used_high, long long* reserved_high, int reset);

/* Default option structs (as listed in the comments above). */
void rich_default_newton_opts(rich_newton_opts* o);
void rich_default_amg_opts(rich_amg_opts* o);

/* ---- request server (serving many time-step solves at once) -------------- */
/* A server takes time-step requests of any grid size and soil as they arrive
 * and runs up to `slots` of them on the device at once: each slot is a host
 * worker thread with its own CUDA stream, so the kernels of different requests
 * overlap on the GPU.  A request is admitted, in arrival order, as soon as a
 * slot is free and its device-memory estimate fits in the budget next to the
 * requests in flight and the resident sessions (least recently used idle
 * sessions are evicted to make room).  Device memory is stream-ordered, so
 * admitting or finishing one request never waits for another.  Each request
 * runs the same kernels, in the same order, as a lone rich_step on its own
 * context, so its result does not depend on what else is in flight.  The
 * paper has no serving layer; this is the deployment form of Sec. 3's step. */
typedef struct rich_server rich_server;

typedef struct {
  int slots;               /* requests in flight at once (8) */
  double mem_budget_bytes; /* device bytes requests and sessions may hold; <= 0: 80 % of the free memory at creation */
  int max_sessions;        /* resident sessions kept at most (64) */
  int batch_max;           /* 1 (default): one request per slot.  B > 1: a worker that takes a one-off
                              request also takes up to B-1 more queued one-off requests of the same grid,
                              soil parameters, mean, boundary values, precision, dt and options (FCG,
                              no time-step control) and steps them together as one batch
                              (rich_create_batch / rich_step_batch); a member whose step fails in the
                              batch is rerun alone, so every result is the lone path's wherever the
                              batch cannot match it.  A class (grid, mean, precision) of which more than
                              a quarter of the batched members failed, once 16 were recorded, is served
                              alone from then on */
  int batch_min_cells;     /* only requests of at most this many cells are batched (300000) */
} rich_server_opts;

typedef struct {
  rich_grid grid;
  rich_soil soil;              /* ks_field_dev is ignored: see ks_field_host */
  const double* ks_field_host; /* n cells of K_s (host), or NULL for soil.ks_const */
  int kmean;                   /* RICH_KMEAN_* */
  rich_bc bc;                  /* constant face values (value_field_dev must be NULL) */
  int precision;               /* RICH_PREC_* */
  double dt;                   /* time step */
  rich_newton_opts opts;
  const double* p0_host;       /* n cells of p^{l-1}; NULL continues the session's resident pressure */
  double* p_out_host;          /* n cells, receives p^l when the request finishes (may be NULL); after a
                                  failed step, the last accepted Newton iterate */
  long long session;           /* 0: one-off.  Otherwise the server keeps this problem's context (pressure,
                                  AMG hierarchy) on the device for later requests with the same id, which
                                  must have the same grid, soil, kmean, bc and precision (else RICH_EINVAL);
                                  once evicted, a request with p0_host NULL returns RICH_ESTATE */
} rich_request;

typedef struct {
  int status;                  /* the step's status (RICH_OK or an error code) */
  rich_step_stats stats;
  double t_submit, t_admit, t_done; /* seconds since the server was created */
  int slot;                    /* worker slot that ran it */
  double mem_estimate;         /* device bytes reserved for it at admission */
  double mem_in_flight;        /* bytes reserved by all admitted requests and sessions, itself included */
  int batch_size;              /* requests stepped together with this one (1: alone) */
  int batch_rerun;             /* 1 if its step failed in a batch and was rerun alone */
} rich_request_result;

void rich_default_server_opts(rich_server_opts* o);
/* Starts the worker threads on the current device.  RICH_EINVAL for slots < 1
 * or max_sessions < 0. */
int rich_server_create(const rich_server_opts* opts, rich_server** out);
/* Queues a request (the struct is copied; the host arrays it points to must stay
 * valid until the request has finished) and returns its id (> 0).  RICH_EINVAL
 * for a malformed request, RICH_ELIMIT if its estimate exceeds the whole budget. */
int rich_server_submit(rich_server* s, const rich_request* req, long long* id_out);
/* RICH_OK with *out filled once request id has finished (the id is then
 * released), RICH_EBUSY while it is queued or running, RICH_EINVAL for an
 * unknown id. */
int rich_server_poll(rich_server* s, long long id, rich_request_result* out);
/* Blocks until request id has finished; then as rich_server_poll. */
int rich_server_wait(rich_server* s, long long id, rich_request_result* out);
/* Blocks until every submitted request has finished. */
int rich_server_drain(rich_server* s);
/* Requests admitted so far, the most that were in flight at once, and the
 * device bytes reserved now (any pointer may be NULL). */
int rich_server_counters(rich_server* s, long long* admitted, int* max_in_flight, double* reserved_bytes);
/* Finishes the queued and running requests, stops the workers and frees every
 * resident session. */
int rich_server_destroy(rich_server* s);

#ifdef __cplusplus
}
#endif
#endif /* RICHARDS_GB300_H */
