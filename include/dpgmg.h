/*
 * dpgmg.h -- C ABI of the GB300 DPG multigrid solver for 3D time-harmonic
 * acoustics (Badger, Henneking, Petrides, Demkowicz, arXiv 2304.01728).
 *
 * Problem (Sec. 2, Eq. helmholtz, with the wavespeed reading rho = 1, bulk
 * modulus c^2, impedance Z = c):
 *     i w c^-2 p + div u = f,   i w u + grad p = g   in Omega (an axis-aligned box)
 *     Z^-1 p - u.n = u0                               on Gamma = boundary of Omega
 * discretised by the broken ultraweak DPG method of Sec. 2 (trial fields in
 * L^2 of order p, traces p-hat in H^{1/2}, u-hat_n in H^{-1/2}, test space
 * enriched by dp = 1, adjoint graph test norm Eq. Gnorm with alpha = 1),
 * statically condensed onto the trace unknowns (Sec. 1.2), and solved by
 * conjugate gradients preconditioned with the DPG-MG V-cycle of Sec. 3
 * (macro-grid prolongation, vertex-patch additive Schwarz smoothing, coarse
 * operators restricted from the fine grid).  The impedance condition is
 * built in by eliminating u-hat_n on Gamma: boundary faces carry p-hat only.
 *
 * Conventions for every call:
 *   - Return value: DPGMG_OK (0) or a negative DPGMG_ERR_* code; no
 *     exception or signal crosses the ABI.  dpgmg_strerror() names the code;
 *     dpgmg_last_error() gives a message for the calling thread.
 *   - Complex arrays are interleaved (re, im) doubles ("c128").
 *   - Input arrays are host arrays owned by the caller and are copied during
 *     the call.  Output arrays are owned by the caller; they are host arrays
 *     unless the call says otherwise.
 *   - A handle owns one CUDA device (and optionally one caller stream) and all
 *     device memory of the systems set up through it, until dpgmg_release() /
 *     dpgmg_destroy().  Calls on one handle are serialised by an internal
 *     mutex; distinct handles may be used from distinct threads.
 *
 * Global trace numbering (the order of dpgmg_solve's trace output), for an
 * nx x ny x nz mesh of order p:
 *   block V  vertices, 1 DOF each; vertex (i,j,k) -> i + (nx+1)(j + (ny+1)k)
 *   block E  edges along x, then y, then z; an edge along axis d at lattice
 *            position (i,j,k) has index extents n_e + (e != d) and p-1 DOFs
 *            (H^1 modes 2..p of that axis)
 *   block F  faces normal to x, then y, then z (p-hat); extents n_e + (e == d);
 *            (p-1)^2 DOFs, modes (m1, m2) of the tangential axes (increasing
 *            axis order), index (m1-2) + (p-1)(m2-2)
 *   block U  interior faces only (u-hat_n, the flux along the +axis normal),
 *            same face order with boundary faces skipped; p^2 DOFs, Legendre
 *            modes (a, b) of the tangential axes, index a + p b.
 * The 1D bases on an element's unit interval: Legendre L_a(x) = P_a(2x-1);
 * H^1: phi_0 = 1-x, phi_1 = x, phi_k = (P_k - P_{k-2})(2x-1)/sqrt(2(2k-1)).
 * Element-local trace order: p-hat functions phi_a phi_b phi_c, (a,b,c) in
 * {0..p}^3 by a + (p+1)(b + (p+1)c) keeping triples with an index < 2, then
 * u-hat of faces x-, x+, y-, y+, z-, z+ with modes a + p b.
 * Field output per element: [p, u_x, u_y, u_z], each sum_abc coef L_a L_b L_c
 * with a, b, c < p, index a + p(b + p c); elements ordered i + nx(j + ny k).
 */
#ifndef DPGMG_H
#define DPGMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DPGMG_OK                  0
#define DPGMG_ERR_ARG            -1  /* invalid argument or unsupported option */
#define DPGMG_ERR_NOMEM          -2  /* device-memory budget or allocation exceeded */
#define DPGMG_ERR_NOT_HPD        -3  /* a Cholesky pivot <= 0 (element, patch, coarse) */
#define DPGMG_ERR_BREAKDOWN      -4  /* CG breakdown: (p, Ap) <= 0 or not finite */
#define DPGMG_ERR_NOT_CONVERGED  -5  /* max_iter reached; outputs and stats still written */
#define DPGMG_ERR_TIMEOUT        -6  /* a bounded device wait expired */
#define DPGMG_ERR_PENDING        -7  /* serving: request not finished yet */
#define DPGMG_ERR_CUDA           -8  /* a CUDA runtime call failed */

/* ---- enums ------------------------------------------------------------- */
#define DPGMG_SRC_GAUSSIAN      0   /* f = A exp(-|x-x0|^2/(2 s^2)), g = 0, u0 = 0 */
#define DPGMG_SRC_PLANE_WAVE    1   /* u0 of p = exp(-i w d.x/c), u = d p / c; f = g = 0 */
#define DPGMG_SRC_MANUFACTURED  2   /* f, g, u0 of given polynomials p_ex, u_ex */

#define DPGMG_PREC_FP64   0         /* V-cycle in complex128 */
#define DPGMG_PREC_MIXED  1         /* V-cycle in complex64 (patch factors in FP32), CG in complex128 */

#define DPGMG_COARSEST_CHOLESKY 0   /* dense Cholesky solve on level 0 */
#define DPGMG_COARSEST_NONE     1   /* no level-0 correction (Sec. 4 list) */
#define DPGMG_COARSEST_AUTO     2   /* CHOLESKY if level 0 has at most 20,000 DOFs, else NONE */
#define DPGMG_COARSEST_SMOOTH   3   /* one damped additive-Schwarz step on level 0 (vertex patches of
                                       its own mesh, damping by the same power iteration) instead of
                                       a solve; a single-level system still uses CHOLESKY */

/* ---- problem and options ----------------------------------------------- */
typedef struct dpgmg_problem {
  int n[3];                /* elements per axis, each >= 1 */
  double x0[3], x1[3];     /* box corners, x1 > x0 */
  int p;                   /* trial order, 1..5 */
  int dp;                  /* test enrichment; must be 1 (Sec. 2) */
  double omega;            /* angular frequency w > 0 */
  const double* wavespeed; /* host [n0*n1*n2] per element (> 0), or NULL for c = 1 */
  int source;              /* DPGMG_SRC_* */
  double src_center[3];    /* Gaussian centre x0 */
  double src_width;        /* Gaussian standard deviation s > 0 */
  double src_amp;          /* Gaussian amplitude A */
  double wave_dir[3];      /* plane wave direction d (normalised internally); needs constant c */
  int mf_order;            /* manufactured: polynomial degree + 1 per axis (m >= 1) */
  const double* mf_coeffs; /* manufactured: host c128 [4][m][m][m] (comp, c, b, a):
                              comp 0 = p_ex, 1..3 = u_ex components; tensor Legendre
                              L_a(X) L_b(Y) L_c(Z) in box coordinates X = (x-x0)/(x1-x0) */
  const double* u0_samples;/* optional impedance load of the caller, added to the source's own
                              u0 (Sec. 2, impedance condition Z^-1 p - u.n = u0 on Gamma):
                              host c128 [n_points] (re, im) of u0 at the boundary points that
                              dpgmg_boundary_points lists, in that order; NULL = none.  The
                              element stage integrates <u0, q> over each boundary face with
                              the same Gauss rule, so u0 enters exactly as sampled. */
} dpgmg_problem;

typedef struct dpgmg_opts {
  double tol;              /* relative residual target ||r||/||b|| (Sec. 4: 1e-7; default 1e-8) */
  int max_iter;            /* CG iteration cap */
  int nu_pre, nu_post;     /* smoothing steps per level (V(1,1) default, Sec. 4) */
  int n_levels;            /* levels incl. finest and coarsest, >= 1 */
  int p_min;               /* lowest order of the p-coarsening stage (>= 1) */
  int precision;           /* DPGMG_PREC_* */
  int coarsest;            /* DPGMG_COARSEST_* */
  int flags;               /* DPGMG_FLAG_* bits, 0 by default */
  double theta;            /* smoother damping; <= 0 => estimate by power iteration */
} dpgmg_opts;

/* CG steps after the first are replayed from one captured CUDA graph unless
   this bit is set (or the stream cannot be captured); results are the same. */
#define DPGMG_FLAG_EAGER 1
/* Mixed path: the coarsest complex64 factorisation (Cholesky and triangular
   inverse) on the FP32 CUDA cores, in 64-wide blocks, instead of the default:
   panels of up to 512 columns whose panel solves, trailing updates and
   inverse updates are complex products on the tensor cores (tcgen05, 3xTF32
   operand splitting, each 8-column K stage accumulated in TMEM and added to
   FP32 registers with round-to-nearest), with only the diagonal blocks on the
   CUDA cores.  Both give coarse solves of FP32 accuracy. */
#define DPGMG_FLAG_CUDA_CORES 2
/* Coarse operators "stored" instead of restricted (Sec. 3, the paper's
   alternative construction): every coarser level's operator is the DPG system
   assembled directly on its own mesh and order (enriched test order p_c + 1)
   rather than I^T M I of the finer operator.  Needs a constant wavespeed
   (DPGMG_ERR_ARG otherwise); transfers and smoothers are unchanged. */
#define DPGMG_FLAG_STORE_COARSE 4
/* Warm start: dpgmg_solve takes its initial CG iterate from the trace_out
   buffer (host or device per out_is_device) instead of 0, e.g. the solution of
   a nearby load or frequency (Sec. 5 starts each adaptive mesh from the
   previous solution); the stopping test stays ||r|| <= tol ||b||, and an
   initial guess that already meets it returns after 0 iterations.  The
   serving path always starts from 0. */
#define DPGMG_FLAG_WARM_START 8
/* CG operator in complex128 on the FP64 pipe instead of the default
   double-float form (complex64 high and low parts of every FP64 entry, products
   and sums by error-free FP32 transformations, ~48 significant bits; Sec. 3
   runs CG on the condensed FP64 system).  The damping estimate of setup then
   iterates with the complex128 operator and patch inverses too.  With
   DPGMG_PREC_FP64 every step of the path is then complex128.  Same results to
   rounding; the FP64 pipe of this GPU makes the CG operator several times
   slower. */
#define DPGMG_FLAG_CG_C128 16
/* Mixed path: factor the vertex-patch blocks in FP64 and round their inverses
   to complex64 afterwards, instead of the default complex64 blocks factored in
   FP32 (Cholesky, triangular inverse and L^-H L^-1), the V-cycle's own
   precision.  Setup is slower (the FP64 pipe of this GPU); the smoother then
   differs from the FP64 one by the rounding of its entries only. */
#define DPGMG_FLAG_PATCH_FP64 32
/* Vertex-patch membership rule R2 instead of R1 (Sec. 3, "V-cycle and
   smoother": one block per vertex of the next coarser mesh; the paper does not
   say how blocks end at the boundary).  R1, the default: a DOF is in the block
   of vertex w when every (macro-)element adjacent to its entity has w as a
   corner.  R2: when w lies in the closure of the coarse entity carrying the DOF
   (its own entity on p levels, the coarse entity whose interior holds it on h
   levels).  They differ on boundary entities only, which R1 also gives to the
   vertices one layer inside: R2 blocks are smaller there (largest block 67
   against 104 on a 4^3 p = 2 mesh).  Applies to every smoothed level,
   including level 0 under DPGMG_COARSEST_SMOOTH. */
#define DPGMG_FLAG_PATCH_R2 64
/* Memory-lean smoother (Sec. 5: patch storage limits the order; recomputing
   the patches during the solve is the paper's proposed remedy on GPUs): the
   patch inverses are not stored.  Every smoother application gathers the
   complex64 blocks from the level operator, factors them in FP32 and applies
   them, window by window (consecutive patches, largest first, a quarter of
   the level's blocks and at most 256 MiB per window), so a level holds two
   window buffers instead of its sum n_j^2 stored entries.
   Same arithmetic as the stored FP32 factors: the same results.  Far more
   work per iteration; several loads per solve (dpgmg_solve_block) share it.
   Mixed path only, without DPGMG_FLAG_PATCH_FP64 and DPGMG_FLAG_CG_C128
   (ARG otherwise); dpgmg_smooth_noalloc is not available (ARG). */
#define DPGMG_FLAG_RECOMPUTE_PATCHES 128
/* Mixed path: keep every stored matrix of the solve in complex64 (the
   comparison for the default real packing).  By default a block that is real
   once the unit phases of the real form are taken out (p-hat DOFs carry i;
   true of everything that only elements without an impedance face and with a
   real source touch: Sec. 2, impedance condition) is stored as reals at half
   the bytes:
     patch inverses: A_j^-1[r][c] = w[r][c] i^(s_r - s_c), s = 1 on p-hat DOFs;
     operators (V-cycle complex64 values, and the CG operator's high and low
     parts): every row of an entity whose entries are all of that form.
   The products apply the phases exactly; their results differ from the
   complex64 ones by FP32 rounding order only. */
#define DPGMG_FLAG_COMPLEX_STORAGE 256
/* Host-made failures for testing the error paths (the paper has no
   counterpart; no GPU fault is involved):
   FAULT_NOT_HPD: the host overwrites the first diagonal entry of the dense
     coarsest matrix with -1 before its factorisation, which then reports a
     non-positive pivot: dpgmg_setup returns DPGMG_ERR_NOT_HPD (needs a dense
     coarsest level).
   FAULT_TC_WAIT: on the mixed path (tensor-core coarsest factorisation,
     level 0 above 128 DOFs), the first tensor-core product issues no MMA and
     no commit, so its bounded waits (about half a second) run out with only
     its own operand copies in flight, which it lets land: dpgmg_setup returns
     DPGMG_ERR_TIMEOUT and the later products of the setup skip their work.
   In both cases the handle stays usable. */
#define DPGMG_FLAG_FAULT_NOT_HPD (1 << 28)
#define DPGMG_FLAG_FAULT_TC_WAIT (1 << 29)

typedef struct dpgmg_stats {
  int iters;               /* CG iterations (= V-cycle applications) */
  double relres;           /* final recursive relative residual */
  double true_relres;      /* ||b - A x|| / ||b|| recomputed at exit (FP64) */
  double t_setup_ms;       /* device time of dpgmg_setup */
  double t_pcg_ms;         /* device time from the first CG step to convergence */
  long long bytes_per_iter;/* algorithmic bytes of one CG iteration (matrix entries read once) */
  long long n_dof;         /* finest trace DOFs */
  long long dev_bytes_peak;/* peak device bytes held by the system */
} dpgmg_stats;

typedef struct dpgmg_level_desc {
  int n[3], p;
  long long n_dof;         /* trace DOFs of the level's mesh and order */
  long long n_smooth;      /* DOFs the smoother acts on (macro DOFs on h levels) */
  int kind;                /* transition to the level below: 0 none, 1 p, 2 h */
  long long n_patches;
  long long patch_max;
  long long sum_patch_sq;  /* sum of squared patch sizes */
  long long op_nnz;        /* stored entries of the level's smoothing operator */
  double theta;
  long long patch_stored;  /* stored patch-inverse entries (sum n_j^2, or sum n_j(n_j+1)/2 in
                              Hermitian half storage) */
  long long patch_real_sq; /* sum of n_j^2 over the patches whose inverses are stored as real
                              blocks (mixed path, see DPGMG_FLAG_COMPLEX_STORAGE): half the bytes */
  long long op_real_nnz;   /* entries of the level's complex64 operator stored as reals (the same) */
} dpgmg_level_desc;

typedef struct dpgmg_handle_s* dpgmg_handle;
typedef struct dpgmg_system_s* dpgmg_system;
typedef long long dpgmg_ticket;

/* Create a handle bound to CUDA device `device`.  mem_budget_bytes caps the
 * device memory of all systems of this handle (0 = 90% of free memory).
 * cuda_stream: a cudaStream_t to issue work on, or NULL for a private stream. */
int dpgmg_create(dpgmg_handle* h, int device, size_t mem_budget_bytes, void* cuda_stream);
void dpgmg_destroy(dpgmg_handle h);

/* Sizes of a problem without touching the device: finest trace DOFs, field
 * DOFs (n_elem * 4 p^3) and the device bytes dpgmg_setup would hold. */
int dpgmg_query_sizes(const dpgmg_problem* pb, const dpgmg_opts* op,
                      long long* n_trace, long long* n_field, size_t* dev_bytes);

/* Entity and mode of every global trace DOF of a problem's finest mesh (the
 * numbering documented above), without touching the device.  out: host int
 * [n_trace][7], per DOF (kind, cx, cy, cz, axis, m1, m2):
 *   kind 0 vertex, 1 edge, 2 face (p-hat), 3 interior face (u-hat_n);
 *   (cx, cy, cz) the entity's centre in half-element units (vertex (i,j,k)
 *   at (2i, 2j, 2k), the x-edge from it at (2i+1, 2j, 2k));
 *   axis the edge direction (edges) or face normal (faces), -1 for vertices;
 *   (m1, m2) the H^1 mode of an edge (m1 = 2..p, m2 = -1), the H^1 modes of
 *   a face's tangential axes in increasing axis order (2..p each), or the
 *   Legendre modes (a, b) of a u-hat face (0..p-1 each); -1 for vertices.
 * n_trace must equal the count dpgmg_query_sizes reports.  Errors: ARG. */
int dpgmg_dof_map(const dpgmg_problem* pb, long long n_trace, int* out);

/* Points at which to sample a caller's impedance load u0 (dpgmg_problem
 * u0_samples), without touching the device.  On return *n_points = the count:
 * 2 (n1 n2 + n0 n2 + n0 n1) boundary faces times q^2 points, q = p + 5 (the
 * element stage's Gauss-Legendre load rule).  Order: sides (d, s) for d = 0,
 * 1, 2 and s = 0 (x_d = x0_d), 1 (x_d = x1_d); within a side the faces (j1, j2)
 * along the tangential axes t1 < t2, j1 fastest; within a face the points
 * (a, b) at (x_t1, x_t2) = corner + (xi_a h_t1, xi_b h_t2), a fastest.
 * xyz: host double [n][3] of capacity *n_points on entry, or NULL to query
 * the count only.  Errors: ARG (invalid problem, capacity too small). */
int dpgmg_boundary_points(const dpgmg_problem* pb, long long* n_points, double* xyz);

/* Default options: tol 1e-8, max_iter 2000, V(1,1), 2 levels, p_min 2, FP64,
 * Cholesky coarsest, theta estimated. */
void dpgmg_default_opts(dpgmg_opts* op);

/* Build the whole hierarchy on the device (Sec. 2-3): batched element DPG
 * matrices (enriched-test Gram Cholesky, B^* G^-1 B, static condensation),
 * assembly, p-restriction / macro condensation + natural inclusion +
 * restriction per level, patch factorisations, damping, coarsest factor.
 * Errors: ARG (invalid problem/options), NOMEM (over budget; nothing kept),
 * NOT_HPD (a factorisation failed), CUDA. */
int dpgmg_setup(dpgmg_handle h, const dpgmg_problem* pb, const dpgmg_opts* op,
                dpgmg_system* sys);

/* MG-preconditioned CG from x0 = 0 (Sec. 3-4) and field recovery.
 * trace_out: c128[n_trace] (global numbering above) or NULL;
 * field_out: c128[n_elem*4p^3] or NULL; both device pointers when
 * out_is_device != 0, else host.  st may be NULL.
 * Errors: NOT_CONVERGED (outputs written), BREAKDOWN, TIMEOUT, CUDA. */
int dpgmg_solve(dpgmg_handle h, dpgmg_system sys, void* trace_out, void* field_out,
                int out_is_device, dpgmg_stats* st);

/* Several loads on one system at once (Sec. 5: loads solved together share the
 * cost of the smoothing patches): k independent MG-PCG solves from x0 = 0, one
 * per right-hand side, each with its own scalars and stopping test (the
 * recurrence of dpgmg_solve), sharing every V-cycle.  The V-cycle's smoother
 * and SpMV read their stored matrices once for up to 4 right-hand sides.
 * rhs: c128 [k][n_trace] condensed right-hand sides (e.g. dpgmg_rhs of
 * systems with other sources); trace_out: c128 [k][n_trace]; both device
 * pointers when on_device != 0, else host.  stats: k entries or NULL; each
 * gets its own iterations and residuals, t_pcg_ms is the time of the whole
 * block.  1 <= k <= 64.  Returns the first non-OK status of the columns
 * (NOT_CONVERGED, BREAKDOWN), with every column's outputs written. */
int dpgmg_solve_block(dpgmg_handle h, dpgmg_system sys, int k, const void* rhs, void* trace_out,
                      int on_device, dpgmg_stats* stats);

void dpgmg_release(dpgmg_handle h, dpgmg_system sys);
const char* dpgmg_strerror(int code);

/* ---- serving (continuous batching) ---------------------------------------- */

/* Start the serving loop of a handle with `slots` concurrent solves (1..64);
 * optional, the first dpgmg_submit starts it with 4 slots.  Each slot owns a
 * CUDA stream.  One memory ledger per handle covers both kinds of use: a
 * request is admitted only while its footprint estimate, the estimates of the
 * running requests and the memory held by systems set up with dpgmg_setup
 * together fit the handle's budget, and dpgmg_setup counts the running
 * requests' estimates in the same way.  Errors: ARG (bad count, or already
 * started with another count). */
int dpgmg_serve_start(dpgmg_handle h, int slots);

/* Queue one solve (the same problem and options as dpgmg_setup + dpgmg_solve,
 * copied during the call) and return its ticket without waiting.  Requests
 * are admitted first-fit as a slot is free and their footprint estimate
 * (dpgmg_query_sizes) fits the handle's memory not held by running requests
 * or set-up systems, so requests arriving while others run start as memory
 * frees up and their work overlaps on the device.  Errors: ARG; NOMEM if the
 * footprint exceeds the handle's whole budget (the request is refused, not
 * queued). */
int dpgmg_submit(dpgmg_handle h, const dpgmg_problem* pb, const dpgmg_opts* op, dpgmg_ticket* ticket);

/* Collect a finished request: DPGMG_ERR_PENDING while it is queued or running;
 * otherwise copies the trace (c128[n_trace]) and fields (c128[n_elem*4p^3])
 * into the host buffers (either may be NULL), fills st and latency_ms
 * (completion minus submission, host clock) and returns the request's status
 * (OK, NOT_CONVERGED, NOMEM, NOT_HPD, ...).  A collected ticket is forgotten;
 * polling it again returns ARG.  dpgmg_destroy stops the loop and drops
 * requests not yet collected. */
int dpgmg_poll(dpgmg_handle h, dpgmg_ticket ticket, void* trace_out, void* field_out, dpgmg_stats* st,
               double* latency_ms);
const char* dpgmg_last_error(void);

/* ---- introspection (one call per step of the hot path, used by tests) ---- */

/* Level l (0 = coarsest) description. */
int dpgmg_level_info(dpgmg_handle h, dpgmg_system sys, int level, dpgmg_level_desc* out);

/* Element matrix of level `level` for element e (local trace order above;
 * absent u-hat rows/columns are zero): host c128 [nloc*nloc], row-major.
 * On the finest level this is the condensed DPG element matrix
 * K_tt - K_tf K_ff^-1 K_ft of Sec. 1.2; below it the restricted coarse
 * element matrices of Sec. 3.  load_out (finest only, may be NULL): host
 * c128 [nloc], the condensed element load. */
int dpgmg_element_matrix(dpgmg_handle h, dpgmg_system sys, int level, long long e,
                         double* mat_out, double* load_out);

/* Assembled right-hand side b of the finest trace system: host c128 [n_trace]. */
int dpgmg_rhs(dpgmg_handle h, dpgmg_system sys, double* b_out);

#define DPGMG_OP_A          0  /* y = A_l x: the level's smoothing operator (A_l on p
                                  levels and the finest, macro M_l on h levels); on the
                                  finest level in CG precision (FP64) */
#define DPGMG_OP_SMOOTH     1  /* y = theta_l S_l x (additive Schwarz, Sec. 3) */
#define DPGMG_OP_VCYCLE     2  /* y = B_l x (V-cycle from level l down) */
#define DPGMG_OP_RESTRICT   3  /* y = P_l^* x  (level l -> l-1; x full level-l vector) */
#define DPGMG_OP_PROLONG    4  /* y = P_l x    (level l-1 -> l) */
#define DPGMG_OP_CONDENSE   5  /* y = x with macro-interior residual condensed (h levels) */
#define DPGMG_OP_COARSE     6  /* y = A_0^-1 x (level 0) */
#define DPGMG_OP_AFULL      7  /* y = A_L x on the finest level, FP64 (the CG operator) */

/* Apply one operator of level `level` to a host c128 vector x; y is a host
 * c128 vector.  Sizes: n_dof of the level (n_dof of level-1 for RESTRICT's y
 * and PROLONG's x).  On the mixed-precision path the V-cycle operators run
 * in complex64 (inputs rounded, outputs widened). */
int dpgmg_apply(dpgmg_handle h, dpgmg_system sys, int op, int level,
                const double* x, double* y);

/* ---- measurement hooks --------------------------------------------------- */

/* Number of CUDA kernels this library has launched in this process (all
 * handles), for counting the launches inside a timed region. */
long long dpgmg_launch_count(void);

#define DPGMG_PROF_OFF         0
#define DPGMG_PROF_SMOOTH_FINE 1  /* patch products of the finest smoother */
#define DPGMG_PROF_SPMV_FINE   2  /* residual SpMVs of the finest V-cycle level */
#define DPGMG_PROF_SPMV_CG     3  /* the FP64 CG operator application */

/* SpMV work decomposition, chosen at setup by timing.  The operators are
 * applied by one warp per group of G rows of one mesh entity (G = 1, 2, 4 or
 * 8; the rows of an entity share their column list, so larger G loads each
 * column index and vector entry once for G rows), or (G = 16) by one warp
 * per row with the column indices loaded one step ahead of the gathers they
 * feed, or (G = 32) by one warp per row with the warp's stream of values and
 * column indices copied 8 steps ahead into shared memory by asynchronous
 * copies (cp.async), or (G = 64, V-cycle operators only) by one half-warp
 * per row, two rows of a warp at a time.  dpgmg_setup times every variant on each operator and
 * keeps the fastest; choices are cached per (product type, p, level kind,
 * log2 of the row count) for the life of the process.  level >= 1 addresses
 * that level's V-cycle operator, level == -1 the CG operator.  set = 1, 2, 4,
 * 8, 16, 32 or 64 overrides the choice (0 leaves it; 64 is refused for the CG
 * operator); *group (may be NULL)
 * receives the value in force.  Returns DPGMG_ERR_ARG for an invalid level or
 * size.  Results do not depend on the variant beyond rounding order (G = 1,
 * 16 and 32: bitwise). */
int dpgmg_spmv_group(dpgmg_handle h, dpgmg_system sys, int level, int set, int* group);

/* DPG error indicator (Sec. 1.2: the residual that DPG minimises, in the
 * dual test norm, is the method's built-in error indicator; Sec. 3 refines
 * by it).  For the trace vector x (host, interleaved complex128 [n_trace],
 * e.g. the output of dpgmg_solve) the fields are recovered element by element
 * and every finest element's
 *     eta_K^2 = (l_K - B_K u_K)^* G_K^-1 (l_K - B_K u_K)
 * is written to eta2 (host double [n0*n1*n2], element order of the mesh),
 * u_K = [fields, local traces].  The global DPG residual is sum_K eta_K^2.
 * Recomputes G_K, B_K, l_K and the Gram Cholesky per element (FP64).
 * Errors: ARG (null argument), NOT_HPD, CUDA. */
int dpgmg_error_indicator(dpgmg_handle h, dpgmg_system sys, const double* x, double* eta2);

/* Setup phases of a system: device time of the batched element stage
 * (Sec. 2: Gram, B and load, Cholesky, optimal test functions, DPG matrix,
 * field condensation), the algorithmic GFLOP it executed (an FMA counts 2
 * flops, a complex FMA 8; per element of the full pipeline: Gram Cholesky
 * nt^3/6, W = L^-1 [B l] nt^2 (m+1)/2, K = W^H W (m+1)^2 nt/2, condensation
 * nf^3/6 + nf^2 (ntr+1) + ntr (ntr+1) nf multiply-adds; with element classes
 * (elements sharing impedance faces and wavespeed under a Gaussian source)
 * one representative per class runs the full pipeline and the others only
 * their load: nt^2/2 + m nt + nf^2 + ntr nf multiply-adds), and the whole
 * setup's device time.  Outputs may be NULL.  Returns DPGMG_ERR_ARG for a
 * null handle or system. */
int dpgmg_setup_profile(dpgmg_handle h, dpgmg_system sys, double* element_ms, double* element_gflop,
                        double* setup_ms);

/* Device time of each setup phase of a system, in ms, from CUDA events
 * recorded at the phase boundaries (the setup stream and the side stream of
 * the coarsest factorisation):
 *   [0] batched element stage (Sec. 2);
 *   [1] level operators and transfer data, finest to coarsest (restriction
 *       A_c = I^* M I, macro condensation of the h-levels, Sec. 3);
 *   [2] smoothers of all levels (patch extraction and inversion, damping
 *       theta, complex64 copies on the mixed path);
 *   [3] coarsest factorisation on the side stream, overlapping [2]
 *       (0 when it ran on the setup stream);
 *   [4] wait for the coarsest factorisation after [2] (its whole time when
 *       it ran on the setup stream);
 *   [5] load assembly and solve preparation (CG operator split, tuning).
 * [0] + [1] + [2] + [4] + [5] is the setup's device time.  Writes
 * min(n, DPGMG_SETUP_NPHASES) values to ms (host).  Errors: ARG (null
 * argument, n < 1). */
#define DPGMG_SETUP_NPHASES 6
int dpgmg_setup_phases(dpgmg_handle h, dpgmg_system sys, double* ms, int n);

/* Bracket every launch of one kernel with CUDA events on the launching
 * stream during subsequent dpgmg_solve calls (which = DPGMG_PROF_*; OFF
 * clears).  dpgmg_profile_read() synchronises, returns the summed device
 * time, the launch count and the algorithmic bytes per launch (stored
 * matrix entries read once), and resets the accumulators. */
int dpgmg_profile(dpgmg_handle h, dpgmg_system sys, int which);
int dpgmg_profile_read(dpgmg_handle h, dpgmg_system sys, double* total_ms, long long* launches,
                       long long* bytes_per_launch);

/* ---- allocation-free smoother ---------------------------------------------- */

/* The paper has no counterpart to this call; it serves callers that cannot let
 * a library allocate device memory: programs that give all device memory to
 * their own fixed arena or pool up front, and latency-critical loops that
 * cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * y = theta_l S_l r, the same operator as dpgmg_apply(DPGMG_OP_SMOOTH), on
 * caller-owned DEVICE buffers r_dev, y_dev (c128, n_dof of level l each).
 * `level` is 1..n_levels-1.  It allocates nothing: its only scratch (one
 * complex entry per patch slot) is a fixed array compiled into the library,
 * DPGMG_NOALLOC_MAX_SLOTS entries (64 MiB), which every GPU that loads the
 * library holds until the process exits.  A level with more patch slots is
 * rejected with DPGMG_ERR_ARG (message in dpgmg_last_error).  Every call looks
 * up the array's device address on the handle's device
 * (cudaGetSymbolAddress), so an address is never reused after the caller
 * resets the device context; the first call on a device also loads the
 * library's device code there, so make it before any stream capture on that
 * device.  Every
 * entry of the scratch that is read is written first in the same call, so
 * leftover contents of earlier calls do not matter; but all calls share the
 * one array, so calls whose work overlaps on the GPU (other handles, other
 * streams) race on it.  The work runs on the handle's stream and the call
 * returns after y is written.  Errors: ARG, CUDA. */
#define DPGMG_NOALLOC_MAX_SLOTS 4194304LL
int dpgmg_smooth_noalloc(dpgmg_handle h, dpgmg_system sys, int level, const double* r_dev, double* y_dev);

#ifdef __cplusplus
}
#endif

#endif /* DPGMG_H */
