/*
 * rbffd.h -- C ABI of the GB300 (sm_103a) implementation of the
 * semi-implicit PHS-RBF-FD incompressible Navier-Stokes method of
 * Shahane & Vanka, "A Semi-Implicit Meshless Method for Incompressible Flows
 * in Complex Geometries" (arXiv 2106.07616).
 *
 * Conventions for every call:
 *   - Return value: RBFFD_OK (0) or a negative RBFFD_E* code.  No C++
 *     exception crosses this boundary.  rbffd_last_error() gives a
 *     thread-local text for the last failure on the calling thread.
 *   - Pointers documented as "device" must point to device memory of the
 *     context's GPU; "host or device" pointers may be either (the library
 *     copies with cudaMemcpyDefault, which needs unified addressing, true on
 *     every 64-bit CUDA platform).  The caller owns every buffer it passes;
 *     the library owns what it allocates behind a handle.
 *   - Work is issued on the context's stream.  Calls that return a host
 *     value (a norm, a count, a status) synchronise that stream.
 *   - Handles are not thread-safe: serialise calls on one context.
 *   - Arrays of per-point data are indexed by point number 0..n-1; stencil
 *     arrays are row-major n x q (row i = the cloud of point i).
 */
#ifndef RBFFD_H
#define RBFFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RBFFD_OK = 0,
  RBFFD_EINVAL = -1,     /* bad argument (sizes, q < m, q > n, null pointer) */
  RBFFD_ENOMEM = -2,     /* device allocation failed, HBM budget exceeded, or host memory
                            or a host thread could not be had */
  RBFFD_ESINGULAR = -3,  /* a local collocation matrix had an exactly zero pivot */
  RBFFD_ENOCONV = -4,    /* a Krylov solve or the outer loop hit its limit */
  RBFFD_EDIVERGED = -5,  /* a non-finite value appeared */
  RBFFD_ETIMEOUT = -6,   /* a bounded device-side wait gave up */
  RBFFD_ECUDA = -7,      /* a CUDA runtime call failed */
  RBFFD_ENOTIMPL = -8
};

/* Boundary tags (paper Sec. 3.1, "Boundary Conditions").  Every non-interior
 * point has a one-sided cloud (itself and interior points only). */
enum {
  RBFFD_TAG_INTERIOR = 0,
  RBFFD_TAG_DIRICHLET = 1, /* wall / inlet: u, v prescribed (ubc, vbc); p from the normal
                              momentum equation; p' homogeneous Neumann */
  RBFFD_TAG_OUTFLOW = 2,   /* fixed-pressure outlet: p held at its current value (0 from
                              create; rbffd_set_field changes it), p' = 0, and zero normal
                              derivative of u and v; ubc, vbc are initial values only */
  RBFFD_TAG_SYMMETRY = 3   /* symmetry line: the normal velocity component prescribed
                              (ubc if the normal is along x, vbc if along y), zero normal
                              derivative of the tangential one; p from the normal momentum
                              equation; p' homogeneous Neumann.  The normal must be
                              axis-aligned (its smaller component |.| <= 1e-12). */
};

/* Operators of the problem (rbffd_apply, rbffd_get_operators). */
enum {
  RBFFD_OP_DX = 0,        /* d/dx weights */
  RBFFD_OP_DY = 1,        /* d/dy weights */
  RBFFD_OP_LAP = 2,       /* Laplacian weights */
  RBFFD_OP_PCORR = 3,     /* pressure-correction matrix */
  RBFFD_OP_MOMENTUM = 4,  /* u-momentum matrix of the last outer iteration */
  RBFFD_OP_MOMENTUM_V = 5 /* v-momentum matrix: equal to the u one except on symmetry lines */
};

/* Fields of a problem (rbffd_get_field / rbffd_set_field). */
enum {
  RBFFD_FIELD_U = 0, RBFFD_FIELD_V = 1, RBFFD_FIELD_P = 2,   /* current iterate */
  RBFFD_FIELD_UN = 3, RBFFD_FIELD_VN = 4,                     /* time level n */
  RBFFD_FIELD_UNM1 = 5, RBFFD_FIELD_VNM1 = 6,                 /* time level n-1 */
  RBFFD_FIELD_UT = 7, RBFFD_FIELD_VT = 8,                     /* u~, v~ of the last iteration */
  RBFFD_FIELD_PC = 9,                                         /* p' of the last iteration */
  RBFFD_FIELD_UBC = 10, RBFFD_FIELD_VBC = 11                  /* prescribed boundary velocity */
};

/* Arithmetic of the Krylov solves.  Every mode stops on the same FP64
 * relative residual (krylov_tol); the mixed modes run their inner iterations
 * on the FP32 pipe and correct in FP64 (defect correction). */
enum {
  RBFFD_PREC_FP64 = 0,     /* FP64 operators and Krylov vectors throughout */
  RBFFD_PREC_MIXED = 1,    /* FP32 inner BiCGSTAB inside FP64 defect correction;
                              converges while cond(A) * 6e-8 < 1 */
  RBFFD_PREC_MIXED_FF = 2  /* float-float (FP32 pairs, ~1e-14) inner BiCGSTAB inside
                              FP64 defect correction */
};

/* Preconditioner of the pressure-correction BiCGSTAB.  The paper only says
 * "preconditioned" (Sec. 3); either choice stops on the same relative
 * residual, so it changes the iteration count, not the solution. */
enum {
  RBFFD_PRECOND_JACOBI = 0, /* diagonal scaling (default) */
  RBFFD_PRECOND_AMG = 1,    /* one V-cycle of a smoothed-aggregation multigrid hierarchy;
                               two cycles per BiCGSTAB iteration, FP64 */
  RBFFD_PRECOND_AMG_FGMRES = 2 /* the same hierarchy stored in FP32, one cycle per step of
                               a flexible GMRES(30) instead of BiCGSTAB */
};
/* The hierarchy's host part is built on a thread of its own, started when
 * the problem is built (create, reload); the first call that needs it (the
 * first outer iteration or step, a batch iteration, rbffd_problem_amg_info)
 * waits for it and uploads it, and returns its errors (RBFFD_ESINGULAR for
 * a singular coarsest matrix, RBFFD_ENOMEM). */
#define RBFFD_AMG_MAX_LEVELS 10

typedef struct rbffd_ctx rbffd_ctx;
typedef struct rbffd_problem rbffd_problem;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps what
 * problems of this context may allocate (0 = no cap).  cuda_stream is a
 * cudaStream_t to issue work on, or NULL for a stream owned by the context.
 * Errors: RBFFD_EINVAL (bad device), RBFFD_ECUDA. */
int rbffd_ctx_create(rbffd_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream);
void rbffd_ctx_destroy(rbffd_ctx *ctx);
/* Text of the last failure on the calling thread ("" if none). */
const char *rbffd_last_error(void);
/* Number of kernel launches this context has issued (for accounting). */
int64_t rbffd_ctx_launch_count(const rbffd_ctx *ctx);

/* Live per-kernel timing.  While enabled, the context brackets the launches
 * of the classes below with CUDA events on its own stream (the stream the
 * kernels run on) and accumulates, per class: launches, device time, the
 * units of work processed and the algorithmic bytes (or flops) those units
 * move.  Units and bytes per unit:
 *   KRYLOV_P    (pressure-correction BiCGSTAB, 1 right-hand side):
 *               unit = one row in one iteration; bytes = 2q(s_w + s_i) + 14 s_v
 *   KRYLOV_MOM  (momentum BiCGSTAB, 2 right-hand sides sharing the matrix):
 *               unit = one row in one iteration; bytes = 2q(s_w + s_i) + 28 s_v
 *   WEIGHTS     unit = one cloud; "bytes" holds FP64 flops: 2N^3/3 + 2 N^2 (3 rhs)
 *               + the matrix build, N = q + m
 *   KNN         unit = one point; bytes = 24 (coordinates in, q indices out)
 *   OUTER       one outer iteration (whole simple_iterate, GPU time)
 * s_w, s_i, s_v: bytes of a matrix value, a column index, a vector entry
 * (8, 4, 8 in the FP64 path and for the 8-byte float-float inner values;
 * 4, 4, 4 for the FP32 inner iterations; the few FP64 residual sweeps of
 * the mixed paths are not counted as units).
 * rbffd_ctx_profile(ctx, 1) resets the counters and enables timing; 0 stops. */
enum {
  RBFFD_KSTAT_KRYLOV_P = 0,
  RBFFD_KSTAT_KRYLOV_MOM = 1,
  RBFFD_KSTAT_WEIGHTS = 2,
  RBFFD_KSTAT_KNN = 3,
  RBFFD_KSTAT_OUTER = 4,
  RBFFD_KSTAT_COUNT = 5
};
typedef struct {
  int64_t launches;
  double ms;     /* summed device time */
  double units;  /* units of work processed */
  double bytes;  /* Bound of every device-side wait (the grid exchanges and barriers of the
 * persistent Krylov kernels) of the launches this context issues from now
 * on: 2^log2_cycles SM clock cycles; 0 restores the default 2^31 (about a
 * second at 2 GHz).  A wait that runs out makes its block record a timeout
 * and leave; the other blocks leave at their next wait, and the call returns
 * RBFFD_ETIMEOUT with the solve's outputs unspecified.  Nothing is left
 * running and the context stays usable.  The paper has no counterpart: this
 * is failure handling of the library.  Errors: RBFFD_EINVAL outside 0..40. */
int rbffd_ctx_set_wait_limit(rbffd_ctx *ctx, int32_t log2_cycles);

/* algorithmic bytes (flops for WEIGHTS) */
} rbffd_kernel_stat;
int rbffd_ctx_profile(rbffd_ctx *ctx, int enable);
int rbffd_ctx_kernel_stat(const rbffd_ctx *ctx, int32_t which, rbffd_kernel_stat *out);

/* ------------------------------------------------------- S1: the clouds */

/* Cloud selection (paper Sec. 2, "a cloud of neighboring points", and
 * Sec. 3.1, one-sided clouds at boundaries).  For every point i, writes
 * idx[i*q .. i*q+q-1]: i itself first, then the q-1 nearest candidates in
 * the order (d^2, index) ascending, with d^2 = dx*dx + dy*dy evaluated in
 * FP64 without fused multiply-add (so the result is reproducible bit for
 * bit).  Candidates of a point whose tag is not RBFFD_TAG_INTERIOR are the
 * interior points only (its cloud is one-sided); tag == NULL treats all
 * points as interior.
 *   x, y: device, n doubles.  tag: device, n int8, or NULL.
 *   idx:  device, n*q int32 (output).
 * Errors: RBFFD_EINVAL if n < 1, q < 1, q > n, or a boundary point has
 * fewer than q-1 interior candidates; RBFFD_ENOMEM; RBFFD_ECUDA. */
int rbffd_build_stencils(rbffd_ctx *ctx, int32_t n, const double *x, const double *y,
                         const int8_t *tag, int32_t q, int32_t *idx);

/* Same result as rbffd_build_stencils, for callers that cannot allocate
 * device memory once they are running: a loop that must keep a fixed device
 * footprint, or an application whose other streams must not be stalled by
 * the device synchronisation that cudaMalloc / cudaFree imply.  The paper
 * has no counterpart: this is a property of the library, not of the method.
 * It allocates nothing.  The cell-grid workspace comes from a fixed array of
 * RBFFD_STATIC_SCRATCH_BYTES in device global memory inside the library,
 * which every GPU that loads the library holds until the process exits.
 *   - n is limited to RBFFD_STATIC_MAX_POINTS; larger n returns RBFFD_EINVAL
 *     with a message, before anything runs on the GPU.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, once per device even
 *     when several host threads make their first call together.
 *   - Like rbffd_build_stencils, every call synchronises the context's
 *     stream (it reads the kernels' error word back to the host), so it must
 *     not be called while that stream is being captured into a CUDA graph.
 *   - All calls share the one array and it keeps the last call's contents
 *     (the call clears what it needs cleared).  Calls that overlap on the GPU
 *     -- from two streams, or two contexts on one device -- race on it: issue
 *     them on one stream or serialise them.
 * Arguments, layout and other errors are those of rbffd_build_stencils. */
#define RBFFD_STATIC_MAX_POINTS 262144
#define RBFFD_STATIC_SCRATCH_BYTES (4u << 20)
int rbffd_build_stencils_static(rbffd_ctx *ctx, int32_t n, const double *x, const double *y,
                                const int8_t *tag, int32_t q, int32_t *idx);

/* -------------------------------------------------- S2: operator weights */

/* PHS-RBF-FD weights (paper Sec. 2, Eqs. RBF_interp .. RBF_interp_mat_vec_L_solve):
 * phi(r) = r^3 with the m = (k+1)(k+2)/2 monomials of degree <= k appended.
 * For cloud i, with local coordinates xi = (x - x_i)/h, h = max distance
 * in the cloud, the collocation system A c = [L phi(|x_i - x_j|)]_j ++
 * [L P(x_i)] (A = [Phi P; P^T 0], symmetric) is solved by LU with partial
 * pivoting in FP64, and the first q entries of c, rescaled by 1/h (d/dx,
 * d/dy) or 1/h^2 (Laplacian), are the weights B1 of the cloud.
 *   idx: device n*q int32 (from rbffd_build_stencils).
 *   wx, wy, wl: device n*q doubles (outputs; any may be NULL to skip).
 *   first_singular: host int32 (nullable): lowest point index whose matrix
 *   had an exactly zero pivot, or -1.
 * Errors: RBFFD_EINVAL (q < m, q + m > 96, degree < 0, degree > 8),
 * RBFFD_ESINGULAR (weights of those clouds are set to 0), RBFFD_ECUDA. */
int rbffd_weights(rbffd_ctx *ctx, int32_t n, const double *x, const double *y, int32_t q,
                  const int32_t *idx, int32_t degree, double *wx, double *wy, double *wl,
                  int32_t *first_singular);

/* ------------------------------------------------------- flow problems */

typedef struct {
  int32_t n;       /* points */
  int32_t q;       /* cloud size */
  int32_t degree;  /* appended polynomial degree k */
  int32_t pin;     /* Dirichlet or symmetry point whose p' row is the identity
                      (fixes the free constant of a pure-Neumann p' equation), or
                      -1 when an outflow point fixes the level */
  double rho, mu;  /* density, dynamic viscosity */
  int32_t precision; /* RBFFD_PREC_* */
  /* host or device arrays of n entries (copied at create / reload): */
  const double *x, *y;
  const int8_t *tag;     /* RBFFD_TAG_* */
  const double *nx, *ny; /* outward unit normal at boundary points (0 inside) */
  const double *ubc, *vbc; /* prescribed velocity at boundary points */
  int32_t precond;         /* RBFFD_PRECOND_* of the p' solve */
  double period[2];        /* periods of x and y, 0 for a bounded axis (Sec. 3.1,
                              periodic boundaries): clouds near one side take points
                              from the other, at their nearest periodic image.  Put
                              no boundary points on a periodic side; a period must
                              exceed twice any cloud's radius */
  double force[2];         /* body force per unit volume added to the momentum
                              equations (the paper's mean pressure gradient that
                              drives a periodic flow); 0 for none */
} rbffd_problem_desc;

/* Allocate a problem and build everything that depends only on the points
 * (S1 clouds, S2 weights, S3 packed operators, the pressure-correction
 * matrix: Laplacian rows inside, n . grad rows at Dirichlet and symmetry
 * points, identity at outflow points and at `pin`).  Initial state:
 * u = v = p = 0 in the interior, ubc / vbc on the boundary, flat time
 * history.  Errors: RBFFD_EINVAL (also: an unknown tag, an oblique symmetry
 * normal, pin not a Dirichlet / symmetry point, pin = -1 without an outflow
 * point), RBFFD_ENOMEM (allocation or budget), RBFFD_ESINGULAR, RBFFD_ECUDA. */
int rbffd_problem_create(rbffd_ctx *ctx, const rbffd_problem_desc *desc, rbffd_problem **out);
/* Same as create for a problem of identical n, q, degree and precision,
 * reusing its memory (no allocation): re-copies the inputs, rebuilds the
 * clouds, weights and operators, and resets the state. */
int rbffd_problem_reload(rbffd_problem *prob, const rbffd_problem_desc *desc);
void rbffd_problem_destroy(rbffd_problem *prob);
/* Device bytes held by the problem. */
size_t rbffd_problem_bytes(const rbffd_problem *prob);
/* Multigrid hierarchy of the p' preconditioner: *levels (0 with Jacobi),
 * rows and nonzeros per level (arrays of RBFFD_AMG_MAX_LEVELS, nullable)
 * and the host time its build took (nullable): the copy of the p' matrix,
 * the hierarchy and its staging, from the moment the matrix is ready (not
 * the upload).  Finishes a build still running first. */
int rbffd_problem_amg_info(const rbffd_problem *prob, int32_t *levels, int32_t *rows,
                           int64_t *nnz, double *setup_ms);
/* The same hierarchy built on the host only, for a CSR matrix (host arrays:
 * rowptr[n+1], col and val[rowptr[n]]); no device work.  Errors:
 * RBFFD_EINVAL, RBFFD_ESINGULAR (singular coarsest matrix), RBFFD_ENOTIMPL
 * (coarsening stalled above 600 rows). */
int rbffd_amg_analyze(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                      int32_t *levels, int32_t *rows, int64_t *nnz, double *setup_ms);

/* The composed V-cycle (the library's own regrouping of the cycle above; no
 * counterpart in the paper, whose preconditioner is unspecified).  The
 * smoothing-folded V-cycle is one linear map of its right-hand side: below
 * level 1, every deeper right-hand side is b_l = Rh_l b_1 with Rh_l the
 * restriction straight from level 1, and the corrections of all deeper
 * levels prolong to level 1 at once through Q = [Q_2 | Q_3 | ...].  The
 * launches whose shared memory holds the stacked coarse vector (levels 2 to
 * L-1, nc entries) run the cycle in four dependent phases instead of
 * 2 L - 1, the others level by level; both give the same result up to
 * rounding.  Built for hierarchies of three or more levels. */
/* Whether hierarchies built on this context from now on get the composed
 * cycle (on != 0: yes, the default).  Errors: RBFFD_EINVAL. */
int rbffd_ctx_set_amg_compose(rbffd_ctx *ctx, int on);
/* The problem's composed cycle (finishes a build still running first):
 * *coarse_entries (nc; 0: not built), *chunks of its stacked restriction,
 * *restrict_nnz and *q_nnz its entries, *device_level0 1 when level 0 of
 * the hierarchy was built on the device (all nullable).  Zeros with Jacobi.
 * Errors: RBFFD_EINVAL, the hierarchy build's errors. */
int rbffd_problem_amg_cycle(const rbffd_problem *prob, int32_t *coarse_entries, int32_t *chunks,
                            int64_t *restrict_nnz, int64_t *q_nnz, int32_t *device_level0);
/* Where level 0 of the multigrid hierarchies built on this context from now
 * on is built (the library's own setup path).  on != 0 (the default): on
 * the device for p' matrices of 16384 rows or more -- the strength graph,
 * the aggregation, the prolongation and the products R (A P), A P and
 * A^T P by rows, synchronous with the build -- so that the host thread
 * only builds the coarse levels; off, or where the device build does not
 * apply (more than 64 neighbours, a product row with more than 96 distinct
 * columns), the whole hierarchy on the host.  Level 0 is aggregated the
 * same way in both (a distance-2 maximal independent set of roots with
 * fixed priorities), so both give the same aggregates.  Errors:
 * RBFFD_EINVAL. */
int rbffd_ctx_set_amg_device_setup(rbffd_ctx *ctx, int on);
/* Orthogonalisation of the flexible GMRES Arnoldi process for solves issued
 * on this context from now on (the library's own choice): mode 1 (the
 * default), classical Gram-Schmidt with one reorthogonalisation, two
 * reductions a step; 0, one classical pass with the new norm by Pythagoras
 * (h_{j+1,j}^2 = |w|^2 - sum h_{ij}^2), one reduction and one grid exchange
 * fewer a step; 2, two passes with the second delayed to the next step
 * (DCGS2, Bielich et al. 2022): one reduction a step, every basis vector
 * still orthogonalised twice, a restart's last column completed by one more
 * reduction.  Either way a solve stops on its FP64 true residual.
 * Errors: RBFFD_EINVAL (mode outside 0..2). */
int rbffd_ctx_set_fgmres_reorth(rbffd_ctx *ctx, int mode);
/* One cycle of the hierarchy of a CSR matrix (host arrays as in
 * rbffd_amg_analyze) applied to b[n] on the host in FP64, level by level
 * into out_levels[n] and composed into out_composed[n] (zeros when the
 * composed cycle is not built for this matrix); *coarse_entries and
 * *chunks as above (nullable).  No device work.  Errors: RBFFD_EINVAL, the
 * build's errors. */
int rbffd_amg_cycle_host(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                         const double *b, double *out_levels, double *out_composed,
                         int32_t *coarse_entries, int32_t *chunks);
/* Level 0's aggregates of the hierarchy of a CSR matrix (host arrays as in
 * rbffd_amg_analyze), on the host: agg[n] receives each row's aggregate,
 * *naggs their number.  The aggregation: strength |a_ij| >= 0.08 max_k
 * |a_ik| (k != i), symmetrised; a distance-2 maximal independent set of
 * roots with fixed priorities key(i) = (h(i) 2^32 | i) + 1, h the 32-bit
 * finaliser of MurmurHash3; points next to roots join the root of largest
 * key, the rest the first-pass neighbour of largest key, isolated points
 * become singletons after the roots (index order).  The device build gives
 * the same aggregates.  No device work.  Errors: RBFFD_EINVAL. */
int rbffd_amg_aggregates_host(int32_t n, const int32_t *rowptr, const int32_t *col,
                              const double *val, int32_t *agg, int32_t *naggs);

typedef struct {
  double dt;             /* time step */
  double alpha[3];       /* BDF2: 1.5, -2, 0.5 (paper Sec. 3) */
  double krylov_tol;     /* FP64 relative residual of each Krylov solve */
  int32_t krylov_maxit;  /* iteration cap of each Krylov solve */
  /* RBFFD_PREC_MIXED only (0 = default): relative reduction asked of each
     FP32 inner solve (default 1e-3) and its iteration cap (default 4000) */
  double inner_tol;
  int32_t inner_maxit;
} rbffd_step_params;

typedef struct {
  int32_t iters[3];   /* BiCGSTAB iterations: u~, v~, p' (inner FP32 ones if mixed) */
  double relres[3];   /* final FP64 relative residuals */
  int32_t sweeps[3];  /* restarts: defect-correction sweeps (mixed precision), BiCGSTAB
                       * restarts after a (near) breakdown, FGMRES restarts */
} rbffd_iter_stats;

/* One outer iteration (paper Sec. 3.2 steps 2-7):
 *   2. momentum predictor, Eqs. (u:tilde), (v:tilde): advection linearised
 *      with the current iterate, diffusion implicit, grad p at the current
 *      iterate; identity rows with the boundary velocity at Dirichlet
 *      points; right-Jacobi BiCGSTAB for u~ and v~ (one matrix, two
 *      right-hand sides, initial guess u^r, v^r);
 *   3. pressure correction, Eq. (pressure poisson), right-Jacobi BiCGSTAB
 *      from p' = 0;
 *   4. p += p' at interior points, Eq. (p:correction);
 *   5. boundary pressure from the normal momentum equation, Eq. (normal
 *      momentum), with convection and diffusion of (u~, v~) and the BDF2
 *      time derivative of the boundary velocity;
 *   6. velocity correction, Eqs. (u:correction), (v:correction), at
 *      interior points;
 *   7. delta_out (host) = mean|u^{r+1} - u^r| + mean|v^{r+1} - v^r|.
 * stats (host, nullable).  Errors: RBFFD_ENOCONV (a Krylov solve hit its
 * cap), RBFFD_EDIVERGED, RBFFD_ETIMEOUT, RBFFD_ECUDA. */
int simple_iterate(rbffd_problem *prob, const rbffd_step_params *params, double *delta_out,
                   rbffd_iter_stats *stats);

typedef struct {
  double dt;
  double resid_tol;       /* steady: stop when R <= resid_tol */
  int32_t max_steps;      /* steady: cap on time steps */
  int32_t max_outer;      /* cap on outer iterations per time step */
  double krylov_tol;
  int32_t krylov_maxit;
  double inner_tol;       /* as in rbffd_step_params */
  int32_t inner_maxit;
  int32_t criterion;      /* steady stop: 0 = R <= resid_tol; 1 = the paper's steady
                             error (Sec. 4.1): (mean|u^{n+1}-u^n| + mean|v^{n+1}-v^n|)/dt
                             <= resid_tol; 2 = exactly max_steps steps (no steady
                             test; the solve ends with RBFFD_OK) */
} rbffd_solve_params;

typedef struct {
  int32_t steps;
  int64_t outer_iters;
  int64_t krylov_iters[3]; /* totals: u~, v~, p' */
  double resid[4];         /* R_m, R_c, R, lambda of the final state (steady only;
                              rbffd_steady_residual) */
  double change;           /* mean|u^{n+1}-u^n| + mean|v^{n+1}-v^n| of the last step */
} rbffd_solve_stats;

/* One BDF2 time step (paper Sec. 3.2 steps 1-8): outer iterations from the
 * state of level n until delta < tol_outer or max_outer, then
 * [u^{n-1}, u^n] <- [u^n, u^{n+1}].  outer_iters, change: host, nullable. */
int rbffd_time_step(rbffd_problem *prob, const rbffd_solve_params *params, double tol_outer,
                    int32_t *outer_iters, double *change);

/* Steady solve by BDF2 pseudo-time marching from the current state.  Outer
 * tolerance 1e-4 for the first step, then min(1e-4, dt * eps_s) with
 * dt * eps_s = the change of the previous step (paper Sec. 3.2).  Stops when
 * R = max(R_m, R_c) <= resid_tol (rbffd_steady_residual), or with
 * criterion 1 when the paper's steady error change/dt <= resid_tol.
 * Errors: RBFFD_ENOCONV if max_steps ran out first. */
int solve_steady(rbffd_problem *prob, const rbffd_solve_params *params, rbffd_solve_stats *stats);

/* n_steps BDF2 steps with the same adaptive outer tolerance.  on_step
 * (nullable) runs on the host after every step; a non-zero return stops
 * the march and is returned. */
int solve_unsteady(rbffd_problem *prob, const rbffd_solve_params *params, int32_t n_steps,
                   int (*on_step)(void *user, int32_t step, double t), void *user,
                   rbffd_solve_stats *stats);

/* Relative residual of the discrete steady equations over interior rows,
 * vector norms over both components:
 *   R_m = |rho (u.grad)u - mu lap u + grad p - f| / (|rho (u.grad)u| + |mu lap u|
 *         + |grad p| + |f|)
 *   d   = Dx u + Dy v at interior rows, lambda = its mean
 *   R_c = |d - lambda| / |grad u| for a pinned problem (no outlet), else
 *         |d| / |grad u|.
 * Why lambda is taken out: with Neumann rows only, the p' equation (paper
 * Sec. 3, Eq. pressure poisson; Sec. 3.1) is singular and solvable only for
 * a compatible right-hand side; the library solves it for the compatible
 * part of (rho a1/dt) div u~, so the part of the divergence that no
 * pressure correction can remove is a constant over the interior rows, and
 * a steady state satisfies continuity up to that constant lambda (a
 * discretisation defect that falls with the point spacing).
 * R4 (host, 4 doubles) = R_m, R_c, R = max(R_m, R_c), lambda. */
int rbffd_steady_residual(rbffd_problem *prob, double *R4);

/* Courant number of the explicit-Euler stability bound quoted in the paper
 * (Sec. 3.2, after the solution steps): lambda * dt / 2, with lambda the
 * spectral radius of the discrete convection-diffusion operator
 * rho (u Dx + v Dy) - mu Lap (interior rows) at the current velocity.
 * lambda: power iteration from a fixed start vector, `iters` steps (>= 2;
 * 200 is typical), geometric mean of the growth over the second half.
 * Outputs nullable.  The time step for a target Courant number Co is
 * 2 Co / lambda. */
int rbffd_courant(rbffd_problem *prob, double dt, int32_t iters, double *lambda_out,
                  double *courant_out);

/* Copy a field (RBFFD_FIELD_*) out of / into the problem; n doubles, host
 * or device.  Setting U, V or P leaves the time history untouched. */
int rbffd_get_field(rbffd_problem *prob, int32_t which, double *out);
int rbffd_set_field(rbffd_problem *prob, int32_t which, const double *in);

/* Stencil indices and weights, row-major n*q, host or device (any NULL). */
int rbffd_get_operators(rbffd_problem *prob, int32_t *idx, double *wx, double *wy, double *wl,
                        double *pcorr);

/* y = W x for one operator (RBFFD_OP_*); x, y: device, n doubles. */
int rbffd_apply(rbffd_problem *prob, int32_t which, const double *x, double *y);

/* ------------------------------------------------------------- batches */

/* Many independent problems advanced together (the batched workloads; the
 * paper has one problem at a time).  Every call runs one outer iteration
 * (the same steps as simple_iterate) for each active member: the row kernels
 * per member, and the two Krylov solves of all members in one cooperative
 * launch each, in which every member owns consecutive CTAs and synchronises
 * only with them (one launch per solver: FP64, FP32-in-FP64 and
 * float-float-in-FP64 momentum BiCGSTAB; Jacobi BiCGSTAB, multigrid
 * BiCGSTAB and flexible GMRES for p').  Members must be problems of the
 * batch's context -- mixed-precision ones with a multigrid p' solver -- and
 * stay owned by the caller (destroy the batch first).  A member
 * solved in a batch matches the same member solved alone to the Krylov
 * tolerance (the sums are ordered differently, the fixed point is not). */
typedef struct rbffd_batch rbffd_batch;
int rbffd_batch_create(rbffd_ctx *ctx, int32_t count, rbffd_problem *const *members,
                       rbffd_batch **out);
void rbffd_batch_destroy(rbffd_batch *batch);
/* dt: host double[count] (nullable): each member's time step in place of
 * params->dt.  active: host int32[count] (nullable = all); deltas: host double[count];
 * stats: host rbffd_iter_stats[count] (nullable); status: host int32[count]
 * (nullable).  With status, a member whose solve failed reports its code
 * there and the call returns RBFFD_OK; without it the first failure is
 * returned.  Entries of inactive members are left untouched.  Errors:
 * RBFFD_EINVAL if more members are active than one launch holds CTAs
 * (several hundred on a GB300), RBFFD_ECUDA. */
int rbffd_batch_iterate(rbffd_batch *batch, const rbffd_step_params *params, const double *dt,
                        const int32_t *active, double *deltas, rbffd_iter_stats *stats,
                        int32_t *status);
/* The batched outer iteration is captured as a CUDA graph the second time it
 * runs in a row for the same active members, builds and step parameters
 * (the first runs directly), and replayed while those stay the same (live
 * kernel timing, rbffd_ctx_profile, launches it directly).  captures / replays / kernels (nullable host
 * outputs): graphs captured and replayed so far, and the kernels one replay
 * launches (0 when capture is off).  Errors: RBFFD_EINVAL (null batch). */
int rbffd_batch_graph_stats(const rbffd_batch *batch, int64_t *captures, int64_t *replays,
                            int64_t *kernels);

/* Launch-shape autotuner of the batched Krylov launches (the library's own
 * tuning; the paper solves one problem at a time).  Each launch runs as a
 * persistent work list: teams of CTAs, each solving its share of the
 * members one after another, the team size planned from the members' work
 * (rows x last iteration count).  The first nine iterations of a batch run
 * directly: one untimed at the planned team size, then eight with it
 * scaled by 1, 2, 1/2, 4, 4, 1/2, 2, 1 (threads per row follow from it);
 * each launch is timed with CUDA events and its time divided by the work
 * it did; every launch slot then keeps the scale of least average cost.  The nine slots: momentum with u~ and v~ as two right-hand sides,
 * momentum as single-RHS systems (members with symmetry lines), p' Jacobi
 * BiCGSTAB, p' multigrid BiCGSTAB, p' flexible GMRES, and the
 * mixed-precision momentum launches (FP32 two-RHS/single, float-float
 * two-RHS/single).  tuned (nullable): 1 once done.  scales
 * (nullable, 9): the current scale per slot.  cost (nullable, 9 x 4, slot
 * major): ms per row-iteration of each candidate, the mean of its two
 * timings (0: slot unused).
 * Errors: RBFFD_EINVAL (null batch). */
int rbffd_batch_tuning(const rbffd_batch *batch, int32_t *tuned, double *scales, double *cost);

/* Switches the work-list autotuner on (on != 0, the default: it starts over
 * at the batch's next iteration) or off (every slot keeps the planned team
 * size, scale 1).  Either way the tuning state is cleared.  Results do not
 * depend on it beyond the order of partial sums.  Errors: RBFFD_EINVAL. */
int rbffd_batch_set_autotune(rbffd_batch *batch, int on);
/* The batched launches' work-list planner on its own (host only, no device
 * work; the library's own scheduling).  m solves with work[i] (rows x
 * iterations), cap[i] (most CTAs the solve's partial sums allow) and
 * rows[i]; cmax co-resident CTAs; scale: the autotuner's team-size factor
 * (1 = as planned).  The CTAs form *nteams teams of *team_size (the team
 * gives the largest solve its share of the grid, at most every cap[i], at
 * least enough CTAs for 8 threads a row of the smallest solve when the grid
 * has room); the solves, largest work first, each go to the least-loaded
 * team (LPT).  member_team[m] (host) receives each solve's team;
 * *nctas = *nteams x *team_size (all three nullable).  Errors:
 * RBFFD_EINVAL. */
int rbffd_plan_work_lists(int32_t m, const double *work, const int32_t *cap, const int32_t *rows,
                          int32_t cmax, double scale, int32_t *nctas, int32_t *team_size,
                          int32_t *nteams, int32_t *member_team);

/* -------------------------------------------------------------- serving */

/* A request server with continuous batching (the serving workload; the
 * paper solves one problem at a time).  Requests are steady solves
 * (solve_steady semantics; FP64 or, with a multigrid p' solver,
 * mixed-precision momentum), submitted from any thread.  A
 * worker thread owns the context's stream (give the server a context of its
 * own) and loops: admit queued requests while the context's HBM budget
 * allows (a request is admitted by building its problem; one that does not
 * fit waits for running requests to finish), run one outer iteration of
 * every running request together (as rbffd_batch_iterate), apply each
 * request's time-step logic and steady-residual test, and retire finished
 * requests with their fields copied to host memory.  Requests join and
 * leave at outer-iteration boundaries. */
typedef struct rbffd_server rbffd_server;
typedef struct {
  size_t hbm_budget_bytes; /* admission budget (0: 80% of the free HBM at create) */
  int32_t max_active;      /* cap on running requests (0: what one launch holds) */
} rbffd_server_params;
typedef struct {
  int32_t state;        /* 0 queued, 1 running, 2 done */
  int32_t status;       /* when done: RBFFD_OK, or the error that ended it */
  double queue_s;       /* arrival -> admission (seconds; 0 if never admitted) */
  double latency_s;     /* arrival -> result (seconds), when done */
  int32_t steps;        /* time steps taken */
  int64_t outer_iters;  /* outer iterations taken */
  double resid[4];      /* R_m, R_c, R, lambda at the last step */
  int32_t admit_attempts; /* admission tries that built or finished the request's
                             multigrid hierarchy (1 unless device memory was short:
                             the problem is built once and only the hierarchy's
                             upload is retried) */
  double arrive_s, admit_s, done_s; /* submission, admission and completion, in
                                       seconds since the server was created */
  int32_t builds;       /* builds of the request's problem (clouds, weights, operators):
                           1, or more only when a build itself found no device memory */
} rbffd_result;
int rbffd_server_create(rbffd_ctx *ctx, const rbffd_server_params *params, rbffd_server **out);
/* desc arrays are host pointers, copied before the call returns; ticket
 * (host) identifies the request.  Errors: RBFFD_EINVAL. */
int rbffd_server_submit(rbffd_server *server, const rbffd_problem_desc *desc,
                        const rbffd_solve_params *params, uint64_t *ticket);
/* Thread-safe.  result: host.  u, v, p: host double[n] (nullable), filled
 * when the request is done with status RBFFD_OK. */
int rbffd_server_poll(rbffd_server *server, uint64_t ticket, rbffd_result *result, double *u,
                      double *v, double *p);
/* Block until every submitted request is done. */
int rbffd_server_drain(rbffd_server *server);
/* Finishes the submitted requests, then stops the worker and frees all. */
void rbffd_server_destroy(rbffd_server *server);

#ifdef __cplusplus
}
#endif
#endif /* RBFFD_H */
