/*
 * gcmg -- global-coarsening matrix-free multigrid on one GPU (sm_103a).
 *
 * C ABI of libgcmg.so.  It solves the Poisson problem -Lap u = f on the cube
 * [lo, hi]^3 with homogeneous Dirichlet values, discretised by continuous
 * Q_k elements (k = 1..4, Gauss-Lobatto support points, (k+1)^3 Gauss
 * points per cell) on an octree mesh with hanging nodes, the set-up of Sec. 5
 * of Munch, Heister, Prieto Saavedra & Kronbichler, "Efficient distributed
 * matrix-free multigrid methods on locally refined meshes for FEM
 * computations" (arXiv:2203.12292).
 *
 * Conventions for every entry point:
 * - Return value: GCMG_OK (0) or a positive GCMG_ERR_* code; the message of
 *   the last failure of the calling thread is gcmg_last_error().  No C++
 *   exception crosses this interface.
 * - Vectors: "device" pointers are CUDA device memory owned by the caller,
 *   length n_free(level) of the level they belong to, in fp64 (double) or
 *   fp32 (float) as the `fp64` flag says.  They hold the free DoFs only:
 *   Dirichlet and hanging-node (constrained) values are not stored.  The
 *   numbering is the library's; gcmg_level_dof_coords gives the support
 *   point of every entry.
 * - Work is queued on the handle's CUDA stream (gcmg_setup / gcmg_set_stream);
 *   calls return without synchronising unless stated otherwise.
 * - Handles own all set-up data; the caller destroys them.  A handle must
 *   not be used from two threads at the same time.
 */
#ifndef GCMG_H
#define GCMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GCMG_OK 0
#define GCMG_ERR_ARG 1           /* invalid argument (level, size, null pointer, degree) */
#define GCMG_ERR_CUDA 2          /* a CUDA call failed */
#define GCMG_ERR_OOM 3           /* device or host allocation failed */
#define GCMG_ERR_NOT_CONVERGED 4 /* CG reached maxit before the tolerance */
#define GCMG_ERR_BREAKDOWN 5     /* CG breakdown: (p, Ap) <= 0 or a NaN */
#define GCMG_ERR_INTERNAL 6      /* inconsistent mesh or set-up data */

/* refinement predicates of one refinement step (Sec. 4, "Examples") */
#define GCMG_PRED_ALL 0            /* every leaf */
#define GCMG_PRED_OCTANT_CENTRE 1  /* leaf centre in the closed box [a, b]^3 */
#define GCMG_PRED_SPHERE 2         /* leaf box meets the sphere |x - (a,a,a)| = b */
#define GCMG_PRED_SHELL 3          /* a <= |leaf centre| <= b */
#define GCMG_PRED_OCTANT_STRICT 4  /* all vertex coordinates in [a, b) */

typedef struct gcmg_mesh gcmg_mesh;
typedef struct gcmg_handle gcmg_handle;

typedef struct {
  int pred;
  double a, b, c, d;
} gcmg_refine_step;

/*
 * Octree mesh from one cell [lo, hi]^3 refined step by step; every step is
 * completed by the closure that keeps leaves sharing a vertex within one
 * level (Sec. 4, "Examples").  The global-coarsening hierarchy (Sec. 2.2:
 * all cells coarsened at once, repeated down to one cell) is built here.
 * `steps` is a host array of n_steps entries, read during the call only.
 */
int gcmg_mesh_create(double lo, double hi, int n_steps, const gcmg_refine_step* steps, gcmg_mesh** out);
void gcmg_mesh_destroy(gcmg_mesh* mesh);
/* number of global-coarsening levels (level 0 = one cell) */
int gcmg_mesh_num_levels(const gcmg_mesh* mesh, int* n);
/* number of cells of a global-coarsening level */
int gcmg_mesh_level_cells(const gcmg_mesh* mesh, int level, int64_t* n_cells);
/*
 * Host-only DoF numbering of a global-coarsening level for degree k (no GPU
 * needed): *n_free receives the number of free DoFs; if xyz is not NULL it
 * receives their support points (3 * n_free doubles, x y z per DoF) in the
 * library's numbering, the same as gcmg_level_dof_coords of a handle set up
 * with the same mesh, degree and tile_cells (0 = default).
 */
int gcmg_mesh_dof_coords(const gcmg_mesh* mesh, int level, int degree, int tile_cells, int64_t* n_free, double* xyz);
/*
 * Host-only check of the tile data of a level (what the kernels rely on):
 * tiles and owned DoF ranges partition cells and DoFs, tile-local indices
 * stay in range and map to the right DoFs, no two cells of one sub-colour
 * and no two tiles of one colour share a DoF, every foreign DoF is owned by
 * a tile of a lower colour, every DoF has exactly one transfer owner.
 * Returns GCMG_OK or GCMG_ERR_INTERNAL with the failed invariant.
 */
int gcmg_mesh_check_level(const gcmg_mesh* mesh, int level, int degree, int tile_cells);

typedef struct {
  int degree;              /* polynomial degree k of the finest level, 1..4 */
  int p_coarsening;        /* 1: k -> floor(k/2) -> ... -> 1 on the finest mesh
                              (Sec. 2.3), then geometric levels with k = 1 */
  int mg_fp32;             /* 1: levels and V-cycle in fp32, 0: fp64 (Sec. 5) */
  int cheb_degree;         /* Chebyshev degree (Sec. 3.3; 3 in Sec. 5) */
  double smoothing_range;  /* lambda_min = lambda_max / range */
  int eig_steps;           /* CG steps of the lambda_max estimate */
  double eig_safety;       /* lambda_max = safety * estimate */
  int tile_cells;          /* cells per tile on large levels, 0 = default (32);
                              levels with fewer than 2 * 152 tiles of that
                              size use halved tiles (down to 8 cells) */
  int cell_kernel;         /* operator kernel: 0 = default (one lane per cell
                              on levels with 32-cell tiles, fp32 and fp64;
                              else line-parallel), 1 = line-parallel (one
                              thread per 1D line of a cell), 2 = slab threads
                              (fp32, k+1 threads per cell, z-slabs in
                              registers; tiles <= 64 cells), 3 = one lane per
                              cell on every level with tiles of <= 32 cells */
  int cell_threads;        /* threads per CTA of the line-parallel fp32 operator:
                              0 = default (256), 128, 256, 384 or 512 */
  int local_smoothing;     /* 1: geometric local smoothing instead of global
                              coarsening (Sec. 2.1, the paper's comparison
                              variant): levels 0..L are the refinement levels
                              (every cell of level l), smoothing on the
                              interior DoFs with the refinement-edge terms of
                              Algorithm 2, copy to/from every active level
                              (Algorithm 1); the handle's last level is then
                              the active mesh (CG operator, right-hand side),
                              not a multigrid level.  Requires
                              p_coarsening = 0; not combinable with the learned
                              smoother, a coefficient or the batch. */
  int transfer_chunk;      /* coarse cells per chunk of the restriction kernel:
                              0 = default (4 on levels whose coarse side has
                              more than 4 tiles per SM, 8 on smaller ones),
                              4 or 8 = that size on every level (the same
                              operator; a test knob for the 4-cell variant
                              on small meshes) */
} gcmg_config;

int gcmg_config_default(gcmg_config* cfg);

/*
 * Set up all levels on the current CUDA device: DoF numbering, tiles and
 * colours, transfer data, Jacobi diagonals (Eqs. 3-4), lambda_max estimates,
 * the inverse of the level-0 matrix.  `stream` is a cudaStream_t (NULL =
 * legacy default stream).  Synchronises the stream before returning.
 */
int gcmg_setup(const gcmg_mesh* mesh, const gcmg_config* cfg, void* stream, gcmg_handle** out);
void gcmg_destroy(gcmg_handle* h);
int gcmg_set_stream(gcmg_handle* h, void* stream);

typedef struct {
  int64_t n_free;    /* DoFs stored in vectors of this level */
  int64_t n_cells;
  int degree;
  int n_tiles;
  int tile_cells;
  int max_local;     /* largest tile-local DoF count */
  int fp32;          /* level vectors of the V-cycle are fp32 */
  int64_t n_halo;    /* DoFs that receive contributions from more than one tile */
} gcmg_level_info;

int gcmg_num_levels(const gcmg_handle* h, int* n);
int gcmg_get_level_info(const gcmg_handle* h, int level, gcmg_level_info* info);
/* support point (x, y, z) of every free DoF of a level into a host array of
 * 3 * n_free doubles (synchronous) */
int gcmg_level_dof_coords(const gcmg_handle* h, int level, double* xyz);
/* local smoothing: the DoFs of a refinement level on its refinement edges
 * (Sec. 2.1: support points on the boundary of the region the level's cells
 * cover, inside the domain; the smoother keeps them fixed).  *n receives
 * their number (0 for global coarsening); if idx is not NULL it receives
 * the increasing DoF indices (host array of *n entries, synchronous). */
int gcmg_level_edge_dofs(const gcmg_handle* h, int level, int64_t* n, int32_t* idx);

/*
 * dst = A_level src, the matrix-free operator of Eq. 2 (Laplace, constraints
 * applied while gathering and scattering).  src, dst: device, n_free(level),
 * distinct.  fp64 selects double or float arithmetic and storage.
 */
int gcmg_vmult(gcmg_handle* h, int level, int fp64, const void* src, void* dst);
/* fp64 diagonal of A_level (Eqs. 3-4) into device memory */
int gcmg_diagonal(gcmg_handle* h, int level, double* dst);
/*
 * b = C^T F on the finest level, F_i = (f, phi_i) by Gauss quadrature, with
 * f = amp * sum_m cos(2 pi kappa_m . x + phi_m) (n_modes > 0; `modes` is a
 * host array kappa_x, kappa_y, kappa_z, phi per mode) or f = 1 (n_modes = 0).
 */
int gcmg_rhs(gcmg_handle* h, int n_modes, const double* modes, double amp, double* b);

/*
 * Inhomogeneous Dirichlet data (Sec. 3.1: constraints x_i = sum_j c_ij x_j
 * + b_i with b_i != 0) for a manufactured solution u: Dirichlet data g = u
 * on the domain boundary and f = -Lap u.  The known values are moved to the
 * right-hand side,
 *     b = C^T (F - A_all u_g),
 * u_g the lifting (u at boundary support points, the interpolated boundary
 * values at hanging support points, zero at free ones); the solution at the
 * free DoFs then approximates u there.  b: device, n_free(finest), fp64.
 *   kind GCMG_FUNC_GAUSSIAN:   n = 1, params = {alpha, x0, y0, z0}:
 *       u = (alpha sqrt(2 pi))^-3 exp(-|x - x0|^2 / alpha^2)   (Table A.1,
 *       with the squared distance of a Gaussian)
 *   kind GCMG_FUNC_POLYNOMIAL: n = 1..64 terms, params = n x {c, a, b, e}:
 *       u = sum c x^a y^b z^e, integer exponents 0..16
 * params is a host array.  Two cell loops: the quadrature of f, then the
 * lifting term (u_g built per cell from geometry, C_e applied in place, the
 * cell operator, C_e^T).  GCMG_ERR_ARG for an unknown kind or bad params.
 */
#define GCMG_FUNC_GAUSSIAN 2
#define GCMG_FUNC_POLYNOMIAL 3
int gcmg_rhs_dirichlet(gcmg_handle* h, int kind, int n, const double* params, double* b);

/*
 * Variable coefficient: the operator becomes -div(nu grad u) with nu
 * constant on every cell, element matrix nu_e h_e A_ref (the set-up of the
 * Stokes application, Sec. 7: nu at the quadrature points of the finest
 * level, harmonically averaged per cell, carried to the coarser levels by
 * the transfer, `interpolate_to_mg` of Sec. 3.5).
 *   values_per_cell = (k+1)^3: nu holds n_cells(finest) x (k+1)^3 values at
 *     the Gauss points of gcmg_quadrature_points (cell order of
 *     gcmg_level_cells, x fastest); nu_e = (sum_q w_q) / (sum_q w_q / nu_q);
 *   values_per_cell = 1: nu holds nu_e per finest cell.
 * Coarser levels: an unrefined cell keeps its value, a refined one takes the
 * mean of its eight children; levels of one mesh share them.  Then the
 * Jacobi diagonals, the coarse inverse and the Chebyshev eigenvalue
 * estimates are recomputed (synchronous; graphs are re-captured).  nu:
 * device, fp64; values must be positive and finite (GCMG_ERR_ARG otherwise,
 * the handle unchanged).  Not combinable with the learned smoother.
 */
int gcmg_set_coefficient(gcmg_handle* h, int values_per_cell, const double* nu);
/*
 * Non-Cartesian geometry (the general form of Eq. 2: Q_e holds the Jacobian
 * of the cell's map at every quadrature point).  The octree lives in
 * parameter space [lo, hi]^3; the physical domain is Phi([lo, hi]^3) with
 *   kind GCMG_GEOM_WARP: Phi(x) = x + eps (x1 x2, 2 x2 x0, x0 x1 / 2),
 * so every cell is a general trilinear hexahedron; kind 0 restores
 * Cartesian cells.  All levels switch to the quadrature-point operator
 * (values and collocation derivatives at the (k+1)^3 Gauss points, the 3x3
 * factor w det(J) J^-1 J^-T per point, transposed sweeps), the diagonal is
 * recomputed cell by cell, then the coarse inverse and the eigenvalue
 * estimates (synchronous).  Right-hand sides evaluate f and the Dirichlet
 * data at Phi(x) and weight with det(J); DoF coordinates stay in parameter
 * space (physical point = Phi(point)).  GCMG_ERR_ARG for an unknown kind,
 * a map with det(J_Phi) <= 0.05 somewhere in the domain, the learned
 * smoother or a batch's problem.
 */
#define GCMG_GEOM_WARP 1
int gcmg_set_geometry(gcmg_handle* h, int kind, double eps);
/* nu_e of every cell of a level into device memory (1 where none was set) */
int gcmg_get_coefficient(gcmg_handle* h, int level, double* nu);
/* Gauss points of every finest cell: device array n_cells x (k+1)^3 x 3 */
int gcmg_quadrature_points(gcmg_handle* h, double* xyz);
/* lambda_max used by the Chebyshev smoother of a level (after the safety factor) */
int gcmg_get_lambda(const gcmg_handle* h, int level, double* lam);
int gcmg_set_lambda(gcmg_handle* h, int level, double lam);
/*
 * Chebyshev iteration around point Jacobi (Sec. 3.3) on a level:
 * x <- smoother(A, x, b); zero_init = 1 ignores x on entry (Algorithm 2
 * presmoothing).  Uses the level's work vectors.
 */
int gcmg_smooth(gcmg_handle* h, int level, int fp64, void* x, const void* b, int zero_init);
/* fine += P coarse, Eqs. 5-7 (fine_level >= 1, coarse = fine_level - 1) */
int gcmg_prolongate_add(gcmg_handle* h, int fine_level, int fp64, const void* coarse, void* fine);
/* coarse += P^T fine (Sec. 3.5: R = P^T) */
int gcmg_restrict_add(gcmg_handle* h, int fine_level, int fp64, const void* fine, void* coarse);
/* x = A_0^{-1} b on level 0 (Sec. 3.4, exact fp64 solve) */
int gcmg_coarse_solve(gcmg_handle* h, int fp64, const void* b, void* x);
/*
 * x = V-cycle(b) (Algorithms 1-2): b, x are fp64 device vectors of the
 * finest level; the levels run in the configured precision.
 */
int gcmg_vcycle(gcmg_handle* h, const double* b, double* x);
/*
 * The same V-cycle stopped on the finest level right after the prolongation
 * (Algorithm 2 without the finest postsmoothing): the coarse-grid corrected
 * iterate, the state the postsmoother (or a learned step) acts on.
 */
int gcmg_vcycle_cgc(gcmg_handle* h, const double* b, double* x);
/* r = b - A x on a level (vectors of the level, precision by fp64; r != x) */
int gcmg_residual(gcmg_handle* h, int level, int fp64, const void* b, const void* x, void* r);

/*
 * *result = x . y in fp64 (CG inner products, Sec. 2): x, y device arrays of
 * n doubles, result a device pointer to one double.  Deterministic: every
 * block sums a fixed contiguous chunk into the handle's partial-sum buffer
 * and one block adds the partials in a fixed order, so repeated calls give
 * identical bits.  Asynchronous on the handle's stream.
 */
int gcmg_dot(gcmg_handle* h, const double* x, const double* y, int64_t n, double* result);

/*
 * The same fp64 inner product for callers that cannot allocate device
 * memory: no handle, no cudaMalloc/cudaFree, no allocating library call.
 * Such callers include code that runs while stream capture is recording a
 * graph (an allocation would synchronise the device and invalidate the
 * capture), plugins embedded in an application that owns and pre-reserves
 * all of the GPU's memory, and real-time loops where a failed or slow
 * allocation is not acceptable.  The paper has no counterpart of this entry
 * point; it is a service of this library.
 *
 * x, y: device arrays of n doubles; result: device pointer to one double;
 * stream: a cudaStream_t (NULL = legacy default stream).  The partial sums
 * (one per 8192 consecutive elements, added in a fixed order, so the result
 * is reproducible bit for bit) are kept in a fixed 512 KiB device array
 * inside the library, one per GPU that loads it, held until the process
 * exits.  Hence n <= 65536 * 8192 = 536,870,912; larger n is rejected with
 * GCMG_ERR_ARG and a message.
 *
 * The first call on a device looks up that device's array (with the device
 * current); make that first call before any stream capture.  All calls on
 * one device share the array and it keeps the last call's partial sums:
 * calls that overlap on the GPU (other streams, other host threads) race
 * and must be ordered by the caller.  Asynchronous on `stream`.
 */
int gcmg_dot_noalloc(const double* x, const double* y, int64_t n, double* result, void* stream);

/*
 * Same operator with host vectors: copies src (host, n_free values) to the
 * device, applies the operator, copies the result into dst (host) and
 * synchronises.  Pinned host memory gives full copy bandwidth.
 */
int gcmg_vmult_host(gcmg_handle* h, int level, int fp64, const void* src, void* dst);
/*
 * The operator applied to n host vectors: dst[i] = A src[i] (host arrays of
 * n pointers to n_free values each, fp64 when fp64 != 0, else fp32).  The
 * copies to the device, the operators and the copies back of neighbouring
 * vectors overlap: vector i + 1 arrives and vector i - 1 leaves while the
 * operator runs on vector i (two device buffer pairs, three streams).  The
 * results equal gcmg_vmult's bit for bit.  Pinned host memory gives full
 * copy bandwidth; synchronises before returning.
 */
int gcmg_vmult_host_many(gcmg_handle* h, int level, int fp64, int n, const void* const* src, void* const* dst);

/* stages of the per-level timers (CUDA events on the handle's stream) */
#define GCMG_STAGE_VMULT 0       /* each operator application of the V-cycle levels */
#define GCMG_STAGE_PRESMOOTH 1   /* Algorithm 2 presmoothing (its operator applications included) */
#define GCMG_STAGE_RESIDUAL 2
#define GCMG_STAGE_RESTRICT 3
#define GCMG_STAGE_COARSE 4
#define GCMG_STAGE_PROLONGATE 5
#define GCMG_STAGE_POSTSMOOTH 6
#define GCMG_STAGE_CG_VMULT 7    /* fp64 operator of CG on the finest level */
#define GCMG_STAGE_CG_VECTOR 8   /* CG inner products, updates, precision casts */
#define GCMG_STAGE_LEARNED 9     /* learned smoother: its residual and correction */
/* switch the timers on/off; both reset the accumulated times */
int gcmg_set_profiling(gcmg_handle* h, int on);
/* accumulated launches and milliseconds of one (level, stage); synchronises */
int gcmg_get_profile(gcmg_handle* h, int level, int stage, int64_t* count, double* ms);

typedef struct {
  int iterations;
  double r0;            /* ||b||_2 */
  double rel_residual;  /* ||b - A x||_2 / ||b||_2 of the CG recurrence */
  int status;           /* GCMG_OK, GCMG_ERR_NOT_CONVERGED or GCMG_ERR_BREAKDOWN */
} gcmg_solve_stats;

/*
 * CG preconditioned by one V-cycle (Sec. 2, Sec. 5), fp64 vectors and inner
 * products, x_0 = 0, stops when ||b - A x||_2 <= rtol ||b||_2.  b, x: fp64
 * device vectors of the finest level.  Synchronises the stream.
 */
int gcmg_cg_solve(gcmg_handle* h, const double* b, double* x, double rtol, int maxit, gcmg_solve_stats* stats);

/*
 * 1 (default): the V-cycle and the operator half of every CG iteration run as
 * CUDA graphs captured on first use; 0: plain stream launches.  Graphs are
 * re-captured after gcmg_set_lambda and gcmg_set_profiling.
 */
int gcmg_set_graphs(gcmg_handle* h, int on);

/* ------------------------------------------------------------------------
 * Learned per-cell smoother.  An extension outside the paper, whose smoother
 * is Chebyshev around point Jacobi (Sec. 3.3); Chebyshev stays the default.
 *
 * Network: y = W3 g(W2 g(W1 x + b1) + b2) + b3, g the exact GELU
 * z (1 + erf(z / sqrt 2)) / 2.  Parameters are packed fp32 in the order W1
 * (n_hidden x n_in, row-major, one row per output unit), b1, W2 (n_hidden x
 * n_hidden), b2, W3 (n_out x n_hidden), b3.  Every matrix product takes
 * bf16 operands (round to nearest even) and accumulates in fp32.
 *
 * Cell features of cell e (Q_k, n3 = (k+1)^3 support points, lexicographic
 * with x fastest): r_e, d_e = values of the residual and of diag(A) at the
 * cell's support points, hanging points interpolated (C_e G_e of Eq. 2),
 * s_e = |r_e|_2, h_e the cell size, a_k the mean diagonal entry of the
 * unit-cell Laplace matrix; x_e = [r_e / s_e, d_e / (h_e a_k)] (2 n3 values,
 * the first n3 zero where s_e = 0).  Correction c_e = y(x_e) s_e / (h_e a_k);
 * every free DoF takes c_e of its owner cell: the first cell in Morton order
 * in which it is a support point off the faces and edges that border a
 * coarser cell.  The inference kernel is specialised for Q4 with
 * (n_in, n_hidden, n_out) = (250, 128, 125).
 * ------------------------------------------------------------------------ */
typedef struct gcmg_mlp gcmg_mlp;

/* network with zero parameters; sizes 1..4096 */
int gcmg_mlp_create(int n_in, int n_hidden, int n_out, gcmg_mlp** out);
void gcmg_mlp_destroy(gcmg_mlp* net);
int gcmg_mlp_num_params(const gcmg_mlp* net, int64_t* n);
/* copy packed parameters from / to device memory; set resets Adam's state */
int gcmg_mlp_set_params(gcmg_mlp* net, const float* params, void* stream);
int gcmg_mlp_get_params(const gcmg_mlp* net, float* params, void* stream);
/* Y (n x n_out, fp32 device) = network(X) (n x n_in, fp32 device) */
int gcmg_mlp_forward(gcmg_mlp* net, const float* X, int64_t n, float* Y, void* stream);
/*
 * Loss L = sum_i w_i |Y_i - T_i|^2 / (2 sum_i w_i) over n <= 2^20 rows
 * (W: device array of n row weights, or NULL for all 1: the mean squared
 * error) and dL/dparams (packed like the parameters) by back-propagation;
 * grad: device array of num_params floats; loss: device pointer to one float
 * or NULL.
 */
int gcmg_mlp_gradient(gcmg_mlp* net, const float* X, const float* T, const float* W, int64_t n, float* grad,
                      float* loss, void* stream);
/*
 * Adam (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected)
 * on the loss of gcmg_mlp_gradient over consecutive batches of `batch`
 * rows: step s uses the rows order[s * batch .. (s+1) * batch) of X
 * (n_samples x n_in), T (n_samples x n_out) and W (n_samples, or NULL);
 * n_order / batch steps; every order entry must lie in [0, n_samples).
 * losses (device, one float per step, may be NULL) receives each step's
 * loss before its update.  All arrays are device memory; asynchronous on
 * `stream`.
 */
int gcmg_mlp_train(gcmg_mlp* net, const float* X, const float* T, const float* W, int64_t n_samples,
                   const int32_t* order, int64_t n_order, int batch, float lr, float* losses, void* stream);

/* (l, i, j, k) of every cell of a level in the library's cell order: host
 * array of 4 * n_cells int32 */
int gcmg_level_cells(const gcmg_handle* h, int level, int32_t* lijk);
/*
 * out[c * n3 + j] = value of the fp64 device vector x (n_free(level)) at
 * support point j of cell cells[c] (hanging points interpolated, Dirichlet
 * points 0).  cells: device int32 array of n_cells indices, or NULL for all
 * cells in order; out: fp64 device array.
 */
int gcmg_cell_gather(gcmg_handle* h, int level, const double* x, int64_t n_cells, const int32_t* cells,
                     double* out);
/*
 * Training rows of the cells `cells` (device int32, n_cells) from an iterate
 * x, the right-hand side b and a reference solution xstar (fp64 device
 * vectors of the level): with r = b - A x and e = xstar - x, X (n_cells x
 * 2 n3) = the cell features x_e of r, T (n_cells x n3) = e_e h_e a_k / s_e
 * (zero where s_e = 0), W (n_cells) = (s_e / (h_e a_k))^2, the weight that
 * turns the error of y into the error of the correction.  xstar and T may
 * both be NULL; W may be NULL.  Cell indices must lie in [0, n_cells of the
 * level).  Uses the level's fp64 work vectors; synchronises the stream.
 */
int gcmg_mlp_samples(gcmg_handle* h, int level, const double* b, const double* x, const double* xstar,
                     int64_t n_cells, const int32_t* cells, float* X, float* T, float* W);
/*
 * x += the owner-selected corrections of `net` for the residual r (Q4 only).
 * r, x: device vectors of n_free(level) entries, fp64 when fp64 != 0, else
 * fp32; r and x must not overlap.  The first call with a network (and the
 * first after its parameters changed) packs its weights and computes the
 * diagonal part of its first layer for every cell of the level; later calls
 * reuse them.
 */
int gcmg_mlp_correct(gcmg_handle* h, int level, const gcmg_mlp* net, int fp64, const void* r, void* x);
/*
 * Number of bounded device waits of the tensor-core kernels (learned
 * smoother inference and training products) that gave up since the library
 * was loaded or last reset; a kernel whose wait gives up counts it, leaves
 * its remaining output unwritten, frees its tensor memory and returns.
 * Synchronises the device.  reset != 0 sets the count back to zero.
 */
int gcmg_wait_timeouts(unsigned int* count, int reset);

#define GCMG_SMOOTHER_CHEBYSHEV 0   /* Chebyshev around point Jacobi (default) */
#define GCMG_SMOOTHER_MLP_AUGMENT 1 /* postsmoothing, then one learned correction */
#define GCMG_SMOOTHER_MLP_REPLACE 2 /* the learned correction instead of postsmoothing */
/*
 * Smoother of one level of the V-cycle (level >= 1, Q4 for the learned
 * kinds).  The handle keeps a copy of the network's current parameters, so
 * later training does not change it.  With a learned kind on any level the
 * preconditioner is no longer a fixed linear map and gcmg_cg_solve switches
 * to flexible CG (beta = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k, Notay 2000).
 */
int gcmg_set_smoother(gcmg_handle* h, int level, int kind, const gcmg_mlp* net);

/* ------------------------------------------------------------------------
 * Batches of independent problems (an extension: the paper solves one
 * problem per run).  Every problem has its own handle; one CUDA graph holds
 * all of them, each as CG prologue -> conditional WHILE node (body: one CG
 * iteration with its V-cycle and a device-side convergence check that sets
 * the node's condition) -> epilogue, so one graph launch solves the whole
 * batch with no host round trip; the problems are independent branches and
 * run concurrently.
 * ------------------------------------------------------------------------ */
typedef struct gcmg_batch gcmg_batch;

typedef struct {
  int degree;
  int tile_cells;   /* cells per tile */
  int cell_kernel;  /* gcmg_config.cell_kernel */
  int cell_threads; /* gcmg_config.cell_threads */
  double gdofs;     /* measured operator throughput (free DoFs per ns) */
} gcmg_tuning;

/*
 * Autotuner of the operator: for one degree, times the finest-level
 * operator (fp32 when mg_fp32, else fp64) on the probe mesh for every
 * candidate configuration over `reps` applications with CUDA events and
 * returns the fastest in *best; all (optional, GCMG_AUTOTUNE_MAX entries)
 * and n_all get every candidate.  Candidates (tile cells, cell_kernel,
 * cell_threads): the default (one lane per cell on 32-cell tiles); one
 * lane per cell on 8- and 16-cell tiles; one thread per line on 8- to 128-cell tiles (256 or 512 threads
 * for tiles above 32 cells); slab threads on 16- to 64-cell tiles (fp32).
 * The probe's finest level needs at least 2 x SMs x 128 cells, or the
 * larger tile sizes are halved like on any small level.  Synchronises
 * `stream`.
 */
#define GCMG_AUTOTUNE_MAX 16
int gcmg_autotune(const gcmg_mesh* probe, int degree, int mg_fp32, int reps, void* stream, gcmg_tuning* best,
                  gcmg_tuning* all, int* n_all);
/*
 * Set-up of n problems (meshes[i], cfgs[i]); the host set-up runs on
 * n_threads threads (0: 16).  The meshes must outlive the call only.
 */
int gcmg_batch_create(int n, const gcmg_mesh* const* meshes, const gcmg_config* cfgs, int n_threads, void* stream,
                      gcmg_batch** out);
void gcmg_batch_destroy(gcmg_batch* b);
int gcmg_batch_size(const gcmg_batch* b, int* n);
/* the handle of problem i (owned by the batch): right-hand sides, sizes */
int gcmg_batch_handle(gcmg_batch* b, int i, gcmg_handle** h);
/*
 * CG with one V-cycle per iteration for every problem (as gcmg_cg_solve;
 * maxit >= 1): b[i], x[i] fp64 device vectors of problem i (host arrays of
 * n device pointers); stats: host array of n entries or NULL.  The graph is
 * built on the first call and re-used while the pointers, rtol and maxit
 * stay the same.  Synchronises the batch's stream.
 */
int gcmg_batch_cg_solve(gcmg_batch* b, const double* const* rhs, double* const* x, double rtol, int maxit,
                        gcmg_solve_stats* stats);
/*
 * The same solve with the whole batch in one persistent kernel: every
 * problem's launch sequence (CG prologue, one CG iteration with its V-cycle,
 * epilogue) is recorded once as a device work list, and one cooperative
 * launch, captured in a CUDA graph, runs all of it: in each step every
 * unfinished problem performs its next operation, the operations' thread
 * blocks spread over all CTAs, then a grid barrier (bounded waits; a wait
 * that gives up fails the call with GCMG_ERR_INTERNAL).  The operators run
 * the line-parallel kernels on every level (the work list's CTAs have 256
 * threads), and the CG reductions sum the same chunks with 256 threads, so
 * results agree with gcmg_batch_cg_solve to rounding.  At most 1024
 * problems; the list is rebuilt when the pointers, rtol or maxit change.
 * Synchronises the batch's stream.
 */
int gcmg_batch_cg_solve_persistent(gcmg_batch* b, const double* const* rhs, double* const* x, double rtol, int maxit,
                                   gcmg_solve_stats* stats);
typedef struct gcmg_persistent_info {
  int grid;        /* CTAs of the persistent kernel (all resident) */
  int smem_bytes;  /* its dynamic shared memory */
  long long ops;   /* operations in the work list (all problems, one copy of each CG iteration) */
  int steps;       /* lockstep steps of the last solve */
  int in_graph;    /* 1: the launch is a captured CUDA graph */
} gcmg_persistent_info;
/* the work list of the last persistent solve (GCMG_ERR_ARG before the first) */
int gcmg_batch_persistent_info(const gcmg_batch* b, gcmg_persistent_info* info);
/*
 * Test of the persistent kernel's failure path, without a GPU fault: from the
 * next persistent solve on, CTA absent_cta (-1: none) leaves the kernel
 * before the first grid barrier, and a barrier wait gives up after
 * spin_limit polls (default 2^25).  The other CTAs' waits then run out, the
 * kernel records the failure and returns, and the solve fails with
 * GCMG_ERR_INTERNAL; the context stays usable.  (-1, 1 << 25) restores the
 * normal launch.
 */
int gcmg_batch_persistent_wait_test(gcmg_batch* b, int absent_cta, unsigned spin_limit);

/*
 * Host utility: out[i] = a uniform value in [-1, 1) attached to the point
 * xyz[3i..3i+2] (coordinates rounded to multiples of 2^-20, mixed with the
 * SplitMix64 output function), independent of any numbering.  The
 * eigenvalue estimate starts from 1 + these values with seed 2203.
 */
int gcmg_point_values(const double* xyz, int64_t n, uint64_t seed, double* out);

const char* gcmg_last_error(void);
/* number of CUDA kernel launches issued by this library since it was loaded */
int64_t gcmg_launch_count(void);

/*
 * Measurement utility (not part of the method; the paper has none): the
 * peak arithmetic rate of the CUDA cores of the current device in TFLOP/s
 * (a fused multiply-add counts two), fp32 (fp64 = 0) or native fp64
 * (fp64 = 1).  One kernel of `iters` (>= 16) steps of 8 independent
 * multiply-add chains per thread, 2048 threads per SM, timed with CUDA
 * events on `stream` after a short warm-up launch; synchronises the
 * stream.  It is the denominator of the ALU fractions of the operator
 * kernels.  Allocates one small device buffer for the duration of the call.
 */
int gcmg_fma_peak(int fp64, int iters, void* stream, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* GCMG_H */
