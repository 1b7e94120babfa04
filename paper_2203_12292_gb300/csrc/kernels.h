// Launch interface of the CUDA kernels of libgcmg (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace gcmg {

// count of kernel launches issued by the library (all host threads)
void note_launches(int n);

enum CellMode { MODE_VMULT = 0, MODE_RHS = 1, MODE_DIAG = 2, MODE_LIFT = 3 };

// arguments of the tile kernels (operator, right-hand side, diagonal)
struct CellLaunch {
  const TileInfo* tiles;
  int n_tiles;
  const CellMeta* meta;
  const int32_t* foreign;
  const uint16_t* subptr;
  const uint8_t* perm;
  const int32_t* cell_ijk;  // per cell i, j, k (right-hand side only)
  // halo: one slot per (tile, foreign DoF); per halo DoF the slots to add
  void* halo;  // n_foreign_total values of the launch precision
  const int32_t* halo_dofs;
  const int32_t* halo_ptr;
  const int32_t* halo_src;
  const int32_t* halo_pos;  // per foreign slot: position in the DoF-ordered halo buffer
  int n_halo;
  int k;
  int tc;
  int max_local;
  int use_lines;  // 1: fp32 operator with the line-parallel kernel
  int threads;    // threads per CTA of the line-parallel operator kernel (128, 256, 384 or 512)
  int n_sm;       // multiprocessors of the device (grid sizes, chunk choices)
  int chunk;      // coarse cells per restriction chunk (0: from the level size)
  int use_lanes;  // 1: fp32 operator with the lane-per-cell kernel (tiles of at most 32 cells)
  const void* lane_tiles;  // per tile LaneTile (null: level without them)
  const int32_t* lane_order;  // launch order of the tiles: those with hanging cells first
  const void* lane_hang;      // per tile LaneHang
  // the same in launch order (block b runs tile lane_order[b]): TileInfo and
  // LaneTile of every tile, LaneHang of the first n_hang_tiles
  const TileInfo* tiles_lo;
  const void* lane_tiles_lo;
  const void* lane_hang_lo;
  int n_hang_tiles;           // tiles with hanging cells
  double lo, dom;
  const double* coef;  // per cell coefficient nu_e (element matrix nu_e h A_ref); null: 1
  int geom;            // 0: Cartesian cells; GEOM_WARP: the cells mapped by the warp below
  double geps;         // its eps
};

// non-Cartesian geometry: the octree cells (parameter space) mapped by
// Phi(x) = x + eps (x1 x2, 2 x2 x0, x0 x1 / 2), the Jacobian evaluated at every
// Gauss point
constexpr int GEOM_WARP = 1;

// analytic function of a right-hand side or of Dirichlet data
enum FuncKind { FUNC_ONE = 0, FUNC_FOURIER = 1, FUNC_GAUSSIAN = 2, FUNC_POLYNOMIAL = 3 };
struct RhsDesc {
  int kind;               // FuncKind
  const double* params;   // FOURIER: per mode kx, ky, kz, phi; GAUSSIAN: alpha, x0, y0, z0;
                          // POLYNOMIAL: per term c, a, b, e (u = sum c x^a y^b z^e)
  int n;                  // modes or terms
  double amp;             // FOURIER: amplitude
};

// dst = A src (add = 0) or dst += A src (add = 1), precision by `fp64`
void launch_vmult(const CellLaunch& L, bool fp64, const void* src, void* dst, int add, cudaStream_t s);
// the tile kernel of the operator for tiles [t0, t1) only (the halo pass is
// launch_halo_add, after all tiles); a tile reads x only below the end of its
// owned range (first-touch ownership), so tile groups can start as the input
// arrives in DoF order.  vmult_tiles_ok: the level's kernels allow it.
bool vmult_tiles_ok(const CellLaunch& L, bool fp64);
void launch_vmult_tiles(const CellLaunch& L, bool fp64, const void* src, void* dst, int t0, int t1, cudaStream_t s);
// the lane-per-cell fp32 operator (tile kernel only, tiles [t0, t1)); lanes_ok:
// the level has its metadata (tiles of at most 32 cells, Cartesian cells)
bool lanes_ok(const CellLaunch& L);
void launch_vmult_lanes(const CellLaunch& L, const void* src, void* dst, int add, int t0, int t1, cudaStream_t s);
// the fp64 operator (double-float arithmetic) with the same structure
void launch_vmult_lanes_df(const CellLaunch& L, const double* src, double* dst, int add, int t0, int t1,
                           cudaStream_t s);
void upload_tables_lanes();
// dst = C^T F: Gauss quadrature of f against the basis (FOURIER, ONE: f
// itself; GAUSSIAN, POLYNOMIAL: f = -Lap u of the manufactured solution u)
void launch_rhs(const CellLaunch& L, const RhsDesc& f, double* dst, cudaStream_t s);
// dst -= C^T A_all u_g: the lifting u_g of the Dirichlet data g = u (u at
// boundary support points, interpolated at hanging points, zero elsewhere)
void launch_rhs_lift(const CellLaunch& L, const RhsDesc& u, double* dst, cudaStream_t s);

// variable coefficient: nu_e = (sum_q w_q) / (sum_q w_q / nu_q) from the
// (k+1)^3 Gauss-point values of every cell; coarse cells from the fine level
// (the fine cell's value, or the mean of the eight children of a refined
// cell); Gauss points of every cell (n_cells x (k+1)^3 x 3, x fastest)
void launch_coef_harmonic(int k, int64_t n_cells, const double* nu_q, double* nu, cudaStream_t s);
void launch_coef_coarsen(int n_coarse, const int32_t* fine_of, const uint8_t* refined, const double* nu_f,
                         double* nu_c, cudaStream_t s);
void launch_quadrature_points(const CellLaunch& L, int64_t n_cells, double* xyz, cudaStream_t s);
// *bad = 1 if any of v[0..n) is not positive and finite (*bad unchanged otherwise)
void launch_check_positive(const double* v, int64_t n, int* bad, cudaStream_t s);
void launch_diag(const CellLaunch& L, const double* diag_tab, double* dst, cudaStream_t s);
// diag_tab[m * (k+1)^3 + j] = (C_m^T A_ref C_m)_{jj} for all 512 masks m
void launch_diag_table(int k, double* diag_tab, cudaStream_t s);
// second pass of every tile loop: dst[g] += halo slots of g, fixed order
void launch_halo_add(const CellLaunch& L, bool fp64, void* dst, cudaStream_t s);
size_t cell_smem_bytes(int k, bool fp64, int tc, int max_local, bool mapped = false);

// transfer between levels; fine_of/refined per coarse cell
struct TransferLaunch {
  int kind;  // 0 = h, 1 = p
  int kf, kc;
  int n_coarse;
  const int32_t* fine_of;
  const uint8_t* refined;
  const int32_t* gstart_f;  // fine cells x 27
  const uint32_t* own_f;    // fine cells
  const int32_t* gstart_c;  // coarse cells x 27
  const uint16_t* mask_c;   // coarse cells
  CellLaunch coarse;        // coarse level tiles (restriction scatter)
};
void launch_prolongate_add(const TransferLaunch& T, bool fp64, const void* coarse, void* fine, cudaStream_t s);
void launch_restrict_add(const TransferLaunch& T, bool fp64, const void* fine, void* coarse, cudaStream_t s);
// coarse (+)= R (b - Ax): the residual formed inside the restriction's gather
// (the same subtraction as launch_residual, so the same values); overwrite:
// coarse = R (b - Ax), no zeroing of coarse needed
void launch_restrict_residual(const TransferLaunch& T, bool fp64, const void* b, const void* Ax, void* coarse,
                              bool overwrite, cudaStream_t s);

// vector kernels
void upload_tables();
void launch_cast(bool to64, const void* src, void* dst, int64_t n, cudaStream_t s);
void launch_zero(bool fp64, void* x, int64_t n, cudaStream_t s);
// x += om c with om = (r.c) / (c.w) (0 when c.w <= 0), w = A c; the two inner
// products in fp64, deterministic; scratch: 2 DOT_BLOCKS + 2 doubles
void launch_galerkin_step(bool fp64, const void* r, const void* c, const void* w, void* x, int64_t n,
                          double* scratch, cudaStream_t s);
// local smoothing, Algorithm 1: dst[idx[i]] = src[g[i]] (to a level, in its
// precision) and dst[g[i]] = src[idx[i]] (back to the fp64 active vector)
void launch_copy_to_level(bool fp64, const double* src, const int32_t* g, const int32_t* idx, int64_t n, void* dst,
                          cudaStream_t s);
void launch_copy_from_level(bool fp64, const void* src, const int32_t* g, const int32_t* idx, int64_t n, double* dst,
                            cudaStream_t s);
// a[idx[i]] = b[idx[i]] = 0 (Jacobi inverse on refinement-edge DoFs)
void launch_zero_at(const int32_t* idx, int64_t n, double* a, float* b, cudaStream_t s);
void launch_invert(const double* d, double* inv64, float* inv32, int64_t n, cudaStream_t s);
void launch_cheb_init(bool fp64, void* x, void* d, const void* b, const void* dinv, double c2, int64_t n, cudaStream_t s);
void launch_cheb_step(bool fp64, void* x, void* d, const void* b, const void* Ax, const void* dinv, double c1,
                      double c2, int64_t n, cudaStream_t s);
void launch_residual(bool fp64, void* r, const void* b, const void* Ax, int64_t n, cudaStream_t s);
void launch_axpy(bool fp64, void* y, const void* x, double a, int64_t n, cudaStream_t s);
void launch_fill(double* x, double v, int64_t n, cudaStream_t s);
void launch_pmul(double* z, const double* a, const double* b, int64_t n, cudaStream_t s);
// p = z + beta p (host scalar)
void launch_xpby(double* p, const double* z, double beta, int64_t n, cudaStream_t s);
void launch_coarse_solve(bool fp64, const double* Ainv, int n, const void* b, void* x, cudaStream_t s);

// deterministic fp64 dot products: partial sums into `scratch` (DOT_BLOCKS
// doubles), then one block combines them in fixed order
constexpr int DOT_BLOCKS = 304;
enum DotOp { DOT_STORE = 0, DOT_ALPHA = 1, DOT_BETA = 2, DOT_BETA_FLEX = 3 };
void launch_dot(const double* x, const double* y, int64_t n, double* scratch, double* scal, int slot, int op,
                cudaStream_t s);
// the same with y in fp32 (widened exactly: equal to the sums over an fp64 copy of y)
void launch_dot(const double* x, const float* y, int64_t n, double* scratch, double* scal, int slot, int op,
                cudaStream_t s);
// inner product with the partial sums in a fixed device array (no allocation);
// n <= dot_noalloc_max_n()
int64_t dot_noalloc_max_n();
cudaError_t launch_dot_noalloc(const double* x, const double* y, int64_t n, double* result, cudaStream_t s);
// CG updates with device scalars: scal[0] = rz, [1] = pq, [2] = rr, [3] = alpha, [4] = beta, [5] = rz_new,
// [6] = r_{k+1}.z_k of flexible CG
// r32 != null: r is also written rounded to fp32 (the fp32 V-cycle's right-hand side)
void launch_cg_update_xr(double* x, double* r, const double* p, const double* q, const double* scal, int64_t n,
                         double* scratch, double* scal_out, cudaStream_t s, float* r32 = nullptr);
void launch_cg_update_p(double* p, const double* z, const double* scal, int64_t n, cudaStream_t s);
void launch_cg_update_p(double* p, const float* z, const double* scal, int64_t n, cudaStream_t s);
// CG inside a graph: scal[7] = |b|^2, scal[8] = iterations; the check kernel
// counts an iteration and sets the while-node condition h; the stats kernel
// writes (iterations, rr, |b|^2, status) to out
void launch_cg_check(cudaGraphConditionalHandle h, double* scal, int maxit, double rtol2, cudaStream_t s);
void launch_cg_stats(const double* scal, double rtol2, double* out, cudaStream_t s);
void launch_scalar_set(double* scal, int slot, double v, cudaStream_t s);
void launch_copy(const double* src, double* dst, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// learned per-cell smoother
// ---------------------------------------------------------------------------
constexpr int MLP_DF = 128;  // bf16 diagonal features stored per cell (Q4: 125 + 3 zeros)
constexpr float MLP_BETA1 = 0.9f, MLP_BETA2 = 0.999f, MLP_EPS = 1e-8f;

// out[c][j] = (C_e G_e v)_j for the cells `cells` (null: 0..n-1), fp64
void launch_cell_gather(int k, const double* v, const int32_t* cells, int64_t n, const int32_t* gstart,
                        const CellMeta* meta, double* out, cudaStream_t s);
// training rows from gathered cell values R (residual), E (error, may be
// null), D (diagonal): X = [R / |R|, D / (h a)], T = E h a / |R|,
// W = (|R| / (h a))^2 (T, W may be null)
void launch_mlp_samples(const double* R, const double* E, const double* D, const int32_t* cells, int64_t n, int n3,
                        const CellMeta* meta, double dom, double abar, float* X, float* T, float* W, cudaStream_t s);
// bf16 rows of MLP_DF diagonal features per cell (all cells of a level)
void launch_mlp_dfeat(const double* D, int64_t n, int n3, const CellMeta* meta, double dom, double abar, void* out,
                      cudaStream_t s);

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]) with bf16 operands and fp32
// accumulation; A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn]
struct GemmArgs {
  const float* A;
  int64_t sam, sak;
  const float* B;
  int64_t sbk, sbn;
  float* C;
  int64_t ldc;
  const float* bias;
  int M, N, K;
  const uint16_t* Ab = nullptr;  // bf16 A (row stride sam, k contiguous) in place of A
};
void launch_gemm_bf16(const GemmArgs& g, cudaStream_t s);
void launch_gelu(const float* Z, float* H, int64_t n, cudaStream_t s);
void launch_gelu_bwd(const float* dH, const float* Z, float* dZ, int64_t n, cudaStream_t s);
// B rows of m outputs, weights W (null: 1): dY = w (Y - T) / sum w,
// *loss = sum w |Y - T|^2 / (2 sum w)
void launch_mse(const float* Y, const float* T, const float* W, float* dY, int B, int m, float* loss,
                cudaStream_t s);
void launch_colsum(const float* X, int M, int N, float* out, cudaStream_t s);
void launch_gather_rows(const float* X, int64_t ld, const int32_t* idx, int B, float* out, cudaStream_t s);
// Adam with bias corrections bc1 = 1 - beta1^t, bc2 = 1 - beta2^t
void launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float bc1, float bc2,
                 cudaStream_t s);

// fused per-cell correction x += owner-selected MLP(r) for Q4 (250-128-128-125)
struct MlpFused {
  const void* wimg;        // packed bf16 weight image (launch_mlp_prepare), 16-byte aligned
  const float* dproj;      // per cell: b1 + the diagonal features times their W1 columns (128)
  const int32_t* gstart;   // cells x 27
  const uint32_t* own;     // per cell: owned slots
  const CellMeta* meta;
  int64_t n_cells;
  double dom;              // edge length of the domain
  double abar;             // mean diagonal entry of the unit-cell matrix
};
size_t mlp_fused_smem_bytes();
size_t mlp_image_bytes();
// weight image of a 250-128-128-125 network from its packed fp32 parameters,
// and the diagonal part of its first layer for every cell of a level (dproj:
// n_cells x 128 fp32, from the bf16 diagonal features dfeat)
void launch_mlp_prepare(const float* params, const uint16_t* dfeat, int64_t n_cells, void* image, float* dproj,
                        cudaStream_t s);
// bounded tensor-core waits that gave up since the last reset (synchronous)
unsigned int wait_timeouts(bool reset);
// multiprocessors of the current device (152 without a usable device)
int device_sm_count();
cudaError_t launch_mlp_correct(const MlpFused& P, bool fp64, const void* r, void* x, cudaStream_t s);

}  // namespace gcmg
