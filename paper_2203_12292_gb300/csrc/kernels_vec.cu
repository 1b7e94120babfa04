// Vector kernels of the smoother, the V-cycle and CG.
//
// * Chebyshev iteration around point Jacobi (Sec. 3.3): one fused pass per
//   step, d <- c1 d + c2 D^{-1} (b - A x), x <- x + d (c1 = 0 starts the
//   recurrence).  Reads b, Ax, D^{-1}, d, x and writes d, x.
// * Algorithm 1: casts between the fp64 CG vectors and the fp32 levels.
// * Sec. 3.4: the level-0 solve is a dense product with the inverse of the
//   (small, fp64) level-0 matrix.
// * CG (Sec. 2): fp64 inner products, reduced deterministically in two
//   stages (fixed grid, fixed order), scalars kept on the device.
#include <mutex>
#include <string>

#include "device.cuh"
#include "gcmg.h"
#include "kernels.h"

namespace gcmg {

namespace {

inline int grid_for(int64_t n) {
  int64_t g = (n + BLOCK - 1) / BLOCK;
  if (g > 152 * 16) g = 152 * 16;
  return (int)std::max<int64_t>(g, 1);
}

// grid-stride loop over [0, n) that loads four elements' operands (i, i + S,
// i + 2S, i + 3S) before it stores any of them: four memory round trips in
// flight per thread instead of one.  Every element is read and written at its
// own index only, so the results are those of the plain loop.
template <typename LOAD, typename STORE>
__device__ __forceinline__ void grid_stride4(int64_t n, LOAD load, STORE store) {
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * S < n; i += 4 * S) {
    const auto v0 = load(i), v1 = load(i + S), v2 = load(i + 2 * S), v3 = load(i + 3 * S);
    store(i, v0);
    store(i + S, v1);
    store(i + 2 * S, v2);
    store(i + 3 * S, v3);
  }
  for (; i < n; i += S) store(i, load(i));
}

template <typename A, typename B>
__global__ void cast_kernel(const A* src, B* dst, int64_t n) {
  pdl_begin();
  grid_stride4(n, [&](int64_t i) { return src[i]; }, [&](int64_t i, A v) { dst[i] = (B)v; });
}

template <typename T>
__global__ void copy_to_level_kernel(const double* __restrict__ src, const int32_t* __restrict__ g,
                                     const int32_t* __restrict__ idx, int64_t n, T* __restrict__ dst) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[idx[i]] = (T)src[g[i]];
}

template <typename T>
__global__ void copy_from_level_kernel(const T* __restrict__ src, const int32_t* __restrict__ g,
                                       const int32_t* __restrict__ idx, int64_t n, double* __restrict__ dst) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[g[i]] = (double)src[idx[i]];
}

__global__ void zero_at_kernel(const int32_t* __restrict__ idx, int64_t n, double* a, float* b) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    a[idx[i]] = 0.0;
    b[idx[i]] = 0.f;
  }
}

// Galerkin step length of the learned correction: (r.c, c.w) in fp64 with a
// fixed grid and a fixed summation order (bit-reproducible), then x += om c
template <typename T>
__global__ void __launch_bounds__(BLOCK) dot_pair_partial(const T* __restrict__ r, const T* __restrict__ c,
                                                           const T* __restrict__ w, int64_t n, double* part) {
  pdl_begin();
  __shared__ double s0[BLOCK], s1[BLOCK];
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * BLOCK) {
    const double ci = (double)c[i];
    a += (double)r[i] * ci;
    b += ci * (double)w[i];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int h = BLOCK / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s0[threadIdx.x] += s0[threadIdx.x + h];
      s1[threadIdx.x] += s1[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0[0];
    part[2 * blockIdx.x + 1] = s1[0];
  }
}

__global__ void dot_pair_final(const double* part, int nb, double* out) {
  pdl_begin();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
      a += part[2 * i];
      b += part[2 * i + 1];
    }
    out[0] = a;
    out[1] = b;
  }
}

template <typename T>
__global__ void axpy_ratio_kernel(T* x, const T* c, const double* nd, int64_t n) {
  pdl_begin();
  const double den = nd[1];
  const T om = den > 0.0 ? (T)(nd[0] / den) : T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += om * c[i];
}

template <typename T>
__global__ void zero_kernel(T* x, int64_t n) {
  pdl_begin();
  grid_stride4(n, [&](int64_t) { return 0; }, [&](int64_t i, int) { x[i] = T(0); });
}

__global__ void invert_kernel(const double* d, double* i64, float* i32, int64_t n) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = 1.0 / d[i];
    if (i64) i64[i] = v;
    if (i32) i32[i] = (float)v;
  }
}

template <typename T>
__global__ void cheb_init_kernel(T* x, T* d, const T* b, const T* dinv, T c2, int64_t n) {
  pdl_begin();
  grid_stride4(
      n, [&](int64_t i) { return c2 * dinv[i] * b[i]; },
      [&](int64_t i, T v) {
        d[i] = v;
        x[i] = v;
      });
}

template <typename T, bool FIRST>
__global__ void cheb_step_kernel(T* x, T* d, const T* b, const T* Ax, const T* dinv, T c1, T c2, int64_t n) {
  pdl_begin();
  struct V {
    T r, di, d, x;
  };
  grid_stride4(
      n, [&](int64_t i) { return V{b[i] - Ax[i], dinv[i], FIRST ? T(0) : d[i], x[i]}; },
      [&](int64_t i, V e) {
        const T v = FIRST ? c2 * e.di * e.r : c1 * e.d + c2 * e.di * e.r;
        d[i] = v;
        x[i] = e.x + v;
      });
}

template <typename T>
__global__ void residual_kernel(T* r, const T* b, const T* Ax, int64_t n) {
  pdl_begin();
  grid_stride4(n, [&](int64_t i) { return b[i] - Ax[i]; }, [&](int64_t i, T v) { r[i] = v; });
}

template <typename T>
__global__ void axpy_kernel(T* y, const T* x, T a, int64_t n) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

template <typename T>
__global__ void coarse_kernel(const double* Ainv, int n, const T* b, T* x) {
  pdl_begin();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += Ainv[(size_t)i * n + j] * (double)b[j];
    x[i] = (T)s;
  }
}

// block sum in a fixed order (tree over the block)
__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = BLOCK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// reductions of the CG vectors: DOT_BLOCKS blocks of RB threads (two per SM,
// full occupancy), every thread keeps RU partial sums so that RU loads per
// array are in flight
constexpr int RB = 1024, RU = 4;

__device__ __forceinline__ double block_sum_rb(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = RB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// each block sums a fixed contiguous chunk in a fixed order: the result does
// not depend on scheduling (y in fp32: the fp32 V-cycle's output, widened
// exactly, so the sums equal those over its fp64 copy)
template <typename TY>
__global__ void __launch_bounds__(RB, 2) dot_partial(const double* x, const TY* y, int64_t n, double* part) {
  pdl_begin();
  __shared__ double sh[RB];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s[RU] = {};
  int64_t i = i0 + threadIdx.x;
  for (; i + (RU - 1) * RB < i1; i += RU * RB) {
#pragma unroll
    for (int u = 0; u < RU; ++u) s[u] += x[i + u * RB] * (double)y[i + u * RB];
  }
  for (; i < i1; i += RB) s[0] += x[i] * (double)y[i];
  const double v = block_sum_rb((s[0] + s[1]) + (s[2] + s[3]), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void __launch_bounds__(BLOCK) dot_final(const double* part, int np, double* scal, int slot, int op) {
  pdl_begin();
  __shared__ double sh[BLOCK];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += BLOCK) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    if (op == DOT_STORE) {
      scal[slot] = s;
    } else if (op == DOT_ALPHA) {  // pq, alpha = rz / pq (0 when pq = 0: zero right-hand side)
      scal[1] = s;
      scal[3] = s != 0.0 ? scal[0] / s : 0.0;
    } else if (op == DOT_BETA) {  // rz_new, beta = rz_new / rz, rz <- rz_new
      scal[5] = s;
      scal[4] = s / scal[0];
      scal[0] = s;
    } else {  // flexible CG: beta = (rz_new - r_{k+1}.z_k) / rz, rz <- rz_new
      scal[5] = s;
      scal[4] = (s - scal[6]) / scal[0];
      scal[0] = s;
    }
  }
}

// x += alpha p, r -= alpha q, partial sums of r.r: DOT_BLOCKS blocks of XB
// threads, XU elements per thread in flight; CAST: r also rounded to fp32
// into r32 (the fp32 V-cycle's right-hand side)
constexpr int XB = 512, XU = 4;

template <bool CAST>
__global__ void __launch_bounds__(XB, 2) cg_xr_kernel(double* x, double* r, const double* p, const double* q,
                                                      const double* scal, int64_t n, double* part, float* r32) {
  pdl_begin();
  __shared__ double sh[XB];
  const double alpha = scal[3];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s[XU] = {};
  int64_t i = i0 + threadIdx.x;
  for (; i + (XU - 1) * XB < i1; i += XU * XB) {
    double xv[XU], rv[XU], pv[XU], qv[XU];
#pragma unroll
    for (int u = 0; u < XU; ++u) {
      xv[u] = x[i + u * XB];
      rv[u] = r[i + u * XB];
      pv[u] = p[i + u * XB];
      qv[u] = q[i + u * XB];
    }
#pragma unroll
    for (int u = 0; u < XU; ++u) {
      x[i + u * XB] = xv[u] + alpha * pv[u];
      const double ri = rv[u] - alpha * qv[u];
      r[i + u * XB] = ri;
      if (CAST) r32[i + u * XB] = (float)ri;
      s[u] += ri * ri;
    }
  }
  for (; i < i1; i += XB) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    if (CAST) r32[i] = (float)ri;
    s[0] += ri * ri;
  }
  sh[threadIdx.x] = (s[0] + s[1]) + (s[2] + s[3]);
  __syncthreads();
  for (int h = XB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

template <typename TZ>
__global__ void cg_p_kernel(double* p, const TZ* z, const double* scal, int64_t n) {
  pdl_begin();
  const double beta = scal[4];
  struct V {
    double z, p;
  };
  grid_stride4(
      n, [&](int64_t i) { return V{(double)z[i], p[i]}; }, [&](int64_t i, V e) { p[i] = e.z + beta * e.p; });
}

__global__ void fill_kernel(double* x, double v, int64_t n) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

__global__ void pmul_kernel(double* z, const double* a, const double* b, int64_t n) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = a[i] * b[i];
}

__global__ void xpby_kernel(double* p, const double* z, double beta, int64_t n) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}


// device-side control of a CG solve inside a CUDA graph: the iteration count
// lives in scal[8]; the loop continues while it < maxit, the residual is above
// the tolerance and (p, Ap) > 0 (a NaN residual stops it as well)
__global__ void cg_check_kernel(cudaGraphConditionalHandle h, double* scal, int maxit, double rtol2) {
  pdl_begin();
  const double it = scal[8] + 1.0;
  scal[8] = it;
  const double rr = scal[2], nb2 = scal[7], pq = scal[1];
  const bool go = (it < (double)maxit) && (rr > rtol2 * nb2) && (pq > 0.0);
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void cg_stats_kernel(const double* scal, double rtol2, double* out) {
  pdl_begin();
  const double it = scal[8], rr = scal[2], nb2 = scal[7], pq = scal[1];
  double status = GCMG_ERR_NOT_CONVERGED;
  if (nb2 == 0.0 || rr <= rtol2 * nb2)
    status = GCMG_OK;
  else if (!(pq > 0.0) || rr != rr)
    status = GCMG_ERR_BREAKDOWN;
  out[0] = nb2 == 0.0 ? 0.0 : it;
  out[1] = rr;
  out[2] = nb2;
  out[3] = status;
}

__global__ void scalar_set_kernel(double* scal, int slot, double v) {
  pdl_begin(); scal[slot] = v; }

__global__ void copy_kernel(const double* src, double* dst, int64_t n) {
  pdl_begin();
  grid_stride4(n, [&](int64_t i) { return src[i]; }, [&](int64_t i, double v) { dst[i] = v; });
}

// the two CG reductions with BLOCK threads, for the persistent kernel of the
// device work list (its CTAs have BLOCK threads): the same fixed chunks of the
// same DOT_BLOCKS partial sums, each summed in a fixed order
template <typename TY>
__global__ void __launch_bounds__(BLOCK) dot_partial_b(const double* x, const TY* y, int64_t n, double* part) {
  pdl_begin();
  __shared__ double sh[BLOCK];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s[RU] = {};
  int64_t i = i0 + threadIdx.x;
  for (; i + (RU - 1) * BLOCK < i1; i += RU * BLOCK) {
#pragma unroll
    for (int u = 0; u < RU; ++u) s[u] += x[i + u * BLOCK] * (double)y[i + u * BLOCK];
  }
  for (; i < i1; i += BLOCK) s[0] += x[i] * (double)y[i];
  const double v = block_sum((s[0] + s[1]) + (s[2] + s[3]), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

template <bool CAST>
__global__ void __launch_bounds__(BLOCK) cg_xr_b(double* x, double* r, const double* p, const double* q,
                                                 const double* scal, int64_t n, double* part, float* r32) {
  pdl_begin();
  __shared__ double sh[BLOCK];
  const double alpha = scal[3];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += BLOCK) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    if (CAST) r32[i] = (float)ri;
    s += ri * ri;
  }
  const double v = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

}  // namespace

#ifndef GCMG_BODIES_ONLY

void launch_fill(double* x, double v, int64_t n, cudaStream_t s) {
  if (n > 0) { launch_pdl(fill_kernel, grid_for(n), BLOCK, 0, s, x, v, n); note_launches(1); }
}

void launch_pmul(double* z, const double* a, const double* b, int64_t n, cudaStream_t s) {
  if (n > 0) { launch_pdl(pmul_kernel, grid_for(n), BLOCK, 0, s, z, a, b, n); note_launches(1); }
}

void launch_xpby(double* p, const double* z, double beta, int64_t n, cudaStream_t s) {
  if (n > 0) { launch_pdl(xpby_kernel, grid_for(n), BLOCK, 0, s, p, z, beta, n); note_launches(1); }
}

void launch_cast(bool to64, const void* src, void* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  if (to64)
    { launch_pdl(cast_kernel<float, double>, grid_for(n), BLOCK, 0, s, static_cast<const float*>(src), static_cast<double*>(dst), n); note_launches(1); }
  else
    { launch_pdl(cast_kernel<double, float>, grid_for(n), BLOCK, 0, s, static_cast<const double*>(src), static_cast<float*>(dst), n); note_launches(1); }
}

void launch_copy_to_level(bool fp64, const double* src, const int32_t* g, const int32_t* idx, int64_t n, void* dst,
                          cudaStream_t s) {
  if (n <= 0) return;
  if (fp64)
    launch_pdl(copy_to_level_kernel<double>, grid_for(n), BLOCK, 0, s, src, g, idx, n, static_cast<double*>(dst));
  else
    launch_pdl(copy_to_level_kernel<float>, grid_for(n), BLOCK, 0, s, src, g, idx, n, static_cast<float*>(dst));
  note_launches(1);
}

void launch_copy_from_level(bool fp64, const void* src, const int32_t* g, const int32_t* idx, int64_t n, double* dst,
                            cudaStream_t s) {
  if (n <= 0) return;
  if (fp64)
    launch_pdl(copy_from_level_kernel<double>, grid_for(n), BLOCK, 0, s, static_cast<const double*>(src), g, idx, n, dst);
  else
    launch_pdl(copy_from_level_kernel<float>, grid_for(n), BLOCK, 0, s, static_cast<const float*>(src), g, idx, n, dst);
  note_launches(1);
}

void launch_zero_at(const int32_t* idx, int64_t n, double* a, float* b, cudaStream_t s) {
  if (n <= 0) return;
  launch_pdl(zero_at_kernel, grid_for(n), BLOCK, 0, s, idx, n, a, b);
  note_launches(1);
}

void launch_galerkin_step(bool fp64, const void* r, const void* c, const void* w, void* x, int64_t n,
                          double* scratch, cudaStream_t s) {
  if (n <= 0) return;
  double* nd = scratch + 2 * DOT_BLOCKS;
  if (fp64) {
    launch_pdl(dot_pair_partial<double>, DOT_BLOCKS, BLOCK, 0, s, static_cast<const double*>(r),
               static_cast<const double*>(c), static_cast<const double*>(w), n, scratch);
    launch_pdl(dot_pair_final, 1, 32, 0, s, (const double*)scratch, DOT_BLOCKS, nd);
    launch_pdl(axpy_ratio_kernel<double>, grid_for(n), BLOCK, 0, s, static_cast<double*>(x),
               static_cast<const double*>(c), (const double*)nd, n);
  } else {
    launch_pdl(dot_pair_partial<float>, DOT_BLOCKS, BLOCK, 0, s, static_cast<const float*>(r),
               static_cast<const float*>(c), static_cast<const float*>(w), n, scratch);
    launch_pdl(dot_pair_final, 1, 32, 0, s, (const double*)scratch, DOT_BLOCKS, nd);
    launch_pdl(axpy_ratio_kernel<float>, grid_for(n), BLOCK, 0, s, static_cast<float*>(x),
               static_cast<const float*>(c), (const double*)nd, n);
  }
  note_launches(3);
}

void launch_zero(bool fp64, void* x, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  if (fp64)
    { launch_pdl(zero_kernel<double>, grid_for(n), BLOCK, 0, s, static_cast<double*>(x), n); note_launches(1); }
  else
    { launch_pdl(zero_kernel<float>, grid_for(n), BLOCK, 0, s, static_cast<float*>(x), n); note_launches(1); }
}

void launch_invert(const double* d, double* inv64, float* inv32, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  { launch_pdl(invert_kernel, grid_for(n), BLOCK, 0, s, d, inv64, inv32, n); note_launches(1); }
}

void launch_cheb_init(bool fp64, void* x, void* d, const void* b, const void* dinv, double c2, int64_t n,
                      cudaStream_t s) {
  if (n <= 0) return;
  if (fp64)
    { launch_pdl(cheb_init_kernel<double>, grid_for(n), BLOCK, 0, s, (double*)x, (double*)d, (const double*)b,
                                                            (const double*)dinv, c2, n); note_launches(1); }
  else
    { launch_pdl(cheb_init_kernel<float>, grid_for(n), BLOCK, 0, s, (float*)x, (float*)d, (const float*)b, (const float*)dinv,
                                                           (float)c2, n); note_launches(1); }
}

void launch_cheb_step(bool fp64, void* x, void* d, const void* b, const void* Ax, const void* dinv, double c1,
                      double c2, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  const bool first = (c1 == 0.0);
  if (fp64) {
    if (first)
      { launch_pdl(cheb_step_kernel<double, true>, grid_for(n), BLOCK, 0, s, (double*)x, (double*)d, (const double*)b,
                                                                   (const double*)Ax, (const double*)dinv, c1, c2, n); note_launches(1); }
    else
      { launch_pdl(cheb_step_kernel<double, false>, grid_for(n), BLOCK, 0, s, (double*)x, (double*)d, (const double*)b,
                                                                    (const double*)Ax, (const double*)dinv, c1, c2, n); note_launches(1); }
  } else {
    if (first)
      { launch_pdl(cheb_step_kernel<float, true>, grid_for(n), BLOCK, 0, s, (float*)x, (float*)d, (const float*)b,
                                                                  (const float*)Ax, (const float*)dinv, (float)c1,
                                                                  (float)c2, n); note_launches(1); }
    else
      { launch_pdl(cheb_step_kernel<float, false>, grid_for(n), BLOCK, 0, s, (float*)x, (float*)d, (const float*)b,
                                                                   (const float*)Ax, (const float*)dinv, (float)c1,
                                                                   (float)c2, n); note_launches(1); }
  }
}

void launch_residual(bool fp64, void* r, const void* b, const void* Ax, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  if (fp64)
    { launch_pdl(residual_kernel<double>, grid_for(n), BLOCK, 0, s, (double*)r, (const double*)b, (const double*)Ax, n); note_launches(1); }
  else
    { launch_pdl(residual_kernel<float>, grid_for(n), BLOCK, 0, s, (float*)r, (const float*)b, (const float*)Ax, n); note_launches(1); }
}

void launch_axpy(bool fp64, void* y, const void* x, double a, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  if (fp64)
    { launch_pdl(axpy_kernel<double>, grid_for(n), BLOCK, 0, s, (double*)y, (const double*)x, a, n); note_launches(1); }
  else
    { launch_pdl(axpy_kernel<float>, grid_for(n), BLOCK, 0, s, (float*)y, (const float*)x, (float)a, n); note_launches(1); }
}

void launch_coarse_solve(bool fp64, const double* Ainv, int n, const void* b, void* x, cudaStream_t s) {
  if (n <= 0) return;
  if (fp64)
    { launch_pdl(coarse_kernel<double>, 1, BLOCK, 0, s, Ainv, n, (const double*)b, (double*)x); note_launches(1); }
  else
    { launch_pdl(coarse_kernel<float>, 1, BLOCK, 0, s, Ainv, n, (const float*)b, (float*)x); note_launches(1); }
}

void launch_dot(const double* x, const double* y, int64_t n, double* scratch, double* scal, int slot, int op,
                cudaStream_t s) {
  if (dwl_recording())
    launch_pdl(dot_partial_b<double>, DOT_BLOCKS, BLOCK, 0, s, x, y, n, scratch);
  else
    launch_pdl(dot_partial<double>, DOT_BLOCKS, RB, 0, s, x, y, n, scratch);
  note_launches(1);
  { launch_pdl(dot_final, 1, BLOCK, 0, s, scratch, DOT_BLOCKS, scal, slot, op); note_launches(1); }
}

void launch_dot(const double* x, const float* y, int64_t n, double* scratch, double* scal, int slot, int op,
                cudaStream_t s) {
  if (dwl_recording())
    launch_pdl(dot_partial_b<float>, DOT_BLOCKS, BLOCK, 0, s, x, y, n, scratch);
  else
    launch_pdl(dot_partial<float>, DOT_BLOCKS, RB, 0, s, x, y, n, scratch);
  note_launches(1);
  { launch_pdl(dot_final, 1, BLOCK, 0, s, scratch, DOT_BLOCKS, scal, slot, op); note_launches(1); }
}

void launch_cg_update_xr(double* x, double* r, const double* p, const double* q, const double* scal, int64_t n,
                         double* scratch, double* scal_out, cudaStream_t s, float* r32) {
  if (dwl_recording()) {
    if (r32)
      launch_pdl(cg_xr_b<true>, DOT_BLOCKS, BLOCK, 0, s, x, r, p, q, scal, n, scratch, r32);
    else
      launch_pdl(cg_xr_b<false>, DOT_BLOCKS, BLOCK, 0, s, x, r, p, q, scal, n, scratch, r32);
  } else if (r32) {
    launch_pdl(cg_xr_kernel<true>, DOT_BLOCKS, XB, 0, s, x, r, p, q, scal, n, scratch, r32);
  } else {
    launch_pdl(cg_xr_kernel<false>, DOT_BLOCKS, XB, 0, s, x, r, p, q, scal, n, scratch, r32);
  }
  note_launches(1);
  { launch_pdl(dot_final, 1, BLOCK, 0, s, scratch, DOT_BLOCKS, scal_out, 2, DOT_STORE); note_launches(1); }
}

// ---------------------------------------------------------------------------
// Inner product without any device allocation: the partial sums live in a
// fixed device array of this translation unit instead of a buffer that a
// handle allocates.  One partial per NOALLOC_CHUNK consecutive elements,
// summed in a fixed order, so results are reproducible bit for bit.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NOALLOC_CHUNK = 8192;
constexpr int NOALLOC_MAX_PARTIALS = 65536;  // 512 KiB per device
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_PARTIALS];

__global__ void __launch_bounds__(BLOCK) dot_chunk_partial(const double* x, const double* y, int64_t n, double* part) {
  pdl_begin();
  __shared__ double sh[BLOCK];
  const int64_t i0 = (int64_t)blockIdx.x * NOALLOC_CHUNK;
  const int64_t i1 = min(n, i0 + NOALLOC_CHUNK);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += BLOCK) s += x[i] * y[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(BLOCK) dot_chunk_final(const double* part, int np, double* result) {
  pdl_begin();
  __shared__ double sh[BLOCK];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += BLOCK) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *result = s;
}

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[MAX_DEVICES] = {};

}  // namespace

int64_t dot_noalloc_max_n() { return NOALLOC_CHUNK * (int64_t)NOALLOC_MAX_PARTIALS; }

// Device address of this device's partial-sum array.  Looked up once per
// device, with that device current, on the first call; host code must not
// pass the symbol itself to a kernel (it is a host-side stand-in).
static cudaError_t noalloc_partials(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

cudaError_t launch_dot_noalloc(const double* x, const double* y, int64_t n, double* result, cudaStream_t s) {
  double* part = nullptr;
  cudaError_t e = noalloc_partials(&part);
  if (e != cudaSuccess) return e;
  if (n == 0) return cudaMemsetAsync(result, 0, sizeof(double), s);
  const int np = (int)((n + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
  { launch_pdl(dot_chunk_partial, np, BLOCK, 0, s, x, y, n, part); note_launches(1); }
  { launch_pdl(dot_chunk_final, 1, BLOCK, 0, s, part, np, result); note_launches(1); }
  return cudaGetLastError();
}

void launch_cg_update_p(double* p, const double* z, const double* scal, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  { launch_pdl(cg_p_kernel<double>, grid_for(n), BLOCK, 0, s, p, z, scal, n); note_launches(1); }
}

void launch_cg_update_p(double* p, const float* z, const double* scal, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  { launch_pdl(cg_p_kernel<float>, grid_for(n), BLOCK, 0, s, p, z, scal, n); note_launches(1); }
}

void launch_cg_check(cudaGraphConditionalHandle h, double* scal, int maxit, double rtol2, cudaStream_t s) {
  launch_pdl(cg_check_kernel, 1, 1, 0, s, h, scal, maxit, rtol2);
  note_launches(1);
}

void launch_cg_stats(const double* scal, double rtol2, double* out, cudaStream_t s) {
  launch_pdl(cg_stats_kernel, 1, 1, 0, s, scal, rtol2, out);
  note_launches(1);
}

void launch_scalar_set(double* scal, int slot, double v, cudaStream_t s) {
  launch_pdl(scalar_set_kernel, 1, 1, 0, s, scal, slot, v);
  note_launches(1);
}

void launch_copy(const double* src, double* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  launch_pdl(copy_kernel, grid_for(n), BLOCK, 0, s, src, dst, n);
  note_launches(1);
}

void dwl_register_vec() {
  int id = DWL_BASE_VEC;
#define GCMG_DWL_REG(fn) dwl_register(reinterpret_cast<const void*>(fn), id++, dwl_args_size(fn));
  GCMG_DWL_VEC(GCMG_DWL_REG)
  GCMG_DWL_VEC_SERIAL(GCMG_DWL_REG)
#undef GCMG_DWL_REG
  // grid-stride elementwise kernels: a quarter of the launch's blocks, four elements per thread each
#define GCMG_DWL_COARSEN(fn) dwl_set_coarsen(reinterpret_cast<const void*>(fn), 4);
  GCMG_DWL_COARSEN((cast_kernel<float, double>)) GCMG_DWL_COARSEN((cast_kernel<double, float>))
  GCMG_DWL_COARSEN((copy_kernel)) GCMG_DWL_COARSEN((zero_kernel<float>)) GCMG_DWL_COARSEN((zero_kernel<double>))
  GCMG_DWL_COARSEN((cheb_init_kernel<float>)) GCMG_DWL_COARSEN((cheb_step_kernel<float, true>))
  GCMG_DWL_COARSEN((cheb_step_kernel<float, false>)) GCMG_DWL_COARSEN((residual_kernel<float>))
  GCMG_DWL_COARSEN((cg_p_kernel<double>)) GCMG_DWL_COARSEN((cg_p_kernel<float>))
#undef GCMG_DWL_COARSEN
  dwl_register(reinterpret_cast<const void*>(cg_check_kernel), DWL_OP_CHECK, dwl_args_size(cg_check_kernel));
#define GCMG_DWL_SERIAL(fn) dwl_set_serial(reinterpret_cast<const void*>(fn));
  GCMG_DWL_VEC_SERIAL(GCMG_DWL_SERIAL)
  dwl_set_serial(reinterpret_cast<const void*>(cg_check_kernel));  // run by thread 0 of the persistent kernel
#undef GCMG_DWL_SERIAL
}

#endif  // GCMG_BODIES_ONLY
}  // namespace gcmg
