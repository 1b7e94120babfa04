// Kernels of the learned per-cell smoother, an extension outside the paper
// (the paper smooths with Chebyshev around point Jacobi, Sec. 3.3).
//
// * cell gather: the values of a free-DoF vector at the (k+1)^3 support
//   points of a list of cells, hanging points interpolated (G_e, then C_e of
//   Eq. 2), in fp64.
// * training: a bf16 GEMM on the fifth-generation tensor cores (tcgen05.mma,
//   fp32 accumulators in TMEM) with arbitrary operand strides, so that every
//   product of the forward and backward passes (X W^T, dY^T H, dY W) is one
//   launch; GELU, loss, column sums and Adam as elementwise kernels.
// * inference: one persistent kernel per application.  Each CTA keeps the
//   bf16 weights in shared memory (one bulk copy) and loops over batches of
//   128 cells: gather the residual, interpolate hanging points, scale by the
//   cell norm, run the three layers as 128 x 128 x 128 tcgen05 products with
//   the accumulators in TMEM, and add the correction to the DoFs the cell
//   owns (each DoF has exactly one owner cell, so there are no races and no
//   atomics).  The diagonal half of the first layer depends only on the cell
//   and the network, so it is computed once per network (a GEMM over all
//   cells) and read back per application.
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace gcmg {

GCMG_DEFINE_UPLOAD(upload_tables_mlp)

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (lower address, low half) = lo
  return *reinterpret_cast<uint32_t*>(&v);
}

// bounded tensor-core waits that gave up (read by gcmg_wait_timeouts)
__device__ unsigned int g_wait_timeouts;

__device__ __forceinline__ float bf16_bits_to_float(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
// GELU of the inference kernel, z Phi(z) with erf from the rational
// approximation of Abramowitz & Stegun, Handbook of Mathematical Functions,
// formula 7.1.26 (|error| <= 1.5e-7 for x >= 0; odd extension), far below the
// bf16 rounding (2^-9 relative) its result goes through
__device__ __forceinline__ float gelu_as(float z) {
  const float x = fabsf(z) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
  const float p =
      t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
  const float erf_abs = fmaf(-p, __expf(-x * x), 1.0f);
  return 0.5f * z * (1.0f + copysignf(erf_abs, z));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---------------------------------------------------------------------------
// cell gather (fp64)
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) cell_gather_kernel(const double* v, const int32_t* cells, int64_t n,
                                                          const int32_t* gstart, const CellMeta* meta,
                                                          double* out) {
  constexpr int N = K + 1, N3 = N * N * N, CPB = 8;
  __shared__ double buf[CPB * N3];
  __shared__ uint16_t sm_mask[CPB];
  const int64_t c0 = (int64_t)blockIdx.x * CPB;
  const int nc = (int)(n - c0 < CPB ? n - c0 : CPB);
  if (threadIdx.x < CPB)
    sm_mask[threadIdx.x] = (int)threadIdx.x < nc ? meta[cells ? cells[c0 + threadIdx.x] : c0 + threadIdx.x].mask : 0;
  for (int t = threadIdx.x; t < CPB * N3; t += blockDim.x) {
    const int i = t / N3, j = t - i * N3;
    double val = 0.0;
    if (i < nc) {
      const int64_t cell = cells ? cells[c0 + i] : c0 + i;
      int slot, off;
      node_slot<K>(j % N, (j / N) % N, j / (N * N), slot, off);
      const int32_t gs = gstart[cell * NSLOT + slot];
      if (gs >= 0) val = v[gs + off];
    }
    buf[t] = val;
  }
  __syncthreads();
  hanging_all<K, false, double>(buf, sm_mask, nc);
  for (int t = threadIdx.x; t < nc * N3; t += blockDim.x) out[c0 * N3 + t] = buf[t];
}

// training samples from gathered cell values: one warp per sample
__global__ void samples_kernel(const double* R, const double* E, const double* D, const int32_t* cells, int64_t n,
                               int n3, const CellMeta* meta, double dom, double abar, float* X, float* T, float* W) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const double* r = R + w * n3;
  double ss = 0.0;
  for (int j = lane; j < n3; j += 32) ss += r[j] * r[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const double s = sqrt(ss);
  const int64_t cell = cells ? cells[w] : w;
  const double h = dom / (double)(1u << meta[cell].level);
  const double sinv = s > 0.0 ? 1.0 / s : 0.0;
  const double ts = s > 0.0 ? h * abar / s : 0.0;
  if (W && lane == 0) W[w] = (float)((s / (h * abar)) * (s / (h * abar)));
  for (int j = lane; j < n3; j += 32) {
    X[w * 2 * n3 + j] = (float)(r[j] * sinv);
    X[w * 2 * n3 + n3 + j] = (float)(D[w * n3 + j] / (h * abar));
    if (T) T[w * n3 + j] = E ? (float)(E[w * n3 + j] * ts) : 0.0f;
  }
}

// inference features of the diagonal: bf16 rows of MLP_DF per cell
__global__ void dfeat_kernel(const double* D, int64_t n, int n3, const CellMeta* meta, double dom, double abar,
                             bf16* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * MLP_DF) return;
  const int64_t c = i / MLP_DF;
  const int j = (int)(i - c * MLP_DF);
  const double h = dom / (double)(1u << meta[c].level);
  out[i] = __float2bfloat16_rn(j < n3 ? (float)(D[c * n3 + j] / (h * abar)) : 0.0f);
}

// ---------------------------------------------------------------------------
// training kernels
// ---------------------------------------------------------------------------
// C = A B (+ bias) with A (M x K) and B (K x N) at arbitrary strides, operands
// rounded to bf16, fp32 accumulation.  One CTA per 128 x 128 tile of C: the
// threads convert a 128 x 64 chunk of A and of B^T into the K-major core
// layout, one thread issues four 128 x 128 x 16 tcgen05 products into TMEM,
// and the chunk's completion (mbarrier, bounded wait) frees the buffers for
// the next one; the eight warps then read the accumulator back (warp w: TMEM
// lanes 32 (w % 4) .., columns 64 (w / 4) ..) and store C.
constexpr int GM = 128, GN = 128, GKC = 64, GTH = 256;

__global__ void __launch_bounds__(GTH) gemm_tc_kernel(GemmArgs g) {
  __shared__ __align__(1024) bf16 As[GM * GKC];
  __shared__ __align__(1024) bf16 Bs[GN * GKC];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
  if (warp == 0) tc::tmem_alloc(&tslot, GN);
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  constexpr uint32_t SBO = GKC / 8 * 128;  // row-group stride of a chunk
  const bool a_kfast = g.Ab != nullptr || g.sak == 1, b_kfast = g.sbk == 1;
  const int nk = (g.K + GKC - 1) / GKC;
  uint32_t phase = 0;
  bool ok = true;
  for (int c = 0; c < nk; ++c) {
    const int k0 = c * GKC;
    // every thread issues eight loads of the chunk before it converts and
    // stores them (consecutive threads along the operand's contiguous dimension)
    constexpr int PER = GM * GKC / GTH, INF = 8;
    static_assert(GM == GN && PER * GTH == GM * GKC && PER % INF == 0, "chunk split");
#pragma unroll 1
    for (int u0 = 0; u0 < PER; u0 += INF) {
      float v[INF];
#pragma unroll
      for (int u = 0; u < INF; ++u) {
        const int e = tid + (u0 + u) * GTH;
        const int i = a_kfast ? e / GKC : e % GM, kk = a_kfast ? e % GKC : e / GM;
        const int m = m0 + i, k = k0 + kk;
        v[u] = 0.0f;
        if (m < g.M && k < g.K)
          v[u] = g.Ab ? bf16_bits_to_float(g.Ab[(int64_t)m * g.sam + k]) : g.A[(int64_t)m * g.sam + (int64_t)k * g.sak];
      }
#pragma unroll
      for (int u = 0; u < INF; ++u) {
        const int e = tid + (u0 + u) * GTH;
        const int i = a_kfast ? e / GKC : e % GM, kk = a_kfast ? e % GKC : e / GM;
        As[tc::core_off(i, kk, GKC)] = __float2bfloat16_rn(v[u]);
      }
    }
#pragma unroll 1
    for (int u0 = 0; u0 < PER; u0 += INF) {
      float v[INF];
#pragma unroll
      for (int u = 0; u < INF; ++u) {
        const int e = tid + (u0 + u) * GTH;
        const int i = b_kfast ? e / GKC : e % GN, kk = b_kfast ? e % GKC : e / GN;
        const int n = n0 + i, k = k0 + kk;
        v[u] = (n < g.N && k < g.K) ? g.B[(int64_t)k * g.sbk + (int64_t)n * g.sbn] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < INF; ++u) {
        const int e = tid + (u0 + u) * GTH;
        const int i = b_kfast ? e / GKC : e % GN, kk = b_kfast ? e % GKC : e / GN;
        Bs[tc::core_off(i, kk, GKC)] = __float2bfloat16_rn(v[u]);
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t a0 = tc::saddr(As), b0 = tc::saddr(Bs);
#pragma unroll
      for (int s = 0; s < GKC / 16; ++s)
        tc::mma_bf16(tmem, tc::sdesc(a0 + s * 256, 128, SBO), tc::sdesc(b0 + s * 256, 128, SBO),
                     tc::idesc_bf16(GM, GN), (c > 0 || s > 0) ? 1u : 0u);
      tc::commit(&bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&bar, phase));
    phase ^= 1u;
    tc::fence_after();
    if (!ok) break;
  }
  if (!ok) {
    if (tid == 0) atomicAdd(&g_wait_timeouts, 1u);
    tc::mbar_wait(&bar, phase ^ 1u);  // once more for the products in flight
  } else {
    const int q = warp & 3, h = warp >> 2, m = m0 + 32 * q + lane;
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      const int col0 = 64 * h + 32 * part;
      float v[32];
      if (nk > 0) {
        tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.0f;
      }
      if (m < g.M)
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + col0 + j;
          if (n < g.N) g.C[(int64_t)m * g.ldc + n] = v[j] + (g.bias ? g.bias[n] : 0.0f);
        }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, GN);
}

__global__ void gelu_kernel(const float* Z, float* H, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    H[i] = gelu_f(Z[i]);
}

__global__ void gelu_bwd_kernel(const float* dH, const float* Z, float* dZ, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dZ[i] = dH[i] * gelu_grad_f(Z[i]);
}

__device__ float block_sum256(float s, float* sh) {
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const float r = sh[0];
  __syncthreads();
  return r;
}

// weighted squared error over B rows of m outputs (W null: all weights 1):
// dY = w (Y - T) / sum w, L = sum w |Y - T|^2 / (2 sum w); one block, fixed order
__global__ void __launch_bounds__(256) loss_kernel(const float* Y, const float* T, const float* W, float* dY, int B,
                                                   int m, float* loss) {
  __shared__ float sh[256];
  float sw = 0.0f;
  if (W)
    for (int b = threadIdx.x; b < B; b += blockDim.x) sw += W[b];
  sw = W ? block_sum256(sw, sh) : (float)B;
  const float inv = sw > 0.0f ? 1.0f / sw : 0.0f;
  float s = 0.0f;
  const int64_t n = (int64_t)B * m;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float w = W ? W[i / m] : 1.0f;
    const float d = Y[i] - T[i];
    dY[i] = w * d * inv;
    s += w * d * d;
  }
  s = block_sum256(s, sh);
  if (threadIdx.x == 0 && loss) *loss = 0.5f * s * inv;
}

// out[j] = sum_i X[i][j] (rows in order)
__global__ void colsum_kernel(const float* X, int M, int N, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.0f;
  for (int i = 0; i < M; ++i) s += X[(int64_t)i * N + j];
  out[j] = s;
}

__global__ void gather_rows_kernel(const float* X, int64_t ld, const int32_t* idx, int B, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * ld) return;
  const int64_t r = i / ld, c = i - r * ld;
  out[i] = X[(int64_t)idx[r] * ld + c];
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t n, float lr, float bc1, float bc2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float mi = MLP_BETA1 * m[i] + (1.0f - MLP_BETA1) * g[i];
    const float vi = MLP_BETA2 * v[i] + (1.0f - MLP_BETA2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + MLP_EPS);
  }
}

// ---------------------------------------------------------------------------
// fused inference for Q4: 250 -> 128 -> 128 -> 125
// ---------------------------------------------------------------------------
constexpr int FK = 4, FN3 = 125, FC = 128, FT = 512;  // degree, nodes, cells per batch, threads
// row stride of the fp32 cell buffer: 16-byte rows for the async copies of
// the first layer's diagonal part, four-row bank period
constexpr int SS = 132;
// shared memory (offsets from a 1024-byte aligned base):
// [W1 residual columns | W2 | W3 (bf16 operand tiles, 128 x 128 each) | b2, b3 (fp32)] = the weight image,
// then the activation tile A (bf16 128 x 128: features, then H1, then H2), the fp32 cell buffer
// (residual, then the diagonal part of layer 1, then the correction), two buffers of slot starts
// (the next batch's arrive by bulk copy while this one runs), per-cell data, barriers
constexpr size_t F_W1 = 0, F_W2 = 32768, F_W3 = 65536, F_B = 98304;
constexpr size_t F_IMG = F_B + 2 * 128 * 4;  // bytes of the weight image
constexpr size_t F_A = F_IMG;
constexpr size_t F_ST = F_A + 32768;
constexpr size_t F_GS = F_ST + (size_t)FC * SS * 4;
constexpr size_t GS_BYTES = (size_t)FC * NSLOT * 4;
constexpr size_t F_OWN = F_GS + 2 * GS_BYTES;
constexpr size_t F_MK = F_OWN + FC * 4;
constexpr size_t F_LV = F_MK + FC * 2;
constexpr size_t F_SI = F_LV + FC * 4;
constexpr size_t F_SC = F_SI + FC * 4;
constexpr size_t F_BAR = F_SC + FC * 4;
constexpr size_t F_END = F_BAR + 48;
constexpr size_t F_BYTES = F_END + 1024;  // room to align the base
static_assert(F_BYTES <= 232448, "fused MLP kernel exceeds the shared memory of a CTA");
static_assert(F_A % 1024 == 0 && F_ST % 16 == 0 && F_GS % 16 == 0 && GS_BYTES % 16 == 0 && F_BAR % 8 == 0,
              "aligned operand tiles, copies and barriers");
static_assert(F_IMG % 16 == 0, "the weight image moves in one bulk copy");
constexpr uint32_t ASBO = 128 / 8 * 128;  // row-group stride of a 128-column operand tile

// weight image in the shared-memory layout of the fused kernel: the first
// layer's residual columns (125, padded to 128), W2 and W3 (rows 125..127
// zero) as K-major operand tiles, then b2 and b3
__global__ void mlp_pack_kernel(const float* __restrict__ P, unsigned char* img) {
  const float* W1 = P;
  const float* b1 = W1 + 128 * 250;
  const float* W2 = b1 + 128;
  const float* b2 = W2 + 128 * 128;
  const float* W3 = b2 + 128;
  const float* b3 = W3 + 125 * 128;
  bf16* W1s = reinterpret_cast<bf16*>(img + F_W1);
  bf16* W2s = reinterpret_cast<bf16*>(img + F_W2);
  bf16* W3s = reinterpret_cast<bf16*>(img + F_W3);
  float* bs = reinterpret_cast<float*>(img + F_B);
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 128 * 128; e += stride) {
    const int n = e >> 7, k = e & 127, o = tc::core_off(n, k, 128);
    W1s[o] = __float2bfloat16_rn(k < FN3 ? W1[n * 250 + k] : 0.0f);
    W2s[o] = __float2bfloat16_rn(W2[n * 128 + k]);
    W3s[o] = __float2bfloat16_rn(n < FN3 ? W3[n * 128 + k] : 0.0f);
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 128; e += stride) {
    bs[e] = b2[e];
    bs[128 + e] = e < FN3 ? b3[e] : 0.0f;
  }
}

// the 32 columns col0.. of this thread's TMEM lane, GELU, as bf16 into row i
// of the activation tile
__device__ __forceinline__ void act_store(uint32_t taddr, const float (&add)[32], unsigned char* A, int i, int col0) {
  float v[32];
  tc::tmem_ld32(taddr, v);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    uint4 w;
    w.x = pack_bf16(gelu_as(v[8 * u + 0] + add[8 * u + 0]), gelu_as(v[8 * u + 1] + add[8 * u + 1]));
    w.y = pack_bf16(gelu_as(v[8 * u + 2] + add[8 * u + 2]), gelu_as(v[8 * u + 3] + add[8 * u + 3]));
    w.z = pack_bf16(gelu_as(v[8 * u + 4] + add[8 * u + 4]), gelu_as(v[8 * u + 5] + add[8 * u + 5]));
    w.w = pack_bf16(gelu_as(v[8 * u + 6] + add[8 * u + 6]), gelu_as(v[8 * u + 7] + add[8 * u + 7]));
    *reinterpret_cast<uint4*>(A + 2 * tc::core_off(i, col0 + 8 * u, 128)) = w;
  }
}

// one layer on the tensor cores: D (TMEM columns dcol..) = A W^T over K = 128
__device__ __forceinline__ void layer_mma(uint32_t tmem, uint32_t dcol, const unsigned char* A,
                                          const unsigned char* W, uint64_t* bar) {
  tc::fence_after();
  const uint32_t a0 = tc::saddr(A), w0 = tc::saddr(W);
#pragma unroll
  for (int s = 0; s < 8; ++s)
    tc::mma_bf16(tmem + dcol, tc::sdesc(a0 + s * 256, 128, ASBO), tc::sdesc(w0 + s * 256, 128, ASBO),
                 tc::idesc_bf16(128, 128), s > 0 ? 1u : 0u);
  tc::commit(bar);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::saddr(dst)), "l"(src) : "memory");
}

// x += v with no value returned (each DoF has one owner: no contention, the
// same sum as a plain read-modify-write, and no wait on the read)
__device__ __forceinline__ void add_global(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void add_global(double* p, double v) { atomicAdd(p, v); }

template <typename T>
__global__ void __launch_bounds__(FT, 1) mlp_correct_kernel(MlpFused P, const T* __restrict__ r, T* x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024u - (tc::saddr(smem_raw) & 1023u)) & 1023u);
  const float* bs = reinterpret_cast<const float*>(sm + F_B);
  unsigned char* Atile = sm + F_A;
  float* St = reinterpret_cast<float*>(sm + F_ST);
  uint32_t* own = reinterpret_cast<uint32_t*>(sm + F_OWN);
  uint16_t* mk = reinterpret_cast<uint16_t*>(sm + F_MK);
  float* hs = reinterpret_cast<float*>(sm + F_LV);
  float* si = reinterpret_cast<float*>(sm + F_SI);
  float* sc = reinterpret_cast<float*>(sm + F_SC);
  uint64_t* wbar = reinterpret_cast<uint64_t*>(sm + F_BAR);
  uint64_t* mbar = wbar + 1;
  uint64_t* gbar = wbar + 2;  // two: one per slot-start buffer
  uint32_t* tslot = reinterpret_cast<uint32_t*>(wbar + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) tc::tmem_alloc(tslot, 256);
  if (tid == 0) {
    tc::mbar_init(wbar, 1);
    tc::mbar_init(mbar, 1);
    tc::mbar_init(gbar, 1);
    tc::mbar_init(gbar + 1, 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const int64_t nbatch = (P.n_cells + FC - 1) / FC;
  // slot starts of batch bt: a bulk copy for full batches, plain loads for the ragged one
  auto full = [&](int64_t bt) { return bt < nbatch && (bt + 1) * FC <= P.n_cells; };
  // copies of slot starts in flight (bit b: buffer b) and the parity each buffer's next completion has
  uint32_t gout = 0, gpar = 0;
  if (tid == 0) {
    tc::bulk_g2s(sm, P.wimg, (uint32_t)F_IMG, wbar);
    if (full(blockIdx.x)) tc::bulk_g2s(sm + F_GS, P.gstart + (int64_t)blockIdx.x * FC * NSLOT, (uint32_t)GS_BYTES, gbar);
  }
  if (full(blockIdx.x)) gout = 1u;
  // per-cell data of the next batch, one cell per thread, prefetched into registers
  uint32_t pm = 0, po = 0;
  if (tid < FC && (int64_t)blockIdx.x < nbatch && (int64_t)blockIdx.x * FC + tid < P.n_cells) {
    const CellMeta& m = P.meta[(int64_t)blockIdx.x * FC + tid];
    pm = m.mask | ((uint32_t)m.level << 16);
    po = P.own[(int64_t)blockIdx.x * FC + tid];
  }
  bool ok = __syncthreads_and(tc::mbar_wait(wbar, 0));

  // gather and update: node jn (entity slot nslot, offset noff) of cells cq, cq + 4, ..
  const int jn = tid & 127, cq = tid >> 7;
  const bool node_ok = jn < FN3;
  int nslot = 0, noff = 0;
  if (node_ok) node_slot<FK>(jn % 5, (jn / 5) % 5, jn / 25, nslot, noff);
  const float dom = (float)P.dom, abar = (float)P.abar;
  const int q = warp & 3, cg = warp >> 2;  // TMEM lanes 32 q .., columns 32 cg ..
  const int row = 32 * q + lane, col0 = 32 * cg;
  const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
  uint32_t phase = 0;
  int it = 0;
  for (int64_t bt = blockIdx.x; ok && bt < nbatch; bt += gridDim.x, ++it) {
    const int64_t c0 = bt * FC;
    const int nc = (int)(P.n_cells - c0 < FC ? P.n_cells - c0 : FC);
    const int buf = it & 1;
    int32_t* gs = reinterpret_cast<int32_t*>(sm + F_GS + buf * GS_BYTES);
    if (tid < FC) {
      mk[tid] = (uint16_t)(pm & 0xFFFFu);
      hs[tid] = dom * __int_as_float((127 - (int)(pm >> 16)) << 23);  // dom 2^-level, exact
      own[tid] = po;
    }
    if (gout >> buf & 1u) {
      ok = tc::mbar_wait(gbar + buf, gpar >> buf & 1u);
      if (ok) {
        gout &= ~(1u << buf);
        gpar ^= 1u << buf;
      }
    } else {
      for (int e = tid; e < FC * NSLOT; e += FT) gs[e] = e < nc * NSLOT ? P.gstart[c0 * NSLOT + e] : -1;
    }
    // the next batch of this CTA: slot starts into the other buffer (its last
    // reader, the previous batch, has passed the barrier at its end)
    const int64_t nb = bt + gridDim.x;
    if (full(nb)) {
      if (tid == 0) {
        tc::fence_async_smem();
        tc::bulk_g2s(sm + F_GS + (buf ^ 1) * GS_BYTES, P.gstart + nb * FC * NSLOT, (uint32_t)GS_BYTES,
                     gbar + (buf ^ 1));
      }
      gout |= 1u << (buf ^ 1);
    }
    pm = 0, po = 0;
    if (tid < FC && nb < nbatch && nb * FC + tid < P.n_cells) {
      const CellMeta& m = P.meta[nb * FC + tid];
      pm = m.mask | ((uint32_t)m.level << 16);
      po = P.own[nb * FC + tid];
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    // gather the residual: thread (jn, cq) fetches node jn of cells cq, cq + 4, ..
    {
      float v[FC / 4];
#pragma unroll
      for (int u = 0; u < FC / 4; ++u) {
        const int32_t base = node_ok ? gs[(cq + 4 * u) * NSLOT + nslot] : -1;
        v[u] = base >= 0 ? (float)r[base + noff] : 0.0f;
      }
      if (node_ok)
#pragma unroll
        for (int u = 0; u < FC / 4; ++u) St[(cq + 4 * u) * SS + jn] = v[u];
    }
    const int hang = __syncthreads_or(tid < nc && (mk[tid] & MASK_HANG));
    if (hang) hanging_all<FK, false, float, SS>(St, mk, nc);
    // cell norms and scales: four threads per cell
    {
      const int i = tid >> 2, p = tid & 3;
      float ss = 0.0f;
#pragma unroll 8
      for (int j = p; j < FN3; j += 4) ss = fmaf(St[i * SS + j], St[i * SS + j], ss);
      ss += __shfl_xor_sync(0xffffffffu, ss, 1);
      ss += __shfl_xor_sync(0xffffffffu, ss, 2);
      if (p == 0) {
        const float s = sqrtf(ss);
        si[i] = s > 0.0f ? 1.0f / s : 0.0f;
        sc[i] = i < nc ? s / (hs[i] * abar) : 0.0f;
      }
    }
    __syncthreads();
    // features bf16(r / s) as the A operand; each warp writes whole core matrices
    for (int e = tid; e < FC * 64; e += FT) {
      const int blk = e >> 5, l = e & 31;
      const int i = 8 * (blk >> 4) + (l & 7), k = 8 * (blk & 15) + 2 * (l >> 3);
      const float v0 = k < FN3 ? St[i * SS + k] * si[i] : 0.0f;
      const float v1 = k + 1 < FN3 ? St[i * SS + k + 1] * si[i] : 0.0f;
      *reinterpret_cast<uint32_t*>(Atile + 2 * tc::core_off(i, k, 128)) = pack_bf16(v0, v1);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    // layer 1: H1 = gelu(X W1r^T + dproj), dproj holding b1 and the diagonal features' part;
    // dproj rows move into the (now free) cell buffer while the tensor cores run
    if (tid == 0) layer_mma(tmem, 0, Atile, sm + F_W1, mbar);
#pragma unroll
    for (int u = 0; u < FC * 32 / FT; ++u) {
      const int e = tid + u * FT, i = e >> 5, c = e & 31;
      float* d = St + i * SS + 4 * c;
      if (i < nc)
        cp_async16(d, P.dproj + (c0 + i) * 128 + 4 * c);
      else
        *reinterpret_cast<float4*>(d) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    ok = __syncthreads_and(tc::mbar_wait(mbar, phase));
    phase ^= 1u;
    tc::fence_after();
    if (!ok) break;
    {
      float add[32];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 w = *reinterpret_cast<const float4*>(St + row * SS + col0 + 4 * u);
        add[4 * u] = w.x, add[4 * u + 1] = w.y, add[4 * u + 2] = w.z, add[4 * u + 3] = w.w;
      }
      act_store(tl + (uint32_t)col0, add, Atile, row, col0);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    // layer 2: H2 = gelu(H1 W2^T + b2), accumulated in TMEM columns 128..
    if (tid == 0) layer_mma(tmem, 128, Atile, sm + F_W2, mbar);
    ok = __syncthreads_and(tc::mbar_wait(mbar, phase));
    phase ^= 1u;
    tc::fence_after();
    if (!ok) break;
    {
      float add[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) add[j] = bs[col0 + j];
      act_store(tl + 128u + (uint32_t)col0, add, Atile, row, col0);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    // layer 3: correction c = (H2 W3^T + b3) s / (h a) into the cell buffer
    if (tid == 0) layer_mma(tmem, 0, Atile, sm + F_W3, mbar);
    ok = __syncthreads_and(tc::mbar_wait(mbar, phase));
    phase ^= 1u;
    tc::fence_after();
    if (!ok) break;
    {
      float v[32];
      tc::tmem_ld32(tl + (uint32_t)col0, v);
      const float scale = sc[row];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float4 w;
        w.x = (v[4 * u] + bs[128 + col0 + 4 * u]) * scale;
        w.y = (v[4 * u + 1] + bs[128 + col0 + 4 * u + 1]) * scale;
        w.z = (v[4 * u + 2] + bs[128 + col0 + 4 * u + 2]) * scale;
        w.w = (v[4 * u + 3] + bs[128 + col0 + 4 * u + 3]) * scale;
        *reinterpret_cast<float4*>(St + row * SS + col0 + 4 * u) = w;
      }
    }
    tc::fence_before();
    __syncthreads();
    // owner-selected update of x, node jn of cells cq, cq + 4, ..
    if (node_ok)
#pragma unroll 8
      for (int u = 0; u < FC / 4; ++u) {
        const int i = cq + 4 * u;
        if ((own[i] >> nslot) & 1u) add_global(x + gs[i * NSLOT + nslot] + noff, (T)St[i * SS + jn]);
      }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicAdd(&g_wait_timeouts, 1u);
    // once more for the copies and products in flight
    tc::mbar_wait(wbar, 0);
    for (int b = 0; b < 2; ++b)
      if (gout >> b & 1u) tc::mbar_wait(gbar + b, gpar >> b & 1u);
    tc::mbar_wait(mbar, phase ^ 1u);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

inline int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  return (int)std::max<int64_t>(g, 1);
}

}  // namespace

void launch_cell_gather(int k, const double* v, const int32_t* cells, int64_t n, const int32_t* gstart,
                        const CellMeta* meta, double* out, cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)((n + 7) / 8);
  switch (k) {
    case 1: cell_gather_kernel<1><<<grid, 256, 0, s>>>(v, cells, n, gstart, meta, out); break;
    case 2: cell_gather_kernel<2><<<grid, 256, 0, s>>>(v, cells, n, gstart, meta, out); break;
    case 3: cell_gather_kernel<3><<<grid, 256, 0, s>>>(v, cells, n, gstart, meta, out); break;
    case 4: cell_gather_kernel<4><<<grid, 256, 0, s>>>(v, cells, n, gstart, meta, out); break;
    default: return;
  }
  note_launches(1);
}

void launch_mlp_samples(const double* R, const double* E, const double* D, const int32_t* cells, int64_t n, int n3,
                        const CellMeta* meta, double dom, double abar, float* X, float* T, float* W, cudaStream_t s) {
  if (n <= 0) return;
  samples_kernel<<<(int)((n * 32 + 255) / 256), 256, 0, s>>>(R, E, D, cells, n, n3, meta, dom, abar, X, T, W);
  note_launches(1);
}

void launch_mlp_dfeat(const double* D, int64_t n, int n3, const CellMeta* meta, double dom, double abar, void* out,
                      cudaStream_t s) {
  if (n <= 0) return;
  dfeat_kernel<<<(int)((n * MLP_DF + 255) / 256), 256, 0, s>>>(D, n, n3, meta, dom, abar, static_cast<bf16*>(out));
  note_launches(1);
}

void launch_gemm_bf16(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return;
  dim3 grid((g.N + GN - 1) / GN, (g.M + GM - 1) / GM);
  gemm_tc_kernel<<<grid, GTH, 0, s>>>(g);
  note_launches(1);
}

void launch_gelu(const float* Z, float* H, int64_t n, cudaStream_t s) {
  gelu_kernel<<<grid_for(n, 256), 256, 0, s>>>(Z, H, n);
  note_launches(1);
}

void launch_gelu_bwd(const float* dH, const float* Z, float* dZ, int64_t n, cudaStream_t s) {
  gelu_bwd_kernel<<<grid_for(n, 256), 256, 0, s>>>(dH, Z, dZ, n);
  note_launches(1);
}

void launch_mse(const float* Y, const float* T, const float* W, float* dY, int B, int m, float* loss,
                cudaStream_t s) {
  loss_kernel<<<1, 256, 0, s>>>(Y, T, W, dY, B, m, loss);
  note_launches(1);
}

void launch_colsum(const float* X, int M, int N, float* out, cudaStream_t s) {
  colsum_kernel<<<(N + 127) / 128, 128, 0, s>>>(X, M, N, out);
  note_launches(1);
}

void launch_gather_rows(const float* X, int64_t ld, const int32_t* idx, int B, float* out, cudaStream_t s) {
  const int64_t n = (int64_t)B * ld;
  gather_rows_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(X, ld, idx, B, out);
  note_launches(1);
}

void launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float bc1, float bc2,
                 cudaStream_t s) {
  adam_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, bc1, bc2);
  note_launches(1);
}

size_t mlp_fused_smem_bytes() { return F_BYTES; }
size_t mlp_image_bytes() { return F_IMG; }

void launch_mlp_prepare(const float* params, const uint16_t* dfeat, int64_t n_cells, void* image, float* dproj,
                        cudaStream_t s) {
  mlp_pack_kernel<<<64, 256, 0, s>>>(params, static_cast<unsigned char*>(image));
  note_launches(1);
  // dproj = b1 + dfeat[:, 0..124] W1[:, 125..249]^T (bf16 operands, fp32 accumulation)
  const float* W1 = params;
  const float* b1 = W1 + 128 * 250;
  GemmArgs g{nullptr, MLP_DF, 1, W1 + FN3, 1, 250, dproj, 128, b1, (int)n_cells, 128, FN3};
  g.Ab = dfeat;
  launch_gemm_bf16(g, s);
}

unsigned int wait_timeouts(bool reset) {
  unsigned int n = 0;
  if (cudaMemcpyFromSymbol(&n, g_wait_timeouts, sizeof(n)) != cudaSuccess) return ~0u;
  if (reset) {
    const unsigned int z = 0;
    if (cudaMemcpyToSymbol(g_wait_timeouts, &z, sizeof(z)) != cudaSuccess) return ~0u;
  }
  return n;
}

cudaError_t launch_mlp_correct(const MlpFused& P, bool fp64, const void* r, void* x, cudaStream_t s) {
  if (P.n_cells <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(P.wimg) & 15) || (reinterpret_cast<uintptr_t>(P.dproj) & 15))
    return cudaErrorMisalignedAddress;
  const int64_t nb = (P.n_cells + FC - 1) / FC;
  const int grid = (int)std::min<int64_t>(nb, device_sm_count());
  cudaError_t e;
  if (fp64) {
    e = smem_allow(mlp_correct_kernel<double>, F_BYTES);
    if (e != cudaSuccess) return e;
    mlp_correct_kernel<double><<<grid, FT, F_BYTES, s>>>(P, static_cast<const double*>(r), static_cast<double*>(x));
  } else {
    e = smem_allow(mlp_correct_kernel<float>, F_BYTES);
    if (e != cudaSuccess) return e;
    mlp_correct_kernel<float><<<grid, FT, F_BYTES, s>>>(P, static_cast<const float*>(r), static_cast<float*>(x));
  }
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace gcmg
