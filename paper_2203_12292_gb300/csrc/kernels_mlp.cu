// Kernels of the learned per-cell smoother, an extension outside the paper
// (the paper smooths with Chebyshev around point Jacobi, Sec. 3.3).
//
// * cell gather: the values of a free-DoF vector at the (k+1)^3 support
//   points of a list of cells, hanging points interpolated (G_e, then C_e of
//   Eq. 2), in fp64.
// * training: a bf16 tensor-core GEMM (mma.sync m16n8k16, fp32 accumulation)
//   with arbitrary operand strides, so that every product of the forward and
//   backward passes (X W^T, dY^T H, dY W) is one launch; GELU, loss, column
//   sums and Adam as elementwise kernels.
// * inference: one persistent kernel per application.  Each CTA keeps the
//   three weight matrices in shared memory (bf16) and loops over batches of
//   64 cells: gather the residual, interpolate hanging points, scale by the
//   cell norm, run the three layers on the tensor cores, and add the
//   correction to the DoFs the cell owns (each DoF has exactly one owner
//   cell, so there are no races and no atomics).
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"

namespace gcmg {

GCMG_DEFINE_UPLOAD(upload_tables_mlp)

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (lower address, low half) = lo
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t lds32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// D = A B + D for one 16x8 tile, A 16x16 (row-major fragments), B 16x8
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// one warp: acc[nt] += A[16 x K] * Bt[8 nt .. 8 nt + 7][K]^T, both operands
// in shared memory with k contiguous (row strides lda, ldb even, K multiple
// of 16).  Fragment layout of m16n8k16: lane = 4 g + t holds A rows g, g + 8
// at columns 2t, 2t+1, 2t+8, 2t+9, B column g at rows 2t, 2t+1, 2t+8, 2t+9,
// and D rows g, g + 8 at columns 2t, 2t+1.
template <int NT>
__device__ __forceinline__ void warp_gemm(const bf16* A, int lda, const bf16* Bt, int ldb, int K,
                                          float (&acc)[NT][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const bf16* pa = A + g * lda + 2 * t;
  const bf16* pb = Bt + g * ldb + 2 * t;
#pragma unroll 2
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    a[0] = lds32(pa + k0);
    a[1] = lds32(pa + 8 * lda + k0);
    a[2] = lds32(pa + k0 + 8);
    a[3] = lds32(pa + 8 * lda + k0 + 8);
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const bf16* q = pb + nt * 8 * ldb + k0;
      mma_bf16(acc[nt], a, lds32(q), lds32(q + 8));
    }
  }
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
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
constexpr int GT = 64, GK = 32, GKS = GK + 8;

__global__ void __launch_bounds__(256) gemm_bf16_kernel(GemmArgs g) {
  __shared__ __align__(16) bf16 As[GT * GKS];
  __shared__ __align__(16) bf16 Bs[GT * GKS];
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int warp = threadIdx.x >> 5, rb = warp & 3, ch = warp >> 2;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
  for (int k0 = 0; k0 < g.K; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += blockDim.x) {
      const int i = e / GK, kk = e - i * GK, k = k0 + kk;
      const int m = m0 + i, nn = n0 + i;
      const float va = (m < g.M && k < g.K) ? g.A[(int64_t)m * g.sam + (int64_t)k * g.sak] : 0.0f;
      const float vb = (nn < g.N && k < g.K) ? g.B[(int64_t)k * g.sbk + (int64_t)nn * g.sbn] : 0.0f;
      As[i * GKS + kk] = __float2bfloat16_rn(va);
      Bs[i * GKS + kk] = __float2bfloat16_rn(vb);
    }
    __syncthreads();
    warp_gemm<4>(As + rb * 16 * GKS, GKS, Bs + ch * 32 * GKS, GKS, GK, acc);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, gg = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int m = m0 + rb * 16 + gg + (e >> 1) * 8;
      const int nn = n0 + ch * 32 + nt * 8 + 2 * t + (e & 1);
      if (m < g.M && nn < g.N) g.C[(int64_t)m * g.ldc + nn] = acc[nt][e] + (g.bias ? g.bias[nn] : 0.0f);
    }
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
constexpr int FK = 4, FN3 = 125, FC = 64, FT = 512;  // degree, nodes, cells per batch, threads
constexpr int XS = 264, HS = 136, SS = 128;           // row strides: X / W1 (bf16), H / W2 / W3 (bf16), staging (fp32)
// shared memory = [weight image (W1, W2, W3 bf16, biases fp32) | X | H | staging | per-cell data]
constexpr size_t F_W1 = 0;
constexpr size_t F_W2 = F_W1 + 128 * XS * 2;
constexpr size_t F_W3 = F_W2 + 128 * HS * 2;
constexpr size_t F_B = F_W3 + 128 * HS * 2;
constexpr size_t F_IMG = F_B + 3 * 128 * 4;  // bytes of the packed weight image
constexpr size_t F_X = F_IMG;
constexpr size_t F_H = F_X + FC * XS * 2;
constexpr size_t F_ST = F_H + FC * HS * 2;
constexpr size_t F_SC = F_ST + FC * SS * 4;
constexpr size_t F_SI = F_SC + FC * 4;
constexpr size_t F_GS = F_SI + FC * 4;
constexpr size_t F_OWN = F_GS + FC * NSLOT * 4;
constexpr size_t F_MK = F_OWN + FC * 4;
constexpr size_t F_BYTES = F_MK + FC * 2;
static_assert(F_BYTES <= 232448, "fused MLP kernel exceeds the shared memory of a CTA");
static_assert(F_IMG % 16 == 0 && F_X % 16 == 0 && (XS * 2) % 16 == 0, "16-byte aligned rows");
constexpr int GPT = (FC * FN3 + FT - 1) / FT;  // gathered values per thread and batch
constexpr int GH = 8;                            // of them in flight at once

// packed bf16 weight image in the shared-memory layout of the fused kernel
// (feature columns: residual 0..124, diagonal 128..252; padding zero)
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
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 128 * XS; e += stride) {
    const int n = e / XS, k = e - n * XS;
    const float v = k < 125 ? W1[n * 250 + k] : ((k >= 128 && k < 253) ? W1[n * 250 + k - 3] : 0.0f);
    W1s[e] = __float2bfloat16_rn(v);
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 128 * HS; e += stride) {
    const int n = e / HS, k = e - n * HS;
    W2s[e] = __float2bfloat16_rn(k < 128 ? W2[n * 128 + k] : 0.0f);
    W3s[e] = __float2bfloat16_rn((k < 128 && n < 125) ? W3[n * 128 + k] : 0.0f);
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 128; e += stride) {
    bs[e] = b1[e];
    bs[128 + e] = b2[e];
    bs[256 + e] = e < 125 ? b3[e] : 0.0f;
  }
}

template <typename T>
__global__ void __launch_bounds__(FT, 1) mlp_correct_kernel(MlpFused P, const T* __restrict__ r, T* x) {
  extern __shared__ __align__(16) unsigned char smem[];
  const bf16* W1s = reinterpret_cast<const bf16*>(smem + F_W1);
  const bf16* W2s = reinterpret_cast<const bf16*>(smem + F_W2);
  const bf16* W3s = reinterpret_cast<const bf16*>(smem + F_W3);
  const float* bs = reinterpret_cast<const float*>(smem + F_B);
  bf16* Xs = reinterpret_cast<bf16*>(smem + F_X);
  bf16* Hs = reinterpret_cast<bf16*>(smem + F_H);
  float* St = reinterpret_cast<float*>(smem + F_ST);
  float* sc = reinterpret_cast<float*>(smem + F_SC);
  float* si = reinterpret_cast<float*>(smem + F_SI);
  int32_t* gs = reinterpret_cast<int32_t*>(smem + F_GS);
  uint32_t* own = reinterpret_cast<uint32_t*>(smem + F_OWN);
  uint16_t* mk = reinterpret_cast<uint16_t*>(smem + F_MK);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // the packed weight image, once per CTA (16-byte copies, all in flight)
  {
    constexpr int NV = (int)(F_IMG / 16), PER = (NV + FT - 1) / FT, CH = 6;
    const uint4* src = reinterpret_cast<const uint4*>(P.wimg);
    uint4* dst = reinterpret_cast<uint4*>(smem);
#pragma unroll 1
    for (int u0 = 0; u0 < PER; u0 += CH) {
      uint4 v[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u)
        if (u0 + u < PER && tid + (u0 + u) * FT < NV) v[u] = src[tid + (u0 + u) * FT];
#pragma unroll
      for (int u = 0; u < CH; ++u)
        if (u0 + u < PER && tid + (u0 + u) * FT < NV) dst[tid + (u0 + u) * FT] = v[u];
    }
  }

  const int rb = warp & 3, cq = warp >> 2;  // rows 16 rb .., columns 32 cq ..
  const int g = lane >> 2, t4 = lane & 3;
  const int64_t nbatch = (P.n_cells + FC - 1) / FC;
  for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
    const int64_t c0 = bt * FC;
    const int nc = (int)(P.n_cells - c0 < FC ? P.n_cells - c0 : FC);
    for (int e = tid; e < FC * NSLOT; e += FT) gs[e] = e < nc * NSLOT ? P.gstart[c0 * NSLOT + e] : -1;
    if (tid < FC) {
      mk[tid] = tid < nc ? P.meta[c0 + tid].mask : 0;
      own[tid] = tid < nc ? P.own[c0 + tid] : 0u;
    }
    __syncthreads();
    // gather the residual at the 125 nodes of every cell (GH loads in flight per thread)
#pragma unroll 1
    for (int u0 = 0; u0 < GPT; u0 += GH) {
      float v[GH];
#pragma unroll
      for (int u = 0; u < GH; ++u) {
        const int e = tid + (u0 + u) * FT;
        v[u] = 0.0f;
        if (e < FC * FN3) {
          const int i = e / FN3, j = e - i * FN3;
          int slot, off;
          node_slot<FK>(j % 5, (j / 5) % 5, j / 25, slot, off);
          const int32_t base = gs[i * NSLOT + slot];
          if (base >= 0) v[u] = (float)r[base + off];
        }
      }
#pragma unroll
      for (int u = 0; u < GH; ++u) {
        const int e = tid + (u0 + u) * FT;
        if (e < FC * FN3) {
          const int i = e / FN3, j = e - i * FN3;
          St[i * SS + j] = v[u];
        }
      }
    }
    const int hang = __syncthreads_or(tid < nc && (mk[tid] & MASK_HANG));
    if (hang) hanging_all<FK, false, float, SS>(St, mk, nc);
    // cell norms and scales: warp w handles cells 4w .. 4w + 3
#pragma unroll
    for (int q = 0; q < FC / (FT / 32); ++q) {
      const int i = warp * (FC / (FT / 32)) + q;
      float ss = 0.0f;
      for (int j = lane; j < FN3; j += 32) ss += St[i * SS + j] * St[i * SS + j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) {
        const float s = sqrtf(ss);
        const float h = i < nc ? (float)(P.dom / (double)(1u << P.meta[c0 + i].level)) : 1.0f;
        si[i] = s > 0.0f ? 1.0f / s : 0.0f;
        sc[i] = s / (h * (float)P.abar);
      }
    }
    __syncthreads();
    // features: bf16(r / s) in columns 0..127, the diagonal features in 128..255
    for (int e = tid; e < FC * 64; e += FT) {
      const int i = e >> 6, j = (e & 63) * 2;
      const float v0 = j < FN3 ? St[i * SS + j] * si[i] : 0.0f;
      const float v1 = j + 1 < FN3 ? St[i * SS + j + 1] * si[i] : 0.0f;
      *reinterpret_cast<uint32_t*>(Xs + i * XS + j) = pack_bf16(v0, v1);
    }
    for (int e = tid; e < FC * 16; e += FT) {
      const int i = e >> 4, q = e & 15;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (i < nc) v = reinterpret_cast<const uint4*>(P.dfeat + (c0 + i) * MLP_DF)[q];
      *reinterpret_cast<uint4*>(Xs + i * XS + 128 + q * 8) = v;
    }
    __syncthreads();
    // layer 1: H = gelu(X W1^T + b1)
    {
      float acc[4][4] = {};
      warp_gemm<4>(Xs + rb * 16 * XS, XS, W1s + cq * 32 * XS, XS, 256, acc);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int col = cq * 32 + nt * 8 + 2 * t4, row = rb * 16 + g;
        *reinterpret_cast<uint32_t*>(Hs + row * HS + col) =
            pack_bf16(gelu_f(acc[nt][0] + bs[col]), gelu_f(acc[nt][1] + bs[col + 1]));
        *reinterpret_cast<uint32_t*>(Hs + (row + 8) * HS + col) =
            pack_bf16(gelu_f(acc[nt][2] + bs[col]), gelu_f(acc[nt][3] + bs[col + 1]));
      }
    }
    __syncthreads();
    // layer 2: X[:, 0..127] = gelu(H W2^T + b2)
    {
      float acc[4][4] = {};
      warp_gemm<4>(Hs + rb * 16 * HS, HS, W2s + cq * 32 * HS, HS, 128, acc);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int col = cq * 32 + nt * 8 + 2 * t4, row = rb * 16 + g;
        *reinterpret_cast<uint32_t*>(Xs + row * XS + col) =
            pack_bf16(gelu_f(acc[nt][0] + bs[128 + col]), gelu_f(acc[nt][1] + bs[128 + col + 1]));
        *reinterpret_cast<uint32_t*>(Xs + (row + 8) * XS + col) =
            pack_bf16(gelu_f(acc[nt][2] + bs[128 + col]), gelu_f(acc[nt][3] + bs[128 + col + 1]));
      }
    }
    __syncthreads();
    // layer 3: correction c = (X W3^T + b3) s / (h a)
    {
      float acc[4][4] = {};
      warp_gemm<4>(Xs + rb * 16 * XS, XS, W3s + cq * 32 * HS, HS, 128, acc);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int col = cq * 32 + nt * 8 + 2 * t4 + (e & 1), row = rb * 16 + g + (e >> 1) * 8;
          if (col < FN3) St[row * SS + col] = (acc[nt][e] + bs[256 + col]) * sc[row];
        }
    }
    __syncthreads();
    // owner-selected update of x (GH loads in flight per thread)
#pragma unroll 1
    for (int u0 = 0; u0 < GPT; u0 += GH) {
      int idx[GH];
      T xv[GH];
#pragma unroll
      for (int u = 0; u < GH; ++u) {
        const int e = tid + (u0 + u) * FT;
        idx[u] = -1;
        if (e < FC * FN3) {
          const int i = e / FN3, j = e - i * FN3;
          int slot, off;
          node_slot<FK>(j % 5, (j / 5) % 5, j / 25, slot, off);
          if (i < nc && ((own[i] >> slot) & 1u)) idx[u] = gs[i * NSLOT + slot] + off;
        }
        if (idx[u] >= 0) xv[u] = x[idx[u]];
      }
#pragma unroll
      for (int u = 0; u < GH; ++u) {
        const int e = tid + (u0 + u) * FT;
        if (idx[u] >= 0) {
          const int i = e / FN3, j = e - i * FN3;
          x[idx[u]] = xv[u] + (T)St[i * SS + j];
        }
      }
    }
    __syncthreads();
  }
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
  dim3 grid((g.N + GT - 1) / GT, (g.M + GT - 1) / GT);
  gemm_bf16_kernel<<<grid, 256, 0, s>>>(g);
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

void launch_mlp_pack(const float* params, void* image, cudaStream_t s) {
  mlp_pack_kernel<<<64, 256, 0, s>>>(params, static_cast<unsigned char*>(image));
  note_launches(1);
}

cudaError_t launch_mlp_correct(const MlpFused& P, bool fp64, const void* r, void* x, cudaStream_t s) {
  if (P.n_cells <= 0) return cudaSuccess;
  static int n_sm = 0;
  static bool attr_set[2] = {false, false};
  if (!n_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (n_sm <= 0) n_sm = 152;
  }
  const int64_t nb = (P.n_cells + FC - 1) / FC;
  const int grid = (int)std::min<int64_t>(nb, n_sm);
  cudaError_t e;
  if (fp64) {
    if (!attr_set[1]) {
      e = cudaFuncSetAttribute(mlp_correct_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F_BYTES);
      if (e != cudaSuccess) return e;
      attr_set[1] = true;
    }
    mlp_correct_kernel<double><<<grid, FT, F_BYTES, s>>>(P, static_cast<const double*>(r), static_cast<double*>(x));
  } else {
    if (!attr_set[0]) {
      e = cudaFuncSetAttribute(mlp_correct_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F_BYTES);
      if (e != cudaSuccess) return e;
      attr_set[0] = true;
    }
    mlp_correct_kernel<float><<<grid, FT, F_BYTES, s>>>(P, static_cast<const float*>(r), static_cast<float*>(x));
  }
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace gcmg
