// Device-side helpers shared by the CUDA translation units of libgcmg:
// per-degree constant tables and the block-cooperative steps of the cell
// pipeline of Eq. 2 (gather with constraints, sum-factorised cell operator,
// transposed constraints, scatter).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace gcmg {

constexpr int BLOCK = 256;

template <typename T>
struct DevTables {
  T B[NMAX][NMAX];          // fast-diagonalisation transform, rows = modes
  T lam[NMAX];              // generalised eigenvalues of (K, M)
  T I[2][NMAX][NMAX];       // child-side interpolation for hanging nodes
  T Pq[NMAX][NMAX];         // Lagrange values at Gauss points
  T gq[NMAX], gw[NMAX];     // Gauss points and weights on [0,1]
  T Ph[2 * KMAX + 1][NMAX]; // h-prolongation onto the 2k+1 child nodes
  T Pp[NMAX][NMAX];         // p-prolongation from degree floor(k/2) to k
};

// every translation unit holds its own copy of the tables (no relocatable
// device code); each one is filled by that unit's upload function
static __constant__ DevTables<double> c_td[KMAX + 1];
static __constant__ DevTables<float> c_tf[KMAX + 1];

template <typename T>
__device__ __forceinline__ const DevTables<T>& tab(int k);
template <>
__device__ __forceinline__ const DevTables<double>& tab<double>(int k) {
  return c_td[k];
}
template <>
__device__ __forceinline__ const DevTables<float>& tab<float>(int k) {
  return c_tf[k];
}

// host: fill the tables of all degrees from the fp64 1D basis
static inline void fill_tables(DevTables<double>* td, DevTables<float>* tf) {
  for (int k = 0; k <= KMAX; ++k) {
    DevTables<double>& d = td[k];
    d = DevTables<double>{};
    if (k == 0) {
      tf[k] = DevTables<float>{};
      continue;
    }
    const Basis1D& b = basis(k);
    for (int i = 0; i < NMAX; ++i) {
      d.lam[i] = b.lam[i];
      d.gq[i] = b.gq[i];
      d.gw[i] = b.gw[i];
      for (int j = 0; j < NMAX; ++j) {
        d.B[i][j] = b.B[i][j];
        d.I[0][i][j] = b.I[0][i][j];
        d.I[1][i][j] = b.I[1][i][j];
        d.Pq[i][j] = b.Pq[i][j];
      }
    }
    for (int i = 0; i < 2 * KMAX + 1; ++i)
      for (int j = 0; j < NMAX; ++j) d.Ph[i][j] = b.Ph[i][j];
    if (k >= 2) p_prolongation(k, k / 2, d.Pp);
    DevTables<float>& f = tf[k];
    const double* src = reinterpret_cast<const double*>(&d);
    float* dstf = reinterpret_cast<float*>(&f);
    for (size_t i = 0; i < sizeof(DevTables<double>) / sizeof(double); ++i) dstf[i] = (float)src[i];
  }
}

#define GCMG_DEFINE_UPLOAD(name)                                             \
  void name() {                                                              \
    static DevTables<double> td[KMAX + 1];                                   \
    static DevTables<float> tf[KMAX + 1];                                    \
    fill_tables(td, tf);                                                     \
    cudaMemcpyToSymbol(c_td, td, sizeof(td));                                \
    cudaMemcpyToSymbol(c_tf, tf, sizeof(tf));                                \
  }

// entity slot and offset of local node (a,b,c) of a degree-K cell: the slot
// is cx + 3 cy + 9 cz with class 0 (low end), 1 (interior), 2 (high end)
// along each axis; DoFs of an entity are numbered lexicographically (x
// fastest) over its interior axes.
template <int K>
__device__ __forceinline__ void node_slot(int a, int b, int c, int& slot, int& off) {
  const int ca = a == 0 ? 0 : (a == K ? 2 : 1);
  const int cb = b == 0 ? 0 : (b == K ? 2 : 1);
  const int cc = c == 0 ? 0 : (c == K ? 2 : 1);
  slot = ca + 3 * cb + 9 * cc;
  int o = 0, mul = 1;
  if (ca == 1) {
    o += (a - 1);
    mul *= (K - 1);
  }
  if (cb == 1) {
    o += (b - 1) * mul;
    mul *= (K - 1);
  }
  if (cc == 1) o += (c - 1) * mul;
  off = o;
}

// Is the line along direction D through the other two coordinates (u, v)
// (u, v ordered as the remaining axes in increasing order) part of a hanging
// face or edge of a cell with mask m?
template <int K, int D>
__device__ __forceinline__ bool line_hangs(uint16_t m, int u, int v) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const int p1 = (m >> A1) & 1, p2 = (m >> A2) & 1;
  const bool on1 = (u == p1 * K), on2 = (v == p2 * K);
  const bool f1 = (m >> (3 + A1)) & 1, f2 = (m >> (3 + A2)) & 1, e = (m >> (6 + D)) & 1;
  return (f1 && on1) || (f2 && on2) || (e && on1 && on2);
}

// base offset and stride of line r (0..N^2-1) along D in an N^3 buffer, and
// its two other coordinates
template <int N, int D>
__device__ __forceinline__ void line_geom(int r, int& base, int& u, int& v) {
  if (D == 0) {
    u = r % N;  // y
    v = r / N;  // z
    base = N * r;
  } else if (D == 1) {
    u = r % N;  // x
    v = r / N;  // z
    base = u + N * N * v;
  } else {
    u = r % N;  // x
    v = r / N;  // y
    base = r;
  }
}

template <int N, int D>
__host__ __device__ constexpr int line_stride() {
  return D == 0 ? 1 : (D == 1 ? N : N * N);
}

// apply an N x N matrix (row-major, constant memory) to one line in place
template <int N, int STRIDE, bool TRANS, typename T>
__device__ __forceinline__ void line_apply(T* p, const T (&M)[NMAX][NMAX]) {
  T v[N];
#pragma unroll
  for (int a = 0; a < N; ++a) v[a] = p[a * STRIDE];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T s = 0;
#pragma unroll
    for (int a = 0; a < N; ++a) s += (TRANS ? M[a][i] : M[i][a]) * v[a];
    p[i * STRIDE] = s;
  }
}

// one direction of the hanging-node interpolation C_e (TRANS: C_e^T) for all
// cells of the block; cell c has mask sm_mask[c]
template <int K, int D, bool TRANS, typename T>
__device__ __forceinline__ void hanging_dir(T* cb, const uint16_t* sm_mask, int ncells) {
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  const DevTables<T>& tb = tab<T>(K);
  for (int t = threadIdx.x; t < ncells * N2; t += blockDim.x) {
    const int cell = t / N2, r = t - cell * N2;
    const uint16_t m = sm_mask[cell];
    if (!(m & MASK_HANG)) continue;
    int base, u, v;
    line_geom<N, D>(r, base, u, v);
    if (!line_hangs<K, D>(m, u, v)) continue;
    T* p = cb + cell * N3 + base;
    if ((m >> D) & 1)
      line_apply<N, line_stride<N, D>(), TRANS>(p, tb.I[1]);
    else
      line_apply<N, line_stride<N, D>(), TRANS>(p, tb.I[0]);
  }
}

template <int K, bool TRANS, typename T>
__device__ __forceinline__ void hanging_all(T* cb, const uint16_t* sm_mask, int ncells) {
  if (!TRANS) {
    hanging_dir<K, 0, false>(cb, sm_mask, ncells);
    __syncthreads();
    hanging_dir<K, 1, false>(cb, sm_mask, ncells);
    __syncthreads();
    hanging_dir<K, 2, false>(cb, sm_mask, ncells);
    __syncthreads();
  } else {
    hanging_dir<K, 2, true>(cb, sm_mask, ncells);
    __syncthreads();
    hanging_dir<K, 1, true>(cb, sm_mask, ncells);
    __syncthreads();
    hanging_dir<K, 0, true>(cb, sm_mask, ncells);
    __syncthreads();
  }
}

// sweep with the matrix B (or B^T) along direction D for all cells
template <int K, int D, bool TRANS, typename T>
__device__ __forceinline__ void sweep_B(T* cb, int ncells) {
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  const DevTables<T>& tb = tab<T>(K);
  for (int t = threadIdx.x; t < ncells * N2; t += blockDim.x) {
    const int cell = t / N2, r = t - cell * N2;
    int base, u, v;
    line_geom<N, D>(r, base, u, v);
    line_apply<N, line_stride<N, D>(), TRANS>(cb + cell * N3 + base, tb.B);
  }
}

// forward z sweep, scaling by h (lam_a + lam_b + lam_c), backward z sweep,
// all on one z-line held in registers
template <int K, typename T>
__device__ __forceinline__ void sweep_z_scale(T* cb, const T* sm_h, int ncells) {
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  const DevTables<T>& tb = tab<T>(K);
  for (int t = threadIdx.x; t < ncells * N2; t += blockDim.x) {
    const int cell = t / N2, r = t - cell * N2;
    const int a = r % N, b = r / N;
    T* p = cb + cell * N3 + r;
    T v[N], w[N];
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = p[c * N2];
    const T hab = sm_h[cell];
    const T lab = tb.lam[a] + tb.lam[b];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T s = 0;
#pragma unroll
      for (int c = 0; c < N; ++c) s += tb.B[i][c] * v[c];
      w[i] = s * hab * (lab + tb.lam[i]);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T s = 0;
#pragma unroll
      for (int c = 0; c < N; ++c) s += tb.B[c][i] * w[c];
      p[i * N2] = s;
    }
  }
}

// the cell operator h (K x M x M + M x K x M + M x M x K) on all cells
template <int K, typename T>
__device__ __forceinline__ void cell_laplace(T* cb, const T* sm_h, int ncells) {
  sweep_B<K, 0, false>(cb, ncells);
  __syncthreads();
  sweep_B<K, 1, false>(cb, ncells);
  __syncthreads();
  sweep_z_scale<K>(cb, sm_h, ncells);
  __syncthreads();
  sweep_B<K, 1, true>(cb, ncells);
  __syncthreads();
  sweep_B<K, 0, true>(cb, ncells);
  __syncthreads();
}

}  // namespace gcmg
