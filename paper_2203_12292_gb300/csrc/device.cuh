// Device-side helpers shared by the CUDA translation units of libgcmg:
// per-degree constant tables and the block-cooperative steps of the cell
// pipeline of Eq. 2 (gather with constraints, sum-factorised cell operator,
// transposed constraints, scatter).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <stdexcept>
#include <unordered_map>

#include "dwl.h"
#include "host.h"
#include "internal.h"

namespace gcmg {

constexpr int BLOCK = 256;

// Programmatic dependent launch.  Every kernel of the multigrid cycle is
// launched with launch_pdl and starts with pdl_begin(): it waits until the
// preceding kernel of the stream has completed and its writes are visible,
// then lets the next kernel be scheduled.  Stream order and results are
// unchanged; the launch of a kernel overlaps the tail of its predecessor
// (the many small kernels of the coarse levels are bound by launch latency).
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// asynchronous global -> shared copies (cp.async): a thread issues all its
// copies of a tile before waiting once, so the latency of the tile's loads is
// paid once instead of once per loop iteration
template <typename T>
__device__ __forceinline__ void cp_async(T* sdst, const T* gsrc) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
// 16 bytes; both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Dynamic shared memory above the 48 KB default needs a per-kernel limit
// (cudaFuncAttributeMaxDynamicSharedMemorySize).  It is raised once per kernel
// and device, under a lock, to the device's opt-in maximum, and never lowered:
// every launch, every replay of a captured launch and launches from several
// host threads then see the same limit whatever level was launched last.
// Returns cudaErrorInvalidValue for a request above that maximum; a failure is
// also recorded for the calling entry point (note_launch_error).
inline cudaError_t smem_allow_impl(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> limit[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && (dev < 0 || dev >= 64)) e = cudaErrorInvalidDevice;
  if (e != cudaSuccess) {
    note_launch_error(e);
    return e;
  }
  size_t lim = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = limit[dev].find(func);
    if (it == limit[dev].end()) {
      int optin = 0;
      cudaFuncAttributes fa{};
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
      const int dyn = optin - (int)fa.sharedSizeBytes;
      if (e == cudaSuccess && dyn > 0)
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
      if (e != cudaSuccess) {
        note_launch_error(e);
        return e;
      }
      it = limit[dev].emplace(func, dyn > 0 ? (size_t)dyn : 0).first;
    }
    lim = it->second;
  }
  if (bytes > lim) {
    note_launch_error(cudaErrorInvalidValue);
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}
template <typename KERN>
inline cudaError_t smem_allow(KERN kernel, size_t bytes) {
  return smem_allow_impl(reinterpret_cast<const void*>(kernel), bytes);
}

// launch with programmatic stream serialisation (see pdl_begin); a rejected
// launch is returned and recorded for the calling entry point.  While a
// device-work-list recorder is installed on this thread, the launch is
// recorded instead (cudaErrorNotSupported for a kernel the persistent kernel
// does not run).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  if (dwl_recording()) {
    const bool ok = grid.y == 1 && grid.z == 1 && block.y == 1 && block.z == 1 &&
                    dwl_record<KArgs...>(reinterpret_cast<const void*>(kernel), grid.x, block.x, smem,
                                         static_cast<KArgs>(args)...);
    const cudaError_t e = ok ? cudaSuccess : cudaErrorNotSupported;
    note_launch_error(e);
    return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
  note_launch_error(e);
  return e;
}

// a double-float value hi + lo (arithmetic further below)
struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};

template <typename T>
struct DevTables {
  T B[NMAX][NMAX];          // fast-diagonalisation transform, rows = modes
  T lam[NMAX];              // generalised eigenvalues of (K, M)
  T I[2][NMAX][NMAX];       // child-side interpolation for hanging nodes
  T Pq[NMAX][NMAX];         // Lagrange values at Gauss points
  T gq[NMAX], gw[NMAX];     // Gauss points and weights on [0,1]
  T Ph[2 * KMAX + 1][NMAX]; // h-prolongation onto the 2k+1 child nodes
  T Pp[NMAX][NMAX];         // p-prolongation from degree floor(k/2) to k
  T Be[NMAX][NMAX];         // rows of B reordered: symmetric modes first, then antisymmetric
  T lame[NMAX];             // eigenvalues in the same order
  T lam3[(KMAX + 1) * (KMAX + 1) * (KMAX + 1)];  // lame[a] + lame[b] + lame[c], a fastest
  T xi[NMAX];               // Gauss-Lobatto support points on [0,1]
  T Dq[NMAX][NMAX];         // collocation derivative on the Gauss points: Dq[i][j] = L'_j(gq_i)
};

// every translation unit holds its own copy of the tables (no relocatable
// device code); each one is filled by that unit's upload function
static __constant__ DevTables<double> c_td[KMAX + 1];
static __constant__ DevTables<float> c_tf[KMAX + 1];
// low parts of the fp64 tables: c_tf + c_tflo represents every entry to
// about 2^-48 (double-float constants)
static __constant__ DevTables<float> c_tflo[KMAX + 1];
// the fp64 tables as double-float pairs (the mapped fp64 operator)
static __constant__ DevTables<df> c_tdf[KMAX + 1];

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
template <>
__device__ __forceinline__ const DevTables<df>& tab<df>(int k) {
  return c_tdf[k];
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
      d.xi[i] = b.xi[i];
      // derivative of the Lagrange polynomial L_j on the k+1 Gauss points at gq_i
      for (int j = 0; j <= k; ++j) {
        double dsum = 0.0;
        if (i <= k)
          for (int c = 0; c <= k; ++c) {
            if (c == j) continue;
            double term = 1.0 / (b.gq[j] - b.gq[c]);
            for (int m = 0; m <= k; ++m)
              if (m != j && m != c) term *= (b.gq[i] - b.gq[m]) / (b.gq[j] - b.gq[m]);
            dsum += term;
          }
        d.Dq[i][j] = dsum;
      }
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
    {
      // even-odd order of the modes: rows of B are symmetric or antisymmetric
      // under x -> 1 - x (the 1D pencil (K, M) is persymmetric)
      const int n = k + 1;
      int order[NMAX], ne = 0, no = 0, odd[NMAX];
      for (int r = 0; r < n; ++r) {
        double se = 0, so = 0, mx = 0;
        for (int j = 0; j < n; ++j) {
          se = std::max(se, std::fabs(b.B[r][j] - b.B[r][n - 1 - j]));
          so = std::max(so, std::fabs(b.B[r][j] + b.B[r][n - 1 - j]));
          mx = std::max(mx, std::fabs(b.B[r][j]));
        }
        if (se <= 1e-9 * mx)
          order[ne++] = r;
        else if (so <= 1e-9 * mx)
          odd[no++] = r;
        else
          throw std::runtime_error("basis mode without parity");
      }
      if (ne != (n + 1) / 2 || no != n / 2) throw std::runtime_error("unexpected mode parities");
      for (int i = 0; i < no; ++i) order[ne + i] = odd[i];
      for (int r = 0; r < n; ++r) {
        d.lame[r] = b.lam[order[r]];
        for (int j = 0; j < n; ++j) d.Be[r][j] = b.B[order[r]][j];
      }
      for (int c = 0; c < n; ++c)
        for (int bb = 0; bb < n; ++bb)
          for (int a = 0; a < n; ++a) d.lam3[a + n * (bb + n * c)] = d.lame[a] + d.lame[bb] + d.lame[c];
    }
    DevTables<float>& f = tf[k];
    const double* src = reinterpret_cast<const double*>(&d);
    float* dstf = reinterpret_cast<float*>(&f);
    static_assert(sizeof(DevTables<double>) == 2 * sizeof(DevTables<float>), "table layout");
    for (size_t i = 0; i < sizeof(DevTables<double>) / sizeof(double); ++i) dstf[i] = (float)src[i];
  }
}

// host: the fp64 tables split into double-float pairs
static inline void fill_tables_df(const DevTables<double>* td, DevTables<df>* out) {
  static_assert(sizeof(DevTables<df>) == sizeof(DevTables<double>), "table layout");
  for (int k = 0; k <= KMAX; ++k) {
    const double* d = reinterpret_cast<const double*>(&td[k]);
    float* o = reinterpret_cast<float*>(&out[k]);
    for (size_t i = 0; i < sizeof(DevTables<double>) / sizeof(double); ++i) {
      const float h = (float)d[i];
      o[2 * i] = h;
      o[2 * i + 1] = (float)(d[i] - (double)h);
    }
  }
}

// host: low parts tflo = fp32(td - tf) of the fp64 tables
static inline void fill_tables_lo(const DevTables<double>* td, const DevTables<float>* tf, DevTables<float>* lo) {
  for (int k = 0; k <= KMAX; ++k) {
    const double* d = reinterpret_cast<const double*>(&td[k]);
    const float* f = reinterpret_cast<const float*>(&tf[k]);
    float* l = reinterpret_cast<float*>(&lo[k]);
    for (size_t i = 0; i < sizeof(DevTables<double>) / sizeof(double); ++i) l[i] = (float)(d[i] - (double)f[i]);
  }
}

#define GCMG_DEFINE_UPLOAD(name)                                             \
  void name() {                                                              \
    static DevTables<double> td[KMAX + 1];                                   \
    static DevTables<float> tf[KMAX + 1];                                    \
    static DevTables<float> tl[KMAX + 1];                                    \
    static DevTables<df> tdf[KMAX + 1];                                      \
    fill_tables(td, tf);                                                     \
    fill_tables_lo(td, tf, tl);                                              \
    fill_tables_df(td, tdf);                                                 \
    cudaMemcpyToSymbol(c_td, td, sizeof(td));                                \
    cudaMemcpyToSymbol(c_tf, tf, sizeof(tf));                                \
    cudaMemcpyToSymbol(c_tflo, tl, sizeof(tl));                              \
    cudaMemcpyToSymbol(c_tdf, tdf, sizeof(tdf));                             \
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
template <int K, int D, bool TRANS, typename T, int CS = (K + 1) * (K + 1) * (K + 1)>
__device__ __forceinline__ void hanging_dir(T* cb, const uint16_t* sm_mask, int ncells) {
  constexpr int N = K + 1, N2 = N * N, N3 = CS;
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

template <int K, bool TRANS, typename T, int CS = (K + 1) * (K + 1) * (K + 1)>
__device__ __forceinline__ void hanging_all(T* cb, const uint16_t* sm_mask, int ncells) {
  if (!TRANS) {
    hanging_dir<K, 0, false, T, CS>(cb, sm_mask, ncells);
    __syncthreads();
    hanging_dir<K, 1, false, T, CS>(cb, sm_mask, ncells);
    __syncthreads();
    hanging_dir<K, 2, false, T, CS>(cb, sm_mask, ncells);
    __syncthreads();
  } else {
    hanging_dir<K, 2, true, T, CS>(cb, sm_mask, ncells);
    __syncthreads();
    hanging_dir<K, 1, true, T, CS>(cb, sm_mask, ncells);
    __syncthreads();
    hanging_dir<K, 0, true, T, CS>(cb, sm_mask, ncells);
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
  // lam_a + lam_b per z line in shared memory: indexing the constant table
  // with the thread's (a, b) would serialise the warp's constant reads
  __shared__ T s_lab[N2];
  for (int r = threadIdx.x; r < N2; r += blockDim.x) s_lab[r] = tb.lam[r % N] + tb.lam[r / N];
  __syncthreads();
  for (int t = threadIdx.x; t < ncells * N2; t += blockDim.x) {
    const int cell = t / N2, r = t - cell * N2;
    T* p = cb + cell * N3 + r;
    T v[N], w[N];
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = p[c * N2];
    const T hab = sm_h[cell];
    const T lab = s_lab[r];
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

// ---------------------------------------------------------------------------
// register-resident sweeps for one cell held by one thread (array u of
// N^3 values, compile-time indices only so that u stays in registers)
// ---------------------------------------------------------------------------

// forward transform with B along a line (BASE + i*STRIDE), even-odd form:
// symmetric modes from the sums u_j + u_{N-1-j}, antisymmetric ones from
// the differences; results stored in mode order (symmetric modes first)
template <int N, int BASE, int STRIDE, typename T>
__device__ __forceinline__ void eo_forward(T* u, const T (&Be)[NMAX][NMAX]) {
  constexpr int NH = N / 2, NE = (N + 1) / 2;
  T e[NE], o[NH > 0 ? NH : 1];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    e[j] = u[BASE + j * STRIDE] + u[BASE + (N - 1 - j) * STRIDE];
    o[j] = u[BASE + j * STRIDE] - u[BASE + (N - 1 - j) * STRIDE];
  }
  if (N % 2) e[NH] = u[BASE + NH * STRIDE];
#pragma unroll
  for (int r = 0; r < NE; ++r) {
    T s = (N % 2) ? Be[r][NH] * e[NH] : T(0);
#pragma unroll
    for (int j = 0; j < NH; ++j) s += Be[r][j] * e[j];
    u[BASE + r * STRIDE] = s;
  }
#pragma unroll
  for (int r = 0; r < NH; ++r) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < NH; ++j) s += Be[NE + r][j] * o[j];
    u[BASE + (NE + r) * STRIDE] = s;
  }
}

// backward transform with B^T (modes in mode order -> nodal values)
template <int N, int BASE, int STRIDE, typename T>
__device__ __forceinline__ void eo_backward(T* u, const T (&Be)[NMAX][NMAX]) {
  constexpr int NH = N / 2, NE = (N + 1) / 2;
  T E[NE], O[NH > 0 ? NH : 1];
#pragma unroll
  for (int j = 0; j < NE; ++j) {
    T s = T(0);
#pragma unroll
    for (int r = 0; r < NE; ++r) s += Be[r][j] * u[BASE + r * STRIDE];
    E[j] = s;
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    T s = T(0);
#pragma unroll
    for (int r = 0; r < NH; ++r) s += Be[NE + r][j] * u[BASE + (NE + r) * STRIDE];
    O[j] = s;
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    u[BASE + j * STRIDE] = E[j] + O[j];
    u[BASE + (N - 1 - j) * STRIDE] = E[j] - O[j];
  }
  if (N % 2) u[BASE + NH * STRIDE] = E[NH];
}

template <int N, int D, bool FWD, int L = 0, typename T>
__device__ __forceinline__ void eo_sweep(T* u, const T (&Be)[NMAX][NMAX]) {
  if constexpr (L < N * N) {
    constexpr int a = L % N, b = L / N;
    constexpr int BASE = (D == 0) ? N * (a + N * b) : (D == 1 ? a + N * N * b : a + N * b);
    constexpr int STRIDE = (D == 0) ? 1 : (D == 1 ? N : N * N);
    if (FWD)
      eo_forward<N, BASE, STRIDE>(u, Be);
    else
      eo_backward<N, BASE, STRIDE>(u, Be);
    eo_sweep<N, D, FWD, L + 1>(u, Be);
  }
}

// the cell operator h (K x M x M + M x K x M + M x M x K) on one cell in
// registers: B in x, y, z, scale by h (lam_a + lam_b + lam_c), B^T back
template <int K, typename T>
__device__ __forceinline__ void cell_laplace_regs(T* u, T h) {
  constexpr int N = K + 1, N3 = N * N * N;
  const DevTables<T>& tb = tab<T>(K);
  eo_sweep<N, 0, true>(u, tb.Be);
  eo_sweep<N, 1, true>(u, tb.Be);
  eo_sweep<N, 2, true>(u, tb.Be);
#pragma unroll
  for (int n = 0; n < N3; ++n) u[n] *= h * tb.lam3[n];
  eo_sweep<N, 2, false>(u, tb.Be);
  eo_sweep<N, 1, false>(u, tb.Be);
  eo_sweep<N, 0, false>(u, tb.Be);
}

// block-cooperative even-odd sweep along direction D for all cells (one
// thread per line): FWD applies B (nodal values -> modes in mode order),
// otherwise B^T (modes -> nodal values)
template <int K, int D, bool FWD, typename T>
__device__ __forceinline__ void sweep_eo(T* cb, int ncells) {
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  const DevTables<T>& tb = tab<T>(K);
  for (int t = threadIdx.x; t < ncells * N2; t += blockDim.x) {
    const int cell = t / N2, r = t - cell * N2;
    int base, u, v;
    line_geom<N, D>(r, base, u, v);
    T* p = cb + cell * N3 + base;
    if (FWD)
      eo_forward<N, 0, line_stride<N, D>()>(p, tb.Be);
    else
      eo_backward<N, 0, line_stride<N, D>()>(p, tb.Be);
  }
}

// z lines in registers: forward even-odd transform, scaling by
// h (lam_a + lam_b + lam_c) (mode order), backward transform
template <int K, typename T>
__device__ __forceinline__ void sweep_z_scale_eo(T* cb, const T* sm_h, int ncells) {
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  const DevTables<T>& tb = tab<T>(K);
  // the eigenvalue sums in shared memory: indexing the constant table with
  // the thread's line would serialise the warp's constant reads
  __shared__ T s_lam3[N3];
  for (int i = threadIdx.x; i < N3; i += blockDim.x) s_lam3[i] = tb.lam3[i];
  __syncthreads();
  for (int t = threadIdx.x; t < ncells * N2; t += blockDim.x) {
    const int cell = t / N2, r = t - cell * N2;
    T* p = cb + cell * N3 + r;
    T v[N];
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = p[c * N2];
    eo_forward<N, 0, 1>(v, tb.Be);
    const T hab = sm_h[cell];
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] *= hab * s_lam3[r + N2 * c];
    eo_backward<N, 0, 1>(v, tb.Be);
#pragma unroll
    for (int c = 0; c < N; ++c) p[c * N2] = v[c];
  }
}

// the cell operator h (K x M x M + M x K x M + M x M x K) on all cells of
// the block, fast-diagonalisation form.  fp64 (bound by the FP64 pipe on
// GB300) takes the even-odd sweeps, which halve the multiplications; fp32
// (bound by instruction issue) is faster with the plain 5x5 sweeps
constexpr bool FP32_EVEN_ODD = false;

template <int K, typename T>
__device__ __forceinline__ void cell_laplace(T* cb, const T* sm_h, int ncells) {
  if constexpr (sizeof(T) == 8 || FP32_EVEN_ODD) {
    sweep_eo<K, 0, true>(cb, ncells);
    __syncthreads();
    sweep_eo<K, 1, true>(cb, ncells);
    __syncthreads();
    sweep_z_scale_eo<K>(cb, sm_h, ncells);
    __syncthreads();
    sweep_eo<K, 1, false>(cb, ncells);
    __syncthreads();
    sweep_eo<K, 0, false>(cb, ncells);
    __syncthreads();
  } else {
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
}

// ---------------------------------------------------------------------------
// double-float arithmetic (a value = hi + lo, two floats, about 48 bits):
// the fp64 operator runs on the FP32 pipe, several times wider than the FP64
// pipe of GB300.  Error-free transformations (Dekker, Knuth two-sum, and the
// fused multiply-add product error); explicit _rn intrinsics keep the
// compiler from contracting the roundings they rely on.
// ---------------------------------------------------------------------------

__device__ __forceinline__ df df_from(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_norm(float hi, float lo) {  // |lo| small against |hi|
  const float s = __fadd_rn(hi, lo);
  return df{s, __fsub_rn(lo, __fsub_rn(s, hi))};
}

__device__ __forceinline__ df df_add(df a, df b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float z = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
  return df_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * (ch + cl)
__device__ __forceinline__ df df_mulc(df a, float ch, float cl) {
  const float p = __fmul_rn(a.hi, ch);
  float e = __fmaf_rn(a.hi, ch, -p);
  e = __fmaf_rn(a.hi, cl, e);
  e = __fmaf_rn(a.lo, ch, e);
  return df_norm(p, e);
}

__device__ __forceinline__ df df_mul(df a, df b) { return df_mulc(a, b.hi, b.lo); }

// s + a * (ch + cl)
__device__ __forceinline__ df df_fma(df s, df a, float ch, float cl) { return df_add(s, df_mulc(a, ch, cl)); }

// a / b: quotient of the high parts, corrected once by the remainder
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = df_sub(a, df_mulc(b, q1, 0.f));
  return df_norm(q1, __fdiv_rn(r.hi, b.hi));
}

// operators, so that the templated cell pipeline runs in double-float unchanged
__device__ __forceinline__ df operator+(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df operator-(df a, df b) { return df_sub(a, b); }
__device__ __forceinline__ df operator-(df a) { return df_neg(a); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df operator/(df a, df b) { return df_div(a, b); }
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = df_add(a, b); }

// 1D transforms on df lines (BASE + i STRIDE) with the fp64 tables of degree K
template <int K, int STRIDE, bool TRANS>
__device__ __forceinline__ void df_line_apply(df* p, const float (&Mh)[NMAX][NMAX], const float (&Ml)[NMAX][NMAX]) {
  constexpr int N = K + 1;
  df v[N];
#pragma unroll
  for (int a = 0; a < N; ++a) v[a] = p[a * STRIDE];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    df s{0.f, 0.f};
#pragma unroll
    for (int a = 0; a < N; ++a) s = TRANS ? df_fma(s, v[a], Mh[a][i], Ml[a][i]) : df_fma(s, v[a], Mh[i][a], Ml[i][a]);
    p[i * STRIDE] = s;
  }
}

// even-odd forward (B, nodal -> modes in mode order) and backward (B^T)
template <int K, int STRIDE>
__device__ __forceinline__ void df_eo_forward(df* u) {
  constexpr int N = K + 1, NH = N / 2, NE = (N + 1) / 2;
  const float(&Bh)[NMAX][NMAX] = c_tf[K].Be;
  const float(&Bl)[NMAX][NMAX] = c_tflo[K].Be;
  df e[NE], o[NH > 0 ? NH : 1];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    e[j] = df_add(u[j * STRIDE], u[(N - 1 - j) * STRIDE]);
    o[j] = df_sub(u[j * STRIDE], u[(N - 1 - j) * STRIDE]);
  }
  if (N % 2) e[NH] = u[NH * STRIDE];
#pragma unroll
  for (int r = 0; r < NE; ++r) {
    df s = (N % 2) ? df_mulc(e[NH], Bh[r][NH], Bl[r][NH]) : df{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NH; ++j) s = df_fma(s, e[j], Bh[r][j], Bl[r][j]);
    u[r * STRIDE] = s;
  }
#pragma unroll
  for (int r = 0; r < NH; ++r) {
    df s{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NH; ++j) s = df_fma(s, o[j], Bh[NE + r][j], Bl[NE + r][j]);
    u[(NE + r) * STRIDE] = s;
  }
}

template <int K, int STRIDE>
__device__ __forceinline__ void df_eo_backward(df* u) {
  constexpr int N = K + 1, NH = N / 2, NE = (N + 1) / 2;
  const float(&Bh)[NMAX][NMAX] = c_tf[K].Be;
  const float(&Bl)[NMAX][NMAX] = c_tflo[K].Be;
  df E[NE], O[NH > 0 ? NH : 1];
#pragma unroll
  for (int j = 0; j < NE; ++j) {
    df s{0.f, 0.f};
#pragma unroll
    for (int r = 0; r < NE; ++r) s = df_fma(s, u[r * STRIDE], Bh[r][j], Bl[r][j]);
    E[j] = s;
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    df s{0.f, 0.f};
#pragma unroll
    for (int r = 0; r < NH; ++r) s = df_fma(s, u[(NE + r) * STRIDE], Bh[NE + r][j], Bl[NE + r][j]);
    O[j] = s;
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    u[j * STRIDE] = df_add(E[j], O[j]);
    u[(N - 1 - j) * STRIDE] = df_sub(E[j], O[j]);
  }
  if (N % 2) u[NH * STRIDE] = E[NH];
}

// hanging-node interpolation C_e (TRANS: C_e^T) on df cell buffers, one
// direction for all cells of the block
template <int K, int D, bool TRANS>
__device__ __forceinline__ void df_hanging_dir(df* cb, const uint16_t* sm_mask, int ncells) {
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  for (int t = threadIdx.x; t < ncells * N2; t += blockDim.x) {
    const int cell = t / N2, r = t - cell * N2;
    const uint16_t m = sm_mask[cell];
    if (!(m & MASK_HANG)) continue;
    int base, u, v;
    line_geom<N, D>(r, base, u, v);
    if (!line_hangs<K, D>(m, u, v)) continue;
    df* p = cb + cell * N3 + base;
    if ((m >> D) & 1)
      df_line_apply<K, line_stride<N, D>(), TRANS>(p, c_tf[K].I[1], c_tflo[K].I[1]);
    else
      df_line_apply<K, line_stride<N, D>(), TRANS>(p, c_tf[K].I[0], c_tflo[K].I[0]);
  }
}

template <int K, bool TRANS>
__device__ __forceinline__ void df_hanging_all(df* cb, const uint16_t* sm_mask, int ncells) {
  if (!TRANS) {
    df_hanging_dir<K, 0, false>(cb, sm_mask, ncells);
    __syncthreads();
    df_hanging_dir<K, 1, false>(cb, sm_mask, ncells);
    __syncthreads();
    df_hanging_dir<K, 2, false>(cb, sm_mask, ncells);
    __syncthreads();
  } else {
    df_hanging_dir<K, 2, true>(cb, sm_mask, ncells);
    __syncthreads();
    df_hanging_dir<K, 1, true>(cb, sm_mask, ncells);
    __syncthreads();
    df_hanging_dir<K, 0, true>(cb, sm_mask, ncells);
    __syncthreads();
  }
}

}  // namespace gcmg
