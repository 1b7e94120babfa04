// Tile kernels of the cell loop of Eq. 2:
//   v = sum_e G_e^T C_e^T S_e^T Q_e S_e C_e G_e x
// and of the two other cell loops built from it: the right-hand side
// b = C^T F (Gauss quadrature of f against the basis) and the Jacobi
// diagonal of Eqs. 3-4.
//
// One thread block processes one tile of consecutive (Morton-ordered) cells:
//   1. the tile's owned DoFs (contiguous) and foreign DoFs are staged from
//      HBM into shared memory (coalesced loads);
//   2. G_e: every cell gathers its (k+1)^3 values from shared memory through
//      its 27 entity starts; hanging faces/edges point to the constraining
//      coarse entity;
//   3. C_e: in-place interpolation along the hanging lines, direction by
//      direction (Sec. 3.2, hanging-node application);
//   4. S^T Q S: for an axis-parallel cube the Laplace cell operator equals
//      h (K x M x M + M x K x M + M x M x K); it is applied in the fast
//      diagonalisation form h B^T^{(x)3} diag(lam_a+lam_b+lam_c) B^{(x)3}:
//      six 1D sweeps, the middle two fused with the scaling in registers;
//   5. C_e^T, then G_e^T into a shared-memory accumulator, sub-colour by
//      sub-colour (cells sharing an entity never add at the same time);
//   6. owned DoFs are written with plain coalesced stores, foreign DoFs are
//      added; tiles are launched colour by colour, the owner of a DoF having
//      the lowest colour, so no atomics are needed and results are
//      bit-reproducible.
#include <cstdio>

#include "device.cuh"
#include "kernels.h"

namespace gcmg {

GCMG_DEFINE_UPLOAD(upload_tables_cell)

namespace {

template <typename T>
struct CellArgs {
  const TileInfo* tiles;
  const int32_t* tile_list;
  const CellMeta* meta;
  const int32_t* foreign;
  const uint16_t* subptr;
  const uint8_t* perm;
  const int32_t* cell_ijk;
  const T* src;
  T* dst;
  double lo, dom;
  int tc;
  int max_local;
  int add;
  const double* modes;
  int n_modes;
  double amp;
  const double* diag_tab;
};

struct SmemLayout {
  size_t meta, h, mask, cb, xs, ys, total;
};

template <typename T>
__host__ __device__ inline SmemLayout smem_layout(int n3, int tc, int max_local) {
  SmemLayout L;
  size_t o = 0;
  L.meta = o;
  o += (size_t)tc * sizeof(CellMeta);
  L.h = o;
  o += (size_t)tc * sizeof(T);
  L.mask = o;
  o += (size_t)tc * sizeof(uint16_t);
  o = (o + 15) & ~(size_t)15;
  L.cb = o;
  o += (size_t)tc * n3 * sizeof(T);
  L.xs = o;
  o += (size_t)max_local * sizeof(T);
  L.ys = o;
  o += (size_t)max_local * sizeof(T);
  L.total = (o + 15) & ~(size_t)15;
  return L;
}

template <int K, typename T, int MODE>
__global__ void __launch_bounds__(BLOCK) cell_kernel(CellArgs<T> A) {
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout SL = smem_layout<T>(N3, A.tc, A.max_local);
  CellMeta* sm_meta = reinterpret_cast<CellMeta*>(smem + SL.meta);
  T* sm_h = reinterpret_cast<T*>(smem + SL.h);
  uint16_t* sm_mask = reinterpret_cast<uint16_t*>(smem + SL.mask);
  T* cb = reinterpret_cast<T*>(smem + SL.cb);
  T* xs = reinterpret_cast<T*>(smem + SL.xs);
  T* ys = reinterpret_cast<T*>(smem + SL.ys);

  const TileInfo ti = A.tiles[A.tile_list[blockIdx.x]];
  const int nc = ti.n_cells;
  const int nloc = ti.n_owned + ti.n_foreign;
  {
    const uint4* g = reinterpret_cast<const uint4*>(A.meta + ti.cell_begin);
    uint4* s = reinterpret_cast<uint4*>(sm_meta);
    for (int i = threadIdx.x; i < nc * 4; i += blockDim.x) s[i] = g[i];
  }
  if (MODE == MODE_VMULT) {
    const T* src = A.src + ti.dof_begin;
    for (int i = threadIdx.x; i < ti.n_owned; i += blockDim.x) xs[i] = src[i];
    const int32_t* fl = A.foreign + ti.foreign_begin;
    for (int i = threadIdx.x; i < ti.n_foreign; i += blockDim.x) xs[ti.n_owned + i] = A.src[fl[i]];
  }
  for (int i = threadIdx.x; i < nloc; i += blockDim.x) ys[i] = T(0);
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    sm_mask[c] = sm_meta[c].mask;
    sm_h[c] = (T)ldexp(A.dom, -(int)sm_meta[c].level);
  }
  if (MODE == MODE_VMULT) {
    // G_e: gather x-lines of every cell
    for (int t = threadIdx.x; t < nc * N2; t += blockDim.x) {
      const int cell = t / N2, r = t - cell * N2;
      const int b = r % N, c = r / N;
      const uint16_t* ls = sm_meta[cell].ls;
      T* out = cb + cell * N3 + N * r;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        int slot, off;
        node_slot<K>(a, b, c, slot, off);
        const uint16_t l = ls[slot];
        out[a] = (l == LS_NONE) ? T(0) : xs[l + off];
      }
    }
  } else if (MODE == MODE_DIAG) {
    __syncthreads();
    for (int t = threadIdx.x; t < nc * N3; t += blockDim.x) {
      const int cell = t / N3, n = t - cell * N3;
      cb[t] = (T)(A.diag_tab[(sm_mask[cell] & 0x1FF) * N3 + n]) * sm_h[cell];
    }
  } else {  // MODE_RHS: h^3 w_q f(x_q) at the Gauss points, then S^T
    __syncthreads();
    const DevTables<T>& tb = tab<T>(K);
    for (int t = threadIdx.x; t < nc * N3; t += blockDim.x) {
      const int cell = t / N3, n = t - cell * N3;
      const int qa = n % N, qb = (n / N) % N, qc = n / N2;
      const int ci = ti.cell_begin + cell;
      const double h = ldexp(A.dom, -(int)sm_meta[cell].level);
      const double x = A.lo + h * (A.cell_ijk[3 * ci + 0] + (double)tab<double>(K).gq[qa]);
      const double y = A.lo + h * (A.cell_ijk[3 * ci + 1] + (double)tab<double>(K).gq[qb]);
      const double z = A.lo + h * (A.cell_ijk[3 * ci + 2] + (double)tab<double>(K).gq[qc]);
      double f = 1.0;
      if (A.n_modes > 0) {
        f = 0.0;
        for (int m = 0; m < A.n_modes; ++m) {
          const double* md = A.modes + 4 * m;
          f += cos(2.0 * M_PI * (md[0] * x + md[1] * y + md[2] * z) + md[3]);
        }
        f *= A.amp;
      }
      const double w = tab<double>(K).gw[qa] * tab<double>(K).gw[qb] * tab<double>(K).gw[qc];
      cb[t] = (T)(w * h * h * h * f);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nc * N2; t += blockDim.x) {
      const int cell = t / N2, r = t - cell * N2;
      line_apply<N, 1, true>(cb + cell * N3 + N * r, tb.Pq);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nc * N2; t += blockDim.x) {
      const int cell = t / N2, r = t - cell * N2;
      int base, u, v;
      line_geom<N, 1>(r, base, u, v);
      line_apply<N, N, true>(cb + cell * N3 + base, tb.Pq);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nc * N2; t += blockDim.x) {
      const int cell = t / N2, r = t - cell * N2;
      line_apply<N, N2, true>(cb + cell * N3 + r, tb.Pq);
    }
  }
  __syncthreads();
  if (MODE == MODE_VMULT) {
    hanging_all<K, false>(cb, sm_mask, nc);  // C_e
    cell_laplace<K>(cb, sm_h, nc);           // S^T Q S
  }
  if (MODE != MODE_DIAG) hanging_all<K, true>(cb, sm_mask, nc);  // C_e^T
  // G_e^T into the shared accumulator, sub-colour by sub-colour
  for (int s = 0; s < ti.n_sub; ++s) {
    const int q0 = A.subptr[ti.sub_begin + s], q1 = A.subptr[ti.sub_begin + s + 1];
    for (int t = threadIdx.x; t < (q1 - q0) * N2; t += blockDim.x) {
      const int q = q0 + t / N2, r = t % N2;
      const int cell = A.perm[ti.cell_begin + q];
      const int b = r % N, c = r / N;
      const uint16_t* ls = sm_meta[cell].ls;
      const T* in = cb + cell * N3 + N * r;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        int slot, off;
        node_slot<K>(a, b, c, slot, off);
        const uint16_t l = ls[slot];
        if (l != LS_NONE) ys[l + off] += in[a];
      }
    }
    __syncthreads();
  }
  // write back: owned DoFs (contiguous) stored, foreign DoFs added
  {
    T* dst = A.dst + ti.dof_begin;
    if (A.add)
      for (int i = threadIdx.x; i < ti.n_owned; i += blockDim.x) dst[i] += ys[i];
    else
      for (int i = threadIdx.x; i < ti.n_owned; i += blockDim.x) dst[i] = ys[i];
    const int32_t* fl = A.foreign + ti.foreign_begin;
    for (int i = threadIdx.x; i < ti.n_foreign; i += blockDim.x) A.dst[fl[i]] += ys[ti.n_owned + i];
  }
}

// diagonal of C_m^T A_ref C_m for every mask m: virtual cells (m, column j)
// run the same pipeline on the unit vector e_j (Eq. 3 column by column,
// Eq. 4 with the constraints applied on both sides)
template <int K>
__global__ void __launch_bounds__(BLOCK) diag_table_kernel(double* out, int tc) {
  constexpr int N = K + 1, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sm_h = reinterpret_cast<double*>(smem);
  uint16_t* sm_mask = reinterpret_cast<uint16_t*>(sm_h + tc);
  double* cb = reinterpret_cast<double*>(smem + (((size_t)tc * 10 + 15) & ~(size_t)15));
  const int v0 = blockIdx.x * tc;
  const int nv = min(tc, 512 * N3 - v0);
  for (int c = threadIdx.x; c < nv; c += blockDim.x) {
    sm_h[c] = 1.0;
    sm_mask[c] = (uint16_t)((v0 + c) / N3);
  }
  for (int t = threadIdx.x; t < nv * N3; t += blockDim.x) {
    const int c = t / N3, n = t - c * N3;
    cb[t] = (n == (v0 + c) % N3) ? 1.0 : 0.0;
  }
  __syncthreads();
  hanging_all<K, false>(cb, sm_mask, nv);
  cell_laplace<K>(cb, sm_h, nv);
  hanging_all<K, true>(cb, sm_mask, nv);
  for (int c = threadIdx.x; c < nv; c += blockDim.x) {
    const int v = v0 + c;
    out[v] = cb[c * N3 + v % N3];
  }
}

template <int K, typename T, int MODE>
void run_cells(const CellLaunch& L, CellArgs<T> A, cudaStream_t s) {
  const size_t sm = smem_layout<T>((K + 1) * (K + 1) * (K + 1), L.tc, L.max_local).total;
  static bool attr_set = false;
  static size_t attr_bytes = 0;
  if (!attr_set || attr_bytes < sm) {
    cudaFuncSetAttribute(cell_kernel<K, T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max(sm, (size_t)48 * 1024));
    attr_set = true;
    attr_bytes = std::max(sm, (size_t)48 * 1024);
  }
  for (int c = 0; c < L.n_colours; ++c) {
    const int n = L.colour_ptr[c + 1] - L.colour_ptr[c];
    if (n == 0) continue;
    A.tile_list = L.colour_tiles + L.colour_ptr[c];
    { cell_kernel<K, T, MODE><<<n, BLOCK, sm, s>>>(A); note_launches(1); }
  }
}

template <typename T>
CellArgs<T> make_args(const CellLaunch& L) {
  CellArgs<T> A{};
  A.tiles = L.tiles;
  A.meta = L.meta;
  A.foreign = L.foreign;
  A.subptr = L.subptr;
  A.perm = L.perm;
  A.cell_ijk = L.cell_ijk;
  A.lo = L.lo;
  A.dom = L.dom;
  A.tc = L.tc;
  A.max_local = L.max_local;
  return A;
}

template <typename T, int MODE>
void dispatch(const CellLaunch& L, CellArgs<T> A, cudaStream_t s) {
  switch (L.k) {
    case 1: run_cells<1, T, MODE>(L, A, s); break;
    case 2: run_cells<2, T, MODE>(L, A, s); break;
    case 3: run_cells<3, T, MODE>(L, A, s); break;
    case 4: run_cells<4, T, MODE>(L, A, s); break;
    default: break;
  }
}

}  // namespace

size_t cell_smem_bytes(int k, bool fp64, int tc, int max_local) {
  const int n3 = (k + 1) * (k + 1) * (k + 1);
  return fp64 ? smem_layout<double>(n3, tc, max_local).total : smem_layout<float>(n3, tc, max_local).total;
}

void launch_vmult(const CellLaunch& L, bool fp64, const void* src, void* dst, int add, cudaStream_t s) {
  if (fp64) {
    CellArgs<double> A = make_args<double>(L);
    A.src = static_cast<const double*>(src);
    A.dst = static_cast<double*>(dst);
    A.add = add;
    dispatch<double, MODE_VMULT>(L, A, s);
  } else {
    CellArgs<float> A = make_args<float>(L);
    A.src = static_cast<const float*>(src);
    A.dst = static_cast<float*>(dst);
    A.add = add;
    dispatch<float, MODE_VMULT>(L, A, s);
  }
}

void launch_rhs(const CellLaunch& L, const RhsDesc& f, double* dst, cudaStream_t s) {
  CellArgs<double> A = make_args<double>(L);
  A.dst = dst;
  A.modes = f.modes;
  A.n_modes = f.n_modes;
  A.amp = f.amp;
  dispatch<double, MODE_RHS>(L, A, s);
}

void launch_diag(const CellLaunch& L, const double* diag_tab, double* dst, cudaStream_t s) {
  CellArgs<double> A = make_args<double>(L);
  A.dst = dst;
  A.diag_tab = diag_tab;
  dispatch<double, MODE_DIAG>(L, A, s);
}

void launch_diag_table(int k, double* tab_out, cudaStream_t s) {
  const int n3 = (k + 1) * (k + 1) * (k + 1);
  const int tc = 32;
  const size_t sm = (((size_t)tc * 10 + 15) & ~(size_t)15) + (size_t)tc * n3 * sizeof(double);
  const int nb = (512 * n3 + tc - 1) / tc;
  switch (k) {
    { case 1: diag_table_kernel<1><<<nb, BLOCK, sm, s>>>(tab_out, tc); note_launches(1); } break;
    { case 2: diag_table_kernel<2><<<nb, BLOCK, sm, s>>>(tab_out, tc); note_launches(1); } break;
    { case 3: diag_table_kernel<3><<<nb, BLOCK, sm, s>>>(tab_out, tc); note_launches(1); } break;
    { case 4: diag_table_kernel<4><<<nb, BLOCK, sm, s>>>(tab_out, tc); note_launches(1); } break;
    default: break;
  }
}

}  // namespace gcmg
