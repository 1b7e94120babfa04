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
//      diagonalisation form h B^T^{(x)3} diag(lam_a+lam_b+lam_c) B^{(x)3};
//   5. C_e^T, then G_e^T into a shared-memory accumulator, sub-colour by
//      sub-colour (cells that share an entity never add at the same time);
//   6. owned DoFs are written with plain coalesced stores; contributions to
//      DoFs owned by other tiles go to this tile's halo slots, which a second
//      kernel adds in a fixed order.  No atomics: results are reproducible
//      bit for bit.
//
// Two implementations of steps 2-5:
// * cell_kernel: one 1D line per thread, cells in shared memory, processed in
//   chunks (fp64 operator, right-hand side, diagonal);
// * vmult_regs: one cell per thread with all (k+1)^3 values in registers and
//   the sweeps in even-odd form (fp32 operator of the V-cycle).
#include <algorithm>
#include <cstdio>

#include "device.cuh"
#include "kernels.h"

namespace gcmg {

#ifndef GCMG_BODIES_ONLY
GCMG_DEFINE_UPLOAD(upload_tables_cell)
#endif

namespace {

constexpr int CHUNK = 32;  // cells per shared-memory chunk of cell_kernel

template <typename T>
struct CellArgs {
  const TileInfo* tiles;
  const CellMeta* meta;
  const int32_t* foreign;
  const int32_t* halo_pos;
  const uint16_t* subptr;
  const uint8_t* perm;
  const int32_t* cell_ijk;
  const T* src;
  T* dst;
  T* halo;
  double lo, dom;
  int tc;
  int max_local;
  int add;
  RhsDesc fn;
  const double* diag_tab;
  const double* coef;  // per cell nu_e, null: 1
  int geom;            // 0: Cartesian cells; GEOM_WARP: cells mapped by the warp of eps
  double geps;
  int tile0;           // first tile of the launch (the launch covers gridDim.x tiles)
};

// scale of the element matrix of cell ci: nu_e h (h = dom 2^-level)
template <typename T>
__device__ __forceinline__ double cell_scale(const CellArgs<T>& A, double dom, int level, int ci) {
  const double h = ldexp(dom, -level);
  return A.coef ? h * A.coef[ci] : h;
}

// the analytic functions of RhsDesc: f (right-hand side) and u (manufactured
// solution, whose boundary values are the Dirichlet data)
__device__ inline double int_pow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

__device__ inline double func_u(const RhsDesc& F, double x, double y, double z) {
  if (F.kind == FUNC_GAUSSIAN) {
    // (alpha sqrt(2 pi))^-3 exp(-|x - x0|^2 / alpha^2)
    const double al = F.params[0];
    const double dx = x - F.params[1], dy = y - F.params[2], dz = z - F.params[3];
    const double c = 1.0 / (al * sqrt(2.0 * M_PI));
    return c * c * c * exp(-(dx * dx + dy * dy + dz * dz) / (al * al));
  }
  if (F.kind == FUNC_POLYNOMIAL) {
    double u = 0.0;
    for (int m = 0; m < F.n; ++m) {
      const double* t = F.params + 4 * m;
      u += t[0] * int_pow(x, (int)t[1]) * int_pow(y, (int)t[2]) * int_pow(z, (int)t[3]);
    }
    return u;
  }
  return 0.0;
}

__device__ inline double func_f(const RhsDesc& F, double x, double y, double z) {
  switch (F.kind) {
    case FUNC_FOURIER: {
      double f = 0.0;
      for (int m = 0; m < F.n; ++m) {
        const double* md = F.params + 4 * m;
        f += cos(2.0 * M_PI * (md[0] * x + md[1] * y + md[2] * z) + md[3]);
      }
      return f * F.amp;
    }
    case FUNC_GAUSSIAN: {
      // -Lap u = u (6 / alpha^2 - 4 |x - x0|^2 / alpha^4)
      const double a = F.params[0] * F.params[0];
      const double dx = x - F.params[1], dy = y - F.params[2], dz = z - F.params[3];
      const double r2 = dx * dx + dy * dy + dz * dz;
      return func_u(F, x, y, z) * (6.0 / a - 4.0 * r2 / (a * a));
    }
    case FUNC_POLYNOMIAL: {
      double f = 0.0;
      for (int m = 0; m < F.n; ++m) {
        const double* t = F.params + 4 * m;
        const int a = (int)t[1], b = (int)t[2], e = (int)t[3];
        if (a >= 2) f -= t[0] * a * (a - 1) * int_pow(x, a - 2) * int_pow(y, b) * int_pow(z, e);
        if (b >= 2) f -= t[0] * b * (b - 1) * int_pow(x, a) * int_pow(y, b - 2) * int_pow(z, e);
        if (e >= 2) f -= t[0] * e * (e - 1) * int_pow(x, a) * int_pow(y, b) * int_pow(z, e - 2);
      }
      return f;
    }
    default:
      return 1.0;
  }
}

// Is local node (a,b,c) of a cell with hanging mask m on one of its hanging
// faces or edges?  (Such a node takes, before C_e, the value of the parent
// cell's node with the same local index.)
template <int K>
__device__ __forceinline__ bool node_hangs(uint16_t m, int a, int b, int c) {
  if (!(m & MASK_HANG)) return false;
  const bool o0 = a == (m & 1) * K, o1 = b == ((m >> 1) & 1) * K, o2 = c == ((m >> 2) & 1) * K;
  const bool f0 = (m >> 3) & 1, f1 = (m >> 4) & 1, f2 = (m >> 5) & 1;
  const bool e0 = (m >> 6) & 1, e1 = (m >> 7) & 1, e2 = (m >> 8) & 1;
  return (f0 && o0) || (f1 && o1) || (f2 && o2) || (e0 && o1 && o2) || (e1 && o0 && o2) || (e2 && o0 && o1);
}

struct SmemLayout {
  size_t meta, h, mask, cell, cb, xs, ys, gx, gy, gr, total;
};

// mapped: three more chunk buffers (two reference-gradient components and,
// for the diagonal, the collected entries) for the non-Cartesian operator
template <typename T>
__host__ __device__ inline SmemLayout smem_layout(int n3, int tc, int max_local, bool mapped = false,
                                                  bool diag = false) {
  SmemLayout L;
  size_t o = 0;
  L.meta = o;
  o += (size_t)tc * sizeof(CellMeta);
  L.h = o;
  o += (size_t)CHUNK * sizeof(T);
  L.mask = o;
  o += (size_t)CHUNK * sizeof(uint16_t);
  L.cell = o;
  o += (size_t)CHUNK * sizeof(uint16_t);
  o = (o + 15) & ~(size_t)15;
  L.cb = o;
  o += (size_t)CHUNK * n3 * sizeof(T);
  L.xs = o;
  o += (size_t)max_local * sizeof(T);
  L.ys = o;
  o += (size_t)max_local * sizeof(T);
  o = (o + 15) & ~(size_t)15;
  L.gx = L.gy = L.gr = o;
  if (mapped) {
    L.gx = o;
    o += (size_t)CHUNK * n3 * sizeof(T);
    L.gy = o;
    o += (size_t)CHUNK * n3 * sizeof(T);
    L.gr = o;
    if (diag) o += (size_t)CHUNK * n3 * sizeof(T);
  }
  L.total = (o + 15) & ~(size_t)15;
  return L;
}

// stage the tile's cell metadata (64 B per cell, 16-byte loads)
__device__ __forceinline__ void load_meta(CellMeta* sm_meta, const CellMeta* meta, int cell_begin, int nc) {
  const uint4* g = reinterpret_cast<const uint4*>(meta + cell_begin);
  uint4* s = reinterpret_cast<uint4*>(sm_meta);
  for (int i = threadIdx.x; i < nc * 4; i += blockDim.x) s[i] = g[i];
}

template <typename T>
__device__ __forceinline__ void load_tile_dofs(T* xs, const T* src, const int32_t* foreign, const TileInfo& ti) {
  const T* s = src + ti.dof_begin;
  for (int i = threadIdx.x; i < ti.n_owned; i += blockDim.x) xs[i] = s[i];
  const int32_t* fl = foreign + ti.foreign_begin;
  for (int i = threadIdx.x; i < ti.n_foreign; i += blockDim.x) xs[ti.n_owned + i] = src[fl[i]];
}

// owned DoFs: plain stores (or additions); foreign DoFs: into the halo slots
template <typename T>
__device__ __forceinline__ void write_tile_dofs(T* dst, T* halo, const int32_t* halo_pos, const T* ys,
                                                const TileInfo& ti, int add) {
  T* d = dst + ti.dof_begin;
  if (add)
    for (int i = threadIdx.x; i < ti.n_owned; i += blockDim.x) d[i] += ys[i];
  else
    for (int i = threadIdx.x; i < ti.n_owned; i += blockDim.x) d[i] = ys[i];
  const int32_t* hp = halo_pos + ti.foreign_begin;
  for (int i = threadIdx.x; i < ti.n_foreign; i += blockDim.x) halo[hp[i]] = ys[ti.n_owned + i];
}

// ---------------------------------------------------------------------------
// non-Cartesian cells (Eq. 2 with the geometry at the quadrature points)
// ---------------------------------------------------------------------------
// the warp Phi(x) = x + eps (x1 x2, 2 x2 x0, x0 x1 / 2) and its Jacobian
template <typename T>
__device__ __forceinline__ void warp_point(T eps, T& x, T& y, T& z) {
  const T px = x + eps * y * z, py = y + T(2) * eps * z * x, pz = z + T(0.5) * eps * x * y;
  x = px;
  y = py;
  z = pz;
}

// G = sw adj(J) adj(J)^T / det(J) for J = J_Phi(x, y, z): with sw = w h nu
// this is w det(J_cell) J_cell^-1 J_cell^-T of the cell map h J_Phi; G[6] =
// (00, 01, 02, 11, 12, 22); returns det(J_Phi)
template <typename T>
__device__ __forceinline__ T warp_metric(T eps, T x, T y, T z, T sw, T* G) {
  const T j00 = 1, j01 = eps * z, j02 = eps * y;
  const T j10 = T(2) * eps * z, j11 = 1, j12 = T(2) * eps * x;
  const T j20 = T(0.5) * eps * y, j21 = T(0.5) * eps * x, j22 = 1;
  const T a00 = j11 * j22 - j12 * j21, a01 = j02 * j21 - j01 * j22, a02 = j01 * j12 - j02 * j11;
  const T a10 = j12 * j20 - j10 * j22, a11 = j00 * j22 - j02 * j20, a12 = j02 * j10 - j00 * j12;
  const T a20 = j10 * j21 - j11 * j20, a21 = j01 * j20 - j00 * j21, a22 = j00 * j11 - j01 * j10;
  const T det = j00 * a00 + j01 * a10 + j02 * a20;
  const T f = sw / det;
  G[0] = f * (a00 * a00 + a01 * a01 + a02 * a02);
  G[1] = f * (a00 * a10 + a01 * a11 + a02 * a12);
  G[2] = f * (a00 * a20 + a01 * a21 + a02 * a22);
  G[3] = f * (a10 * a10 + a11 * a11 + a12 * a12);
  G[4] = f * (a10 * a20 + a11 * a21 + a12 * a22);
  G[5] = f * (a20 * a20 + a21 * a21 + a22 * a22);
  return det;
}

// one 1D matrix along a line from src into dst (ADD: dst += ...)
template <int N, int STRIDE, bool TRANS, bool ADD, typename T>
__device__ __forceinline__ void line_apply2(const T* src, T* dst, const T (&M)[NMAX][NMAX]) {
  T v[N];
#pragma unroll
  for (int a = 0; a < N; ++a) v[a] = src[a * STRIDE];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T sum = 0;
#pragma unroll
    for (int a = 0; a < N; ++a) sum += (TRANS ? M[a][i] : M[i][a]) * v[a];
    dst[i * STRIDE] = ADD ? dst[i * STRIDE] + sum : sum;
  }
}

template <int N>
__device__ __forceinline__ void line_bases(int t, int& j, int& bx, int& by, int& bz) {
  constexpr int N2 = N * N, N3 = N2 * N;
  j = t / N2;
  const int r = t - j * N2;
  bx = j * N3 + N * r;
  by = j * N3 + r % N + N2 * (r / N);
  bz = j * N3 + r;
}

// the cell operator of mapped cells, in place on the chunk buffer cb (values
// at the support points in, A_e u out): values at the Gauss points (three
// sweeps with the values of the basis), reference gradients by collocation
// derivatives (into gx, gy and, in place, cb), the 3x3 geometry factor of
// every Gauss point, the transposed derivatives summed back into cb, the
// transposed value sweeps.  sm_h[j] = h nu of cell j (negative: -A_e).
template <int K, typename T>
__device__ void cell_laplace_mapped(T* cb, T* gx, T* gy, const T* sm_h, const uint16_t* sm_cell,
                                    const CellMeta* sm_meta, const int32_t* cell_ijk, int cell_begin, double lo,
                                    double dom, T eps, int nch) {
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  const DevTables<T>& tb = tab<T>(K);
  const int nl = nch * N2;
  int j, bx, by, bz;
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply<N, 1, false>(cb + bx, tb.Pq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply<N, N, false>(cb + by, tb.Pq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply<N, N2, false>(cb + bz, tb.Pq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply2<N, 1, false, false>(cb + bx, gx + bx, tb.Dq);
    line_apply2<N, N, false, false>(cb + by, gy + by, tb.Dq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply<N, N2, false>(cb + bz, tb.Dq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nch * N3; t += blockDim.x) {
    const int jj = t / N3, q = t - jj * N3;
    const int qa = q % N, qb = (q / N) % N, qc = q / N2;
    const int ci = cell_begin + sm_cell[jj];
    // the Gauss point in the arithmetic of T (fp32 positions for the fp32 operator)
    const T h = (T)dom / (T)(1 << sm_meta[sm_cell[jj]].level);
    const T x = (T)lo + h * ((T)cell_ijk[3 * ci + 0] + tb.gq[qa]);
    const T y = (T)lo + h * ((T)cell_ijk[3 * ci + 1] + tb.gq[qb]);
    const T z = (T)lo + h * ((T)cell_ijk[3 * ci + 2] + tb.gq[qc]);
    T G[6];
    warp_metric<T>(eps, x, y, z, tb.gw[qa] * tb.gw[qb] * tb.gw[qc] * sm_h[jj], G);
    const T g0 = gx[t], g1 = gy[t], g2 = cb[t];
    gx[t] = G[0] * g0 + G[1] * g1 + G[2] * g2;
    gy[t] = G[1] * g0 + G[3] * g1 + G[4] * g2;
    cb[t] = G[2] * g0 + G[4] * g1 + G[5] * g2;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply<N, N2, true>(cb + bz, tb.Dq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply2<N, N, true, true>(gy + by, cb + by, tb.Dq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply2<N, 1, true, true>(gx + bx, cb + bx, tb.Dq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply<N, N2, true>(cb + bz, tb.Pq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply<N, N, true>(cb + by, tb.Pq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    line_bases<N>(t, j, bx, by, bz);
    line_apply<N, 1, true>(cb + bx, tb.Pq);
  }
  __syncthreads();
}

template <int K, typename T, int MODE, int NT = BLOCK>
__global__ void __launch_bounds__(NT) cell_kernel(CellArgs<T> A) {
  pdl_begin();
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem[];
  const bool mapped = A.geom != 0;
  const SmemLayout SL = smem_layout<T>(N3, A.tc, A.max_local, mapped, MODE == MODE_DIAG);
  T* gx = reinterpret_cast<T*>(smem + SL.gx);
  T* gy = reinterpret_cast<T*>(smem + SL.gy);
  T* gr = reinterpret_cast<T*>(smem + SL.gr);
  const T eps = (T)A.geps;
  CellMeta* sm_meta = reinterpret_cast<CellMeta*>(smem + SL.meta);
  T* sm_h = reinterpret_cast<T*>(smem + SL.h);
  uint16_t* sm_mask = reinterpret_cast<uint16_t*>(smem + SL.mask);
  uint16_t* sm_cell = reinterpret_cast<uint16_t*>(smem + SL.cell);
  T* cb = reinterpret_cast<T*>(smem + SL.cb);
  T* xs = reinterpret_cast<T*>(smem + SL.xs);
  T* ys = reinterpret_cast<T*>(smem + SL.ys);

  const TileInfo ti = A.tiles[A.tile0 + blockIdx.x];
  const int nc = ti.n_cells;
  const int nloc = ti.n_owned + ti.n_foreign;
  load_meta(sm_meta, A.meta, ti.cell_begin, nc);
  if (MODE == MODE_VMULT) load_tile_dofs(xs, A.src, A.foreign, ti);
  for (int i = threadIdx.x; i < nloc; i += blockDim.x) ys[i] = T(0);
  // chunks of CHUNK cells in sub-colour order
  for (int c0 = 0; c0 < nc; c0 += CHUNK) {
    const int nch = min(CHUNK, nc - c0);
    __syncthreads();
    for (int j = threadIdx.x; j < nch; j += blockDim.x) {
      const int cell = A.perm[ti.cell_begin + c0 + j];
      sm_cell[j] = (uint16_t)cell;
      sm_mask[j] = sm_meta[cell].mask;
      // MODE_LIFT applies -A_e: the cell operator is linear in h
      sm_h[j] = (T)cell_scale(A, MODE == MODE_LIFT ? -A.dom : A.dom, sm_meta[cell].level, ti.cell_begin + cell);
    }
    __syncthreads();
    if (MODE == MODE_VMULT) {
      // G_e: gather x-lines of every cell of the chunk
      for (int t = threadIdx.x; t < nch * N2; t += blockDim.x) {
        const int j = t / N2, r = t - j * N2;
        const int b = r % N, c = r / N;
        const uint16_t* ls = sm_meta[sm_cell[j]].ls;
        T* out = cb + j * N3 + N * r;
#pragma unroll
        for (int a = 0; a < N; ++a) {
          int slot, off;
          node_slot<K>(a, b, c, slot, off);
          const uint16_t l = ls[slot];
          out[a] = (l == LS_NONE) ? T(0) : xs[l + off];
        }
      }
    } else if (MODE == MODE_DIAG) {
      if (!mapped)
        for (int t = threadIdx.x; t < nch * N3; t += blockDim.x) {
          const int j = t / N3, n = t - j * N3;
          cb[t] = (T)(A.diag_tab[(sm_mask[j] & 0x1FF) * N3 + n]) * sm_h[j];
        }
    } else if (MODE == MODE_LIFT) {
      // u_g before C_e: at a node of a hanging face or edge the value at the
      // parent's node with the same local index, elsewhere the value at the
      // node; u there if the position is on the domain boundary, else zero
      for (int t = threadIdx.x; t < nch * N3; t += blockDim.x) {
        const int j = t / N3, n = t - j * N3;
        const int nd[3] = {n % N, (n / N) % N, n / N2};
        const int ci = ti.cell_begin + sm_cell[j];
        const int lev = sm_meta[sm_cell[j]].level;
        const bool hang = node_hangs<K>(sm_mask[j], nd[0], nd[1], nd[2]);
        const int l = hang ? lev - 1 : lev;
        const double h = ldexp(A.dom, -l);
        const int last = (1 << l) - 1;
        double p[3];
        bool bnd = false;
        for (int d = 0; d < 3; ++d) {
          const int I = hang ? (A.cell_ijk[3 * ci + d] >> 1) : A.cell_ijk[3 * ci + d];
          bnd |= (nd[d] == 0 && I == 0) || (nd[d] == K && I == last);
          p[d] = A.lo + h * ((double)I + tab<double>(K).xi[nd[d]]);
        }
        if (mapped) warp_point<double>(A.geps, p[0], p[1], p[2]);
        cb[t] = bnd ? (T)func_u(A.fn, p[0], p[1], p[2]) : T(0);
      }
    } else {  // MODE_RHS: h^3 w_q f(x_q) at the Gauss points, then S^T
      for (int t = threadIdx.x; t < nch * N3; t += blockDim.x) {
        const int j = t / N3, n = t - j * N3;
        const int qa = n % N, qb = (n / N) % N, qc = n / N2;
        const int ci = ti.cell_begin + sm_cell[j];
        const double h = ldexp(A.dom, -(int)sm_meta[sm_cell[j]].level);
        const double x = A.lo + h * (A.cell_ijk[3 * ci + 0] + (double)tab<double>(K).gq[qa]);
        const double y = A.lo + h * (A.cell_ijk[3 * ci + 1] + (double)tab<double>(K).gq[qb]);
        const double z = A.lo + h * (A.cell_ijk[3 * ci + 2] + (double)tab<double>(K).gq[qc]);
        const double w = tab<double>(K).gw[qa] * tab<double>(K).gw[qb] * tab<double>(K).gw[qc];
        if (mapped) {  // w det(J) f(Phi(x)), det(J) = h^3 det(J_Phi)
          double G[6];
          const double dj = warp_metric<double>(A.geps, x, y, z, 1.0, G);
          double px = x, py = y, pz = z;
          warp_point<double>(A.geps, px, py, pz);
          cb[t] = (T)(w * h * h * h * dj * func_f(A.fn, px, py, pz));
        } else {
          cb[t] = (T)(w * h * h * h * func_f(A.fn, x, y, z));
        }
      }
      __syncthreads();
      const DevTables<T>& tb = tab<T>(K);
      for (int t = threadIdx.x; t < nch * N2; t += blockDim.x) {
        const int j = t / N2, r = t - j * N2;
        line_apply<N, 1, true>(cb + j * N3 + N * r, tb.Pq);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nch * N2; t += blockDim.x) {
        const int j = t / N2, r = t - j * N2;
        int base, u, v;
        line_geom<N, 1>(r, base, u, v);
        line_apply<N, N, true>(cb + j * N3 + base, tb.Pq);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nch * N2; t += blockDim.x) {
        const int j = t / N2, r = t - j * N2;
        line_apply<N, N2, true>(cb + j * N3 + r, tb.Pq);
      }
    }
    __syncthreads();
    if (MODE == MODE_VMULT) {
      hanging_all<K, false>(cb, sm_mask, nch);  // C_e
      if (mapped)                               // S^T Q S
        cell_laplace_mapped<K, T>(cb, gx, gy, sm_h, sm_cell, sm_meta, A.cell_ijk, ti.cell_begin, A.lo, A.dom, eps, nch);
      else
        cell_laplace<K>(cb, sm_h, nch);
    }
    if (MODE == MODE_DIAG && mapped) {
      // (C_e^T A_e C_e)_nn of every cell, column by column (Eqs. 3-4): no
      // per-mask table for cells with their own geometry
      for (int n = 0; n < N3; ++n) {
        for (int t = threadIdx.x; t < nch * N3; t += blockDim.x) cb[t] = (t % N3 == n) ? T(1) : T(0);
        __syncthreads();
        hanging_all<K, false>(cb, sm_mask, nch);
        cell_laplace_mapped<K, T>(cb, gx, gy, sm_h, sm_cell, sm_meta, A.cell_ijk, ti.cell_begin, A.lo, A.dom, eps, nch);
        hanging_all<K, true>(cb, sm_mask, nch);
        for (int j = threadIdx.x; j < nch; j += blockDim.x) gr[j * N3 + n] = cb[j * N3 + n];
        __syncthreads();
      }
      for (int t = threadIdx.x; t < nch * N3; t += blockDim.x) cb[t] = gr[t];
      __syncthreads();
    }
    if (MODE == MODE_LIFT) {
      hanging_all<K, false>(cb, sm_mask, nch);  // C_e: interpolated boundary values at hanging nodes
      // support points on the boundary carry u itself, hanging or not
      for (int t = threadIdx.x; t < nch * N3; t += blockDim.x) {
        const int j = t / N3, n = t - j * N3;
        const int nd[3] = {n % N, (n / N) % N, n / N2};
        const int ci = ti.cell_begin + sm_cell[j];
        const int lev = sm_meta[sm_cell[j]].level;
        const double h = ldexp(A.dom, -lev);
        const int last = (1 << lev) - 1;
        double p[3];
        bool bnd = false;
        for (int d = 0; d < 3; ++d) {
          const int I = A.cell_ijk[3 * ci + d];
          bnd |= (nd[d] == 0 && I == 0) || (nd[d] == K && I == last);
          p[d] = A.lo + h * ((double)I + tab<double>(K).xi[nd[d]]);
        }
        if (mapped) warp_point<double>(A.geps, p[0], p[1], p[2]);
        if (bnd && node_hangs<K>(sm_mask[j], nd[0], nd[1], nd[2])) cb[t] = (T)func_u(A.fn, p[0], p[1], p[2]);
      }
      __syncthreads();
      if (mapped)  // -A_e u_g
        cell_laplace_mapped<K, T>(cb, gx, gy, sm_h, sm_cell, sm_meta, A.cell_ijk, ti.cell_begin, A.lo, A.dom, eps, nch);
      else
        cell_laplace<K>(cb, sm_h, nch);
    }
    if (MODE != MODE_DIAG) hanging_all<K, true>(cb, sm_mask, nch);  // C_e^T
    // G_e^T into the shared accumulator, sub-colour by sub-colour
    for (int s = 0; s < ti.n_sub; ++s) {
      const int q0 = max(c0, (int)A.subptr[ti.sub_begin + s]);
      const int q1 = min(c0 + nch, (int)A.subptr[ti.sub_begin + s + 1]);
      if (q1 <= q0) continue;
      for (int t = threadIdx.x; t < (q1 - q0) * N2; t += blockDim.x) {
        const int j = q0 - c0 + t / N2, r = t % N2;
        const int b = r % N, c = r / N;
        const uint16_t* ls = sm_meta[sm_cell[j]].ls;
        const T* in = cb + j * N3 + N * r;
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
  }
  __syncthreads();
  write_tile_dofs(A.dst, A.halo, A.halo_pos, ys, ti, A.add);
}

// ---------------------------------------------------------------------------
// fp32 operator for tiles of at most CHUNK cells (the default configuration):
// every thread owns the same lines of the tile in every phase, so their cell,
// position and gather/scatter starts are computed once per tile and kept in
// registers; the tile's metadata and DoFs arrive by asynchronous copies that
// are all in flight together; the hanging-node passes do no work for tiles
// without hanging cells; the accumulation runs sub-colour by sub-colour, each
// sub-colour a contiguous range of the permuted cell list.  LPT, the lines
// per thread, covers the level's largest tile (the small tiles of the coarse
// levels run with LPT = 1: a shorter kernel for a launch that is one chain of
// latencies).
// ---------------------------------------------------------------------------
template <int K, typename T, int LPT>
__global__ void __launch_bounds__(BLOCK) vmult_lines(CellArgs<T> A) {
  static_assert(sizeof(T) == 4, "the fp64 operator is vmult_lines_df");
  pdl_begin();
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout SL = smem_layout<T>(N3, A.tc, A.max_local);
  CellMeta* sm_meta = reinterpret_cast<CellMeta*>(smem + SL.meta);
  T* sm_h = reinterpret_cast<T*>(smem + SL.h);
  uint16_t* sm_mask = reinterpret_cast<uint16_t*>(smem + SL.mask);
  uint16_t* sm_cell = reinterpret_cast<uint16_t*>(smem + SL.cell);
  T* cb = reinterpret_cast<T*>(smem + SL.cb);
  T* xs = reinterpret_cast<T*>(smem + SL.xs);
  T* ys = xs;  // the accumulator reuses the input buffer once the gather is done
  __shared__ T s_lab[N2];
  __shared__ uint16_t s_so[N3];          // per local node: entity slot | offset << 5
  __shared__ uint16_t s_sub[CHUNK + 1];  // sub-colour starts (positions in the permuted cell list)
  const DevTables<T>& tb = tab<T>(K);

  const TileInfo ti = A.tiles[A.tile0 + blockIdx.x];
  const int nc = ti.n_cells;
  const int nl = nc * N2;
  const int nloc = ti.n_owned + ti.n_foreign;
  {  // asynchronous copies of the tile's metadata and DoFs, all in flight at once
    const uint4* gm = reinterpret_cast<const uint4*>(A.meta + ti.cell_begin);
    uint4* smm = reinterpret_cast<uint4*>(sm_meta);
    for (int i = threadIdx.x; i < nc * 4; i += BLOCK) cp_async16(smm + i, gm + i);
    const T* so_ = A.src + ti.dof_begin;
#pragma unroll 4
    for (int i = threadIdx.x; i < ti.n_owned; i += BLOCK) cp_async(xs + i, so_ + i);
    const int32_t* fl = A.foreign + ti.foreign_begin;
    T* xf = xs + ti.n_owned;
    for (int i0 = threadIdx.x; i0 < ti.n_foreign; i0 += 4 * BLOCK) {
      int idx[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) idx[u] = (i0 + u * BLOCK < ti.n_foreign) ? fl[i0 + u * BLOCK] : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (idx[u] >= 0) cp_async(xf + i0 + u * BLOCK, A.src + idx[u]);
    }
  }
  for (int n = threadIdx.x; n < N3; n += BLOCK) {
    int slot, off;
    node_slot<K>(n % N, (n / N) % N, n / N2, slot, off);
    s_so[n] = (uint16_t)(slot | (off << 5));
  }
  if (threadIdx.x < (K > 1 ? K - 1 : 1)) xs[nloc + threadIdx.x] = T(0);  // zero slots: absent DoFs gather 0
  for (int r = threadIdx.x; r < N2; r += BLOCK) s_lab[r] = tb.lam[r % N] + tb.lam[r / N];
  for (int s = threadIdx.x; s <= ti.n_sub; s += BLOCK) s_sub[s] = A.subptr[ti.sub_begin + s];
  cp_async_wait_all();
  __syncthreads();
  int hang = 0;
  if (threadIdx.x < nc) {
    const int cell = A.perm[ti.cell_begin + threadIdx.x];
    const CellMeta& m = sm_meta[cell];
    sm_cell[threadIdx.x] = (uint16_t)cell;
    sm_mask[threadIdx.x] = m.mask;
    sm_h[threadIdx.x] = (T)cell_scale(A, A.dom, m.level, ti.cell_begin + cell);
    hang = (m.mask & MASK_HANG) != 0;
  }
  hang = __syncthreads_or(hang);

  // the thread's lines t = tid + BLOCK i (cell position j = t / N2, r = t % N2 = b + N c) and the
  // tile-local starts of their three x-classes (node a = 0, interior 1..K-1, a = K); absent DoFs
  // point to the zero slots xs[nloc .. nloc+K-2], so gather and scatter need no branch per node
  // (the slots read 0 in the gather and absorb the dropped contributions in the scatter; they are
  // never written out)
  int lj[LPT], lr[LPT], g0[LPT], g1[LPT], g2[LPT];
#pragma unroll
  for (int i = 0; i < LPT; ++i) {
    const int t = threadIdx.x + BLOCK * i;
    lj[i] = t / N2;
    lr[i] = t - lj[i] * N2;
    g0[i] = g1[i] = g2[i] = nloc;
    if (t < nl) {
      const uint16_t* ls = sm_meta[sm_cell[lj[i]]].ls;
      const int so0 = s_so[N * lr[i]], so1 = s_so[N * lr[i] + 1], so2 = s_so[N * lr[i] + K];
      const uint16_t l0 = ls[so0 & 31], l1 = ls[so1 & 31], l2 = ls[so2 & 31];
      if (l0 != LS_NONE) g0[i] = l0 + (so0 >> 5);
      if (l1 != LS_NONE) g1[i] = l1 + (so1 >> 5);
      if (l2 != LS_NONE) g2[i] = l2 + (so2 >> 5);
    }
  }
  // G_e: gather the x-lines
#pragma unroll
  for (int i = 0; i < LPT; ++i) {
    const int t = threadIdx.x + BLOCK * i;
    if (t < nl) {
      T* out = cb + N * t;
      out[0] = xs[g0[i]];
#pragma unroll
      for (int a = 1; a < K; ++a) out[a] = xs[g1[i] + a - 1];  // absent: the K-1 zero slots
      out[K] = xs[g2[i]];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nloc; i += BLOCK) ys[i] = T(0);
  hanging_all<K, false>(cb, sm_mask, hang ? nc : 0);  // C_e (no work without hanging cells)

  // S^T Q S: x, y forward, z forward/scale/backward, y, x backward
#pragma unroll
  for (int i = 0; i < LPT; ++i) {
    const int t = threadIdx.x + BLOCK * i;
    if (t < nl) line_apply<N, 1, false>(cb + N * t, tb.B);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < LPT; ++i) {
    const int t = threadIdx.x + BLOCK * i;
    if (t < nl) line_apply<N, N, false>(cb + lj[i] * N3 + lr[i] % N + N2 * (lr[i] / N), tb.B);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < LPT; ++i) {
    const int t = threadIdx.x + BLOCK * i;
    if (t < nl) {
      T* p = cb + lj[i] * N3 + lr[i];
      T v[N];
#pragma unroll
      for (int c = 0; c < N; ++c) v[c] = p[c * N2];
      const T hab = sm_h[lj[i]], lab = s_lab[lr[i]];
      T w[N];
#pragma unroll
      for (int q = 0; q < N; ++q) {
        T sum = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) sum += tb.B[q][c] * v[c];
        w[q] = sum * hab * (lab + tb.lam[q]);
      }
#pragma unroll
      for (int q = 0; q < N; ++q) {
        T sum = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) sum += tb.B[c][q] * w[c];
        p[q * N2] = sum;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < LPT; ++i) {
    const int t = threadIdx.x + BLOCK * i;
    if (t < nl) line_apply<N, N, true>(cb + lj[i] * N3 + lr[i] % N + N2 * (lr[i] / N), tb.B);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < LPT; ++i) {
    const int t = threadIdx.x + BLOCK * i;
    if (t < nl) line_apply<N, 1, true>(cb + N * t, tb.B);
  }
  __syncthreads();
  hanging_all<K, true>(cb, sm_mask, hang ? nc : 0);  // C_e^T

  // G_e^T, sub-colour by sub-colour (cells of sub-colour s: positions s_sub[s] .. s_sub[s+1])
  for (int sc = 0; sc < ti.n_sub; ++sc) {
    const int t0 = s_sub[sc] * N2, t1 = s_sub[sc + 1] * N2;
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
      const int t = threadIdx.x + BLOCK * i;
      if (t >= t0 && t < t1) {
        const T* in = cb + N * t;
        ys[g0[i]] += in[0];
#pragma unroll
        for (int a = 1; a < K; ++a) ys[g1[i] + a - 1] += in[a];
        ys[g2[i]] += in[K];
      }
    }
    __syncthreads();
  }
  write_tile_dofs(A.dst, A.halo, A.halo_pos, ys, ti, A.add);
}

// ---------------------------------------------------------------------------
// fp64 operator in double-float arithmetic (fp64 vectors, all arithmetic of
// the cell pipeline on the FP32 pipe in hi + lo pairs, about 48 bits): the
// structure of vmult_lines with the tile buffer and the cell buffers in df;
// values are converted once on entry to and once on exit from the tile.
// ---------------------------------------------------------------------------
// shared memory of the mapped variant: the layout of the operator kernel up
// to the tile buffer, then two gradient buffers of MAPPED_SUB cells
constexpr int MAPPED_SUB = 16;
__host__ __device__ inline size_t mapped_df_gx(int n3, int tc, int max_local) {
  const SmemLayout SL = smem_layout<double>(n3, tc, max_local);
  return (SL.xs + (size_t)max_local * sizeof(double) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t mapped_df_smem(int n3, int tc, int max_local) {
  return mapped_df_gx(n3, tc, max_local) + 2 * (size_t)MAPPED_SUB * n3 * sizeof(double);
}

template <int K, bool MAPPED = false>
__global__ void __launch_bounds__(BLOCK) vmult_lines_df(CellArgs<double> A) {
  pdl_begin();
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  static_assert(sizeof(df) == sizeof(double), "df buffers reuse the fp64 layout");
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout SL = smem_layout<double>(N3, A.tc, A.max_local);
  CellMeta* sm_meta = reinterpret_cast<CellMeta*>(smem + SL.meta);
  df* sm_h = reinterpret_cast<df*>(smem + SL.h);
  uint16_t* sm_mask = reinterpret_cast<uint16_t*>(smem + SL.mask);
  uint16_t* sm_cell = reinterpret_cast<uint16_t*>(smem + SL.cell);
  df* cb = reinterpret_cast<df*>(smem + SL.cb);
  df* xs = reinterpret_cast<df*>(smem + SL.xs);
  df* ys = xs;  // the accumulator reuses the input buffer once the gather is done
  __shared__ uint8_t sm_sub[CHUNK];
  __shared__ df s_lam3[N3];      // lam_a + lam_b + lam_c in mode order
  __shared__ uint16_t s_so[N3];  // per local node: entity slot | offset << 5

  const TileInfo ti = A.tiles[A.tile0 + blockIdx.x];
  const int nc = ti.n_cells;  // <= CHUNK
  const int nl = nc * N2;
  const int nloc = ti.n_owned + ti.n_foreign;
  double* xd = reinterpret_cast<double*>(xs);
  {  // asynchronous copies of the metadata and the fp64 DoFs, all in flight at once
    const uint4* gm = reinterpret_cast<const uint4*>(A.meta + ti.cell_begin);
    uint4* smm = reinterpret_cast<uint4*>(sm_meta);
    for (int i = threadIdx.x; i < nc * 4; i += BLOCK) cp_async16(smm + i, gm + i);
    const double* src = A.src + ti.dof_begin;
#pragma unroll 4
    for (int i = threadIdx.x; i < ti.n_owned; i += BLOCK) cp_async(xd + i, src + i);
    const int32_t* fl = A.foreign + ti.foreign_begin;
    double* xf = xd + ti.n_owned;
    for (int i0 = threadIdx.x; i0 < ti.n_foreign; i0 += 4 * BLOCK) {
      int idx[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) idx[u] = (i0 + u * BLOCK < ti.n_foreign) ? fl[i0 + u * BLOCK] : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (idx[u] >= 0) cp_async(xf + i0 + u * BLOCK, A.src + idx[u]);
    }
  }
  for (int n = threadIdx.x; n < N3; n += BLOCK) {
    int slot, off;
    node_slot<K>(n % N, (n / N) % N, n / N2, slot, off);
    s_so[n] = (uint16_t)(slot | (off << 5));
    s_lam3[n] = df_from(c_td[K].lam3[n]);
  }
  cp_async_wait_all();
  // every thread converts the values it copied itself, in place (a df has the size of a double)
  for (int i = threadIdx.x; i < ti.n_owned; i += BLOCK) xs[i] = df_from(xd[i]);
  for (int i = threadIdx.x; i < ti.n_foreign; i += BLOCK) xs[ti.n_owned + i] = df_from(xd[ti.n_owned + i]);
  __syncthreads();
  int hang = 0;
  if (threadIdx.x < nc) {
    const int cell = A.perm[ti.cell_begin + threadIdx.x];
    const CellMeta& m = sm_meta[cell];
    sm_cell[threadIdx.x] = (uint16_t)cell;
    sm_mask[threadIdx.x] = m.mask;
    sm_sub[threadIdx.x] = m.sub;
    sm_h[threadIdx.x] = df_from(cell_scale(A, A.dom, m.level, ti.cell_begin + cell));
    hang = (m.mask & MASK_HANG) != 0;
  }
  hang = __syncthreads_or(hang);

  // G_e
#pragma unroll 1
  for (int t = threadIdx.x; t < nl; t += BLOCK) {
    const int j = t / N2, r = t - j * N2;
    const uint16_t* ls = sm_meta[sm_cell[j]].ls;
    df* out = cb + j * N3 + N * r;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const int so = s_so[N * r + a];
      const uint16_t l = ls[so & 31];
      out[a] = (l == LS_NONE) ? df{0.f, 0.f} : xs[l + (so >> 5)];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nloc; i += BLOCK) ys[i] = df{0.f, 0.f};
  df_hanging_all<K, false>(cb, sm_mask, hang ? nc : 0);  // C_e

  if constexpr (MAPPED) {
    // non-Cartesian cells: the quadrature-point operator in double-float, MAPPED_SUB cells at a time
    df* gx = reinterpret_cast<df*>(smem + mapped_df_gx(N3, A.tc, A.max_local));
    df* gy = gx + MAPPED_SUB * N3;
    for (int s0 = 0; s0 < nc; s0 += MAPPED_SUB)
      cell_laplace_mapped<K, df>(cb + s0 * N3, gx, gy, sm_h + s0, sm_cell + s0, sm_meta, A.cell_ijk, ti.cell_begin,
                                 A.lo, A.dom, df(A.geps), min(MAPPED_SUB, nc - s0));
  } else {
    // S^T Q S with even-odd sweeps
  #pragma unroll 1
    for (int t = threadIdx.x; t < nl; t += BLOCK) df_eo_forward<K, 1>(cb + (t / N2) * N3 + N * (t % N2));
    __syncthreads();
  #pragma unroll 1
    for (int t = threadIdx.x; t < nl; t += BLOCK) {
      const int j = t / N2, r = t - j * N2;
      df_eo_forward<K, N>(cb + j * N3 + r % N + N2 * (r / N));
    }
    __syncthreads();
  #pragma unroll 1
    for (int t = threadIdx.x; t < nl; t += BLOCK) {
      const int j = t / N2, r = t - j * N2;
      df* p = cb + j * N3 + r;
      df v[N];
  #pragma unroll
      for (int c = 0; c < N; ++c) v[c] = p[c * N2];
      df_eo_forward<K, 1>(v);
      const df h = sm_h[j];
  #pragma unroll
      for (int c = 0; c < N; ++c) v[c] = df_mul(df_mul(v[c], s_lam3[r + N2 * c]), h);
      df_eo_backward<K, 1>(v);
  #pragma unroll
      for (int c = 0; c < N; ++c) p[c * N2] = v[c];
    }
    __syncthreads();
  #pragma unroll 1
    for (int t = threadIdx.x; t < nl; t += BLOCK) {
      const int j = t / N2, r = t - j * N2;
      df_eo_backward<K, N>(cb + j * N3 + r % N + N2 * (r / N));
    }
    __syncthreads();
  #pragma unroll 1
    for (int t = threadIdx.x; t < nl; t += BLOCK) df_eo_backward<K, 1>(cb + (t / N2) * N3 + N * (t % N2));
    __syncthreads();
  }
  df_hanging_all<K, true>(cb, sm_mask, hang ? nc : 0);  // C_e^T

  // G_e^T, sub-colour by sub-colour
  for (int sc = 0; sc < ti.n_sub; ++sc) {
#pragma unroll 1
    for (int t = threadIdx.x; t < nl; t += BLOCK) {
      const int j = t / N2;
      if (sm_sub[j] != sc) continue;
      const int r = t - j * N2;
      const uint16_t* ls = sm_meta[sm_cell[j]].ls;
      const df* in = cb + j * N3 + N * r;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const int so = s_so[N * r + a];
        const uint16_t l = ls[so & 31];
        if (l != LS_NONE) ys[l + (so >> 5)] = df_add(ys[l + (so >> 5)], in[a]);
      }
    }
    __syncthreads();
  }
  double* d = A.dst + ti.dof_begin;
  if (A.add)
    for (int i = threadIdx.x; i < ti.n_owned; i += BLOCK) d[i] += df_to(ys[i]);
  else
    for (int i = threadIdx.x; i < ti.n_owned; i += BLOCK) d[i] = df_to(ys[i]);
  const int32_t* hp = A.halo_pos + ti.foreign_begin;
  for (int i = threadIdx.x; i < ti.n_foreign; i += BLOCK) A.halo[hp[i]] = df_to(ys[ti.n_owned + i]);
}

// ---------------------------------------------------------------------------
// fp32 operator, one cell per thread, values in registers
// ---------------------------------------------------------------------------

// Shared-memory position of tile-local DoF l: one pad word after every 64.
// Threads of a warp handle consecutive cells whose DoF blocks lie about 64
// words apart; without the padding they would hit the same bank (26-way
// conflicts on the Q4 octant workload, 1.9-way with it).
__device__ __forceinline__ int swz(int l) { return l + (l >> 6); }

// hanging-node interpolation of one cell, done by the whole warp through a
// small shared-memory scratch (the owner lane writes its values, the lanes
// apply the direction-wise line interpolation, the owner reads back)
template <int K, bool TRANS>
__device__ __forceinline__ void hanging_warp(float* u, uint16_t mask, bool active, float* scratch) {
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  const int lane = threadIdx.x & 31;
  unsigned pending = __ballot_sync(0xffffffffu, active && (mask & MASK_HANG));
  while (pending) {
    const int owner = __ffs(pending) - 1;
    pending &= pending - 1;
    const uint16_t m = __shfl_sync(0xffffffffu, mask, owner);
    if (lane == owner) {
#pragma unroll
      for (int n = 0; n < N3; ++n) scratch[n] = u[n];
    }
    __syncwarp();
    const DevTables<float>& tb = tab<float>(K);
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      const int D = TRANS ? 2 - dd : dd;
      const int stride = D == 0 ? 1 : (D == 1 ? N : N2);
      const int p = (m >> D) & 1;
      for (int r = lane; r < N2; r += 32) {
        const int uu = r % N, vv = r / N;
        int base;
        bool hang;
        if (D == 0) {
          base = N * r;
          hang = line_hangs<K, 0>(m, uu, vv);
        } else if (D == 1) {
          base = uu + N2 * vv;
          hang = line_hangs<K, 1>(m, uu, vv);
        } else {
          base = r;
          hang = line_hangs<K, 2>(m, uu, vv);
        }
        if (!hang) continue;
        float v[N];
#pragma unroll
        for (int a = 0; a < N; ++a) v[a] = scratch[base + a * stride];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          float s = 0.f;
#pragma unroll
          for (int a = 0; a < N; ++a) s += (TRANS ? tb.I[p][a][i] : tb.I[p][i][a]) * v[a];
          scratch[base + i * stride] = s;
        }
      }
      __syncwarp();
    }
    if (lane == owner) {
#pragma unroll
      for (int n = 0; n < N3; ++n) u[n] = scratch[n];
    }
    __syncwarp();
  }
}

template <int K>
__host__ __device__ inline size_t regs_smem(int tc, int max_local) {
  return (size_t)tc * (NSLOT + 3) * sizeof(uint16_t) + 16 +
         ((size_t)4 * (K + 1) * (K + 1) * (K + 1) + (size_t)max_local + max_local / 64 + 32) * sizeof(float);
}

// 27-bit set of the slots of a cell that lie on a hanging face or edge
__device__ __forceinline__ uint32_t hanging_slots(uint16_t m) {
  uint32_t hs = 0;
  if (!(m & MASK_HANG)) return 0;
  const int p0 = m & 1, p1 = (m >> 1) & 1, p2 = (m >> 2) & 1;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    const int c0 = s % 3, c1 = (s / 3) % 3, c2 = s / 9;
    bool h = (((m >> 3) & 1) && c0 == 2 * p0) || (((m >> 4) & 1) && c1 == 2 * p1) ||
             (((m >> 5) & 1) && c2 == 2 * p2) || (((m >> 6) & 1) && c1 == 2 * p1 && c2 == 2 * p2) ||
             (((m >> 7) & 1) && c0 == 2 * p0 && c2 == 2 * p2) || (((m >> 8) & 1) && c0 == 2 * p0 && c1 == 2 * p1);
    if (h) hs |= 1u << s;
  }
  return hs;
}

// G_e^T for the nodes of side step SIG: coordinate == K along the "high"
// axes of SIG, < K along the others.  Two cells that share an entity through
// regular (non-hanging) slots see it from opposite sides along at least one
// axis, so no two lanes add to the same DoF within one step.
template <int K, int SIG, int NODE = 0>
__device__ __forceinline__ void scatter_side(float* buf, const float* u, const uint16_t* sm_ls, int tc, int q,
                                             uint32_t skip) {
  constexpr int N = K + 1, N3 = N * N * N;
  if constexpr (NODE < N3) {
    constexpr int a = NODE % N, b = (NODE / N) % N, c = NODE / (N * N);
    constexpr bool in = ((SIG & 1) ? a == K : a < K) && ((SIG & 2) ? b == K : b < K) && ((SIG & 4) ? c == K : c < K);
    if constexpr (in) {
      constexpr int ca = a == 0 ? 0 : (a == K ? 2 : 1), cb = b == 0 ? 0 : (b == K ? 2 : 1),
                    cc = c == 0 ? 0 : (c == K ? 2 : 1);
      constexpr int slot = ca + 3 * cb + 9 * cc;
      constexpr int off = (ca == 1 ? (a - 1) : 0) + (cb == 1 ? (b - 1) * (ca == 1 ? (K - 1) : 1) : 0) +
                          (cc == 1 ? (c - 1) * ((ca == 1 ? (K - 1) : 1) * (cb == 1 ? (K - 1) : 1)) : 0);
      const uint16_t l = sm_ls[slot * tc + q];
      if (l != LS_NONE && !((skip >> slot) & 1u)) buf[swz(l + off)] += u[NODE];
    }
    scatter_side<K, SIG, NODE + 1>(buf, u, sm_ls, tc, q, skip);
  }
}

// ---------------------------------------------------------------------------
// fp32 operator, N = k+1 threads per cell: thread c of a cell holds the
// z-slab c (N^2 values) in registers; x and y sweeps run in registers, the z
// sweeps after a transpose through the cell's shared-memory region (the N
// threads of a cell sit in one warp, so the transposes need only warp
// synchronisation).  Small code, about 60 registers per thread.
// ---------------------------------------------------------------------------
template <int K>
struct SlabGeom {
  static constexpr int N = K + 1, N2 = N * N, N3 = N2 * N;
  static constexpr int CPW = 32 / N;  // cells per warp
};

template <int K>
__host__ __device__ inline int slab_warps(int tc) {
  return (tc + SlabGeom<K>::CPW - 1) / SlabGeom<K>::CPW;
}

template <int K>
__host__ __device__ inline size_t slab_smem(int tc, int max_local) {
  constexpr int N3 = SlabGeom<K>::N3;
  return (size_t)tc * (NSLOT + 3) * sizeof(uint16_t) + 16 +
         ((size_t)N3 + (size_t)(tc + 1) * N3 + (size_t)max_local + max_local / 64 + 32) * sizeof(float);
}

// slot (runtime class along z) and offset of node (a, b, c)
template <int K, int a, int b>
__device__ __forceinline__ void slab_slot(int c, int cc, int& slot, int& off) {
  constexpr int ca = a == 0 ? 0 : (a == K ? 2 : 1), cb = b == 0 ? 0 : (b == K ? 2 : 1);
  constexpr int m1 = ca == 1 ? (K - 1) : 1;
  constexpr int m2 = m1 * (cb == 1 ? (K - 1) : 1);
  constexpr int o0 = (ca == 1 ? a - 1 : 0) + (cb == 1 ? (b - 1) * m1 : 0);
  slot = ca + 3 * cb + 9 * cc;
  off = o0 + (cc == 1 ? (c - 1) * m2 : 0);
}

template <int K, int P = 0>
__device__ __forceinline__ void slab_gather(float* sv, const float* buf, const uint16_t* sm_ls, int tc, int q, int c,
                                            int cc, bool active) {
  constexpr int N = K + 1;
  if constexpr (P < N * N) {
    int slot, off;
    slab_slot<K, P % N, P / N>(c, cc, slot, off);
    const uint16_t l = sm_ls[slot * tc + q];
    sv[P] = (active && l != LS_NONE) ? buf[swz(l + off)] : 0.f;
    slab_gather<K, P + 1>(sv, buf, sm_ls, tc, q, c, cc, active);
  }
}

// add the slab's nodes of side step SIG (see scatter_side) to the accumulator
template <int K, int SIG, int P = 0>
__device__ __forceinline__ void slab_scatter(float* buf, const float* sv, const uint16_t* sm_ls, int tc, int q, int c,
                                             int cc, uint32_t skip) {
  constexpr int N = K + 1;
  if constexpr (P < N * N) {
    constexpr int a = P % N, b = P / N;
    constexpr bool in = ((SIG & 1) ? a == K : a < K) && ((SIG & 2) ? b == K : b < K);
    if constexpr (in) {
      int slot, off;
      slab_slot<K, a, b>(c, cc, slot, off);
      const uint16_t l = sm_ls[slot * tc + q];
      if (l != LS_NONE && !((skip >> slot) & 1u)) buf[swz(l + off)] += sv[P];
    }
    slab_scatter<K, SIG, P + 1>(buf, sv, sm_ls, tc, q, c, cc, skip);
  }
}

template <int K, bool HANG_ONLY, int P = 0>
__device__ __forceinline__ void slab_scatter_hanging(float* buf, const float* sv, const uint16_t* sm_ls, int tc,
                                                     int q, int c, int cc, uint32_t hs) {
  constexpr int N = K + 1;
  if constexpr (P < N * N) {
    int slot, off;
    slab_slot<K, P % N, P / N>(c, cc, slot, off);
    const uint16_t l = sm_ls[slot * tc + q];
    if (l != LS_NONE && ((hs >> slot) & 1u)) buf[swz(l + off)] += sv[P];
    slab_scatter_hanging<K, HANG_ONLY, P + 1>(buf, sv, sm_ls, tc, q, c, cc, hs);
  }
}

// apply the child-side interpolation matrix I[P] to a register line
template <int N, int BASE, int STRIDE, bool TRANS, int P>
__device__ __forceinline__ void interp_line_p(float* v) {
  const DevTables<float>& tb = tab<float>(N - 1);
  float t[N];
#pragma unroll
  for (int a = 0; a < N; ++a) t[a] = v[BASE + a * STRIDE];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < N; ++a) s += (TRANS ? tb.I[P][a][i] : tb.I[P][i][a]) * t[a];
    v[BASE + i * STRIDE] = s;
  }
}

// the child side p is a runtime value: branch so that the table index stays
// a compile-time constant (constant-bank operands, no generic loads)
template <int N, int BASE, int STRIDE, bool TRANS>
__device__ __forceinline__ void interp_line(float* v, int p) {
  if (p)
    interp_line_p<N, BASE, STRIDE, TRANS, 1>(v);
  else
    interp_line_p<N, BASE, STRIDE, TRANS, 0>(v);
}

// C_x and C_y (or their transposes, in reverse order) on the slab of thread c
template <int K, bool TRANS>
__device__ __forceinline__ void slab_hanging_xy(float* sv, uint16_t m, int c) {
  constexpr int N = K + 1;
  const int px = m & 1, py = (m >> 1) & 1;
  if (!TRANS) {
#pragma unroll
    for (int b = 0; b < N; ++b)  // x-lines (b, c)
      if (line_hangs<K, 0>(m, b, c)) {
        if (b == 0) interp_line<N, 0, 1, false>(sv, px);
        else if (b == 1) interp_line<N, N, 1, false>(sv, px);
        else if (b == 2) interp_line<N, (2 < N ? 2 : 0) * N, 1, false>(sv, px);
        else if (b == 3) interp_line<N, (3 < N ? 3 : 0) * N, 1, false>(sv, px);
        else interp_line<N, (4 < N ? 4 : 0) * N, 1, false>(sv, px);
      }
  }
#pragma unroll
  for (int a = 0; a < N; ++a)  // y-lines (a, c)
    if (line_hangs<K, 1>(m, a, c)) {
      if (a == 0) interp_line<N, 0, N, TRANS>(sv, py);
      else if (a == 1) interp_line<N, 1, N, TRANS>(sv, py);
      else if (a == 2) interp_line<N, (2 < N ? 2 : 0), N, TRANS>(sv, py);
      else if (a == 3) interp_line<N, (3 < N ? 3 : 0), N, TRANS>(sv, py);
      else interp_line<N, (4 < N ? 4 : 0), N, TRANS>(sv, py);
    }
  if (TRANS) {
#pragma unroll
    for (int b = 0; b < N; ++b)
      if (line_hangs<K, 0>(m, b, c)) {
        if (b == 0) interp_line<N, 0, 1, true>(sv, px);
        else if (b == 1) interp_line<N, N, 1, true>(sv, px);
        else if (b == 2) interp_line<N, (2 < N ? 2 : 0) * N, 1, true>(sv, px);
        else if (b == 3) interp_line<N, (3 < N ? 3 : 0) * N, 1, true>(sv, px);
        else interp_line<N, (4 < N ? 4 : 0) * N, 1, true>(sv, px);
      }
  }
}

// C_z (or its transpose) on the z-lines held by thread t in the z layout
template <int K, bool TRANS>
__device__ __forceinline__ void slab_hanging_z(float* zv, uint16_t m, int t) {
  constexpr int N = K + 1;
  const int pz = (m >> 2) & 1;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int pr = t * N + i, a = pr % N, b = pr / N;
    if (line_hangs<K, 2>(m, a, b)) {
      if (i == 0) interp_line<N, 0, 1, TRANS>(zv, pz);
      else if (i == 1) interp_line<N, N, 1, TRANS>(zv, pz);
      else if (i == 2) interp_line<N, (2 < N ? 2 : 0) * N, 1, TRANS>(zv, pz);
      else if (i == 3) interp_line<N, (3 < N ? 3 : 0) * N, 1, TRANS>(zv, pz);
      else interp_line<N, (4 < N ? 4 : 0) * N, 1, TRANS>(zv, pz);
    }
  }
}

// slab layout (thread c: nodes (a, b, c)) <-> z layout (thread t: z-lines of
// the pairs a + N b = t N + i, stored as zv[i N + c]) through the cell region
template <int K>
__device__ __forceinline__ void to_z(const float* sv, float* zv, float* reg, int c) {
  constexpr int N = K + 1, N2 = N * N;
#pragma unroll
  for (int p = 0; p < N2; ++p) reg[p + N2 * c] = sv[p];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int z = 0; z < N; ++z) zv[i * N + z] = reg[c * N + i + N2 * z];
  __syncwarp();
}

template <int K>
__device__ __forceinline__ void to_slab(const float* zv, float* sv, float* reg, int c) {
  constexpr int N = K + 1, N2 = N * N;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int z = 0; z < N; ++z) reg[c * N + i + N2 * z] = zv[i * N + z];
  __syncwarp();
#pragma unroll
  for (int p = 0; p < N2; ++p) sv[p] = reg[p + N2 * c];
  __syncwarp();
}

template <int N, int L = 0>
__device__ __forceinline__ void slab_sweeps_xy(float* sv, const float (&Be)[NMAX][NMAX], bool fwd) {
  if constexpr (L < N) {
    if (fwd) {
      eo_forward<N, L * N, 1>(sv, Be);  // x-line b = L
    } else {
      eo_backward<N, L, N>(sv, Be);  // y-line a = L
    }
    slab_sweeps_xy<N, L + 1>(sv, Be, fwd);
  }
}

template <int N, int L = 0>
__device__ __forceinline__ void slab_sweeps_yx(float* sv, const float (&Be)[NMAX][NMAX], bool fwd) {
  if constexpr (L < N) {
    if (fwd) {
      eo_forward<N, L, N>(sv, Be);  // y-line a = L
    } else {
      eo_backward<N, L * N, 1>(sv, Be);  // x-line b = L
    }
    slab_sweeps_yx<N, L + 1>(sv, Be, fwd);
  }
}

template <int N, int L = 0>
__device__ __forceinline__ void z_lines(float* zv, const float (&Be)[NMAX][NMAX], const float* lam3, int t, float h) {
  if constexpr (L < N) {
    eo_forward<N, L * N, 1>(zv, Be);
    const int pr = t * N + L;  // mode pair (a, b) of this line
#pragma unroll
    for (int z = 0; z < N; ++z) zv[L * N + z] *= h * lam3[pr + N * N * z];
    eo_backward<N, L * N, 1>(zv, Be);
    z_lines<N, L + 1>(zv, Be, lam3, t, h);
  }
}

template <int K>
__global__ void __launch_bounds__(11 * 32, 2) vmult_slab(CellArgs<float> A) {
  pdl_begin();
  using G = SlabGeom<K>;
  constexpr int N = G::N, N2 = G::N2, N3 = G::N3, CPW = G::CPW;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tc = A.tc;
  uint16_t* sm_ls = reinterpret_cast<uint16_t*>(smem);  // [slot][cell]
  uint16_t* sm_mask = sm_ls + NSLOT * tc;
  uint16_t* sm_lev = sm_mask + tc;
  uint16_t* sm_sub = sm_lev + tc;
  float* lam3 = reinterpret_cast<float*>(smem + (((size_t)tc * (NSLOT + 3) * 2 + 15) & ~(size_t)15));
  float* creg = lam3 + N3;           // per-cell transposition regions, (tc + 1) x N3
  float* buf = creg + (tc + 1) * N3;  // tile DoFs (padded): input, then the accumulator
  __shared__ int any_hanging;
  const TileInfo ti = A.tiles[A.tile0 + blockIdx.x];
  const int nc = ti.n_cells;
  const int nloc = ti.n_owned + ti.n_foreign;
  const int nthr = blockDim.x;
  if (threadIdx.x == 0) any_hanging = 0;
  for (int i = threadIdx.x; i < N3; i += nthr) lam3[i] = tab<float>(K).lam3[i];
  for (int i = threadIdx.x; i < nc * 32; i += nthr) {
    const int cell = i >> 5, w = i & 31;
    const uint16_t v = reinterpret_cast<const uint16_t*>(A.meta + ti.cell_begin + cell)[w];
    if (w < NSLOT)
      sm_ls[w * tc + cell] = v;
    else if (w == NSLOT)
      sm_mask[cell] = v;
    else if (w == NSLOT + 1) {
      sm_lev[cell] = v & 0xFF;
      sm_sub[cell] = v >> 8;
    }
  }
  {
    const float* src = A.src + ti.dof_begin;
#pragma unroll 4
    for (int i = threadIdx.x; i < ti.n_owned; i += nthr) buf[swz(i)] = __ldg(src + i);
    const int32_t* fl = A.foreign + ti.foreign_begin;
#pragma unroll 4
    for (int i = threadIdx.x; i < ti.n_foreign; i += nthr) buf[swz(ti.n_owned + i)] = __ldg(A.src + __ldg(fl + i));
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = lane / N, c = lane - j * N;  // cell in warp, slab index
  const int q = warp * CPW + j;
  const bool active = (j < CPW) && (q < nc);
  const int qq = active ? q : 0;
  const int cc = c == 0 ? 0 : (c == K ? 2 : 1);
  const uint16_t m = active ? sm_mask[qq] : 0;
  float* reg = creg + (active ? q : tc) * N3;  // idle lanes use a spare region
  float sv[N2], zv[N2];
  slab_gather<K>(sv, buf, sm_ls, tc, qq, c, cc, active);  // G_e
  __syncthreads();  // the tile DoFs are no longer needed: reuse as accumulator
  for (int i = threadIdx.x; i < nloc + (nloc >> 6) + 1; i += nthr) buf[i] = 0.f;
  if (m & MASK_HANG) any_hanging = 1;
  const DevTables<float>& tb = tab<float>(K);
  const bool hz = (m & MASK_HANG) != 0;  // C_e needs the z layout too
  if (__any_sync(0xffffffffu, hz && active)) {
    to_z<K>(sv, zv, reg, c);
    if (hz) slab_hanging_z<K, false>(zv, m, c);
    to_slab<K>(zv, sv, reg, c);
    if (hz) slab_hanging_xy<K, false>(sv, m, c);
  }
  slab_sweeps_xy<N>(sv, tb.Be, true);   // B along x
  slab_sweeps_yx<N>(sv, tb.Be, true);   // B along y
  to_z<K>(sv, zv, reg, c);
  float h = active ? ldexpf((float)A.dom, -(int)sm_lev[qq]) : 0.f;
  if (A.coef && active) h = (float)cell_scale(A, A.dom, sm_lev[qq], ti.cell_begin + qq);
  z_lines<N>(zv, tb.Be, lam3, c, h);    // B, h (lam_a + lam_b + lam_c), B^T along z
  to_slab<K>(zv, sv, reg, c);
  slab_sweeps_yx<N>(sv, tb.Be, false);  // B^T along y
  slab_sweeps_xy<N>(sv, tb.Be, false);  // B^T along x
  if (__any_sync(0xffffffffu, hz && active)) {
    if (hz) slab_hanging_xy<K, true>(sv, m, c);
    to_z<K>(sv, zv, reg, c);
    if (hz) slab_hanging_z<K, true>(zv, m, c);
    to_slab<K>(zv, sv, reg, c);
  }
  const uint32_t hs = hanging_slots(m);
  const uint32_t skip = active ? hs : 0x7FFFFFFu;
  const bool zlo = c < K;
  __syncthreads();
  // G_e^T in eight side steps (the z side is fixed by the slab index)
  if (zlo) slab_scatter<K, 0>(buf, sv, sm_ls, tc, qq, c, cc, skip);
  __syncthreads();
  if (zlo) slab_scatter<K, 1>(buf, sv, sm_ls, tc, qq, c, cc, skip);
  __syncthreads();
  if (zlo) slab_scatter<K, 2>(buf, sv, sm_ls, tc, qq, c, cc, skip);
  __syncthreads();
  if (zlo) slab_scatter<K, 3>(buf, sv, sm_ls, tc, qq, c, cc, skip);
  __syncthreads();
  if (!zlo) slab_scatter<K, 0>(buf, sv, sm_ls, tc, qq, c, cc, skip);
  __syncthreads();
  if (!zlo) slab_scatter<K, 1>(buf, sv, sm_ls, tc, qq, c, cc, skip);
  __syncthreads();
  if (!zlo) slab_scatter<K, 2>(buf, sv, sm_ls, tc, qq, c, cc, skip);
  __syncthreads();
  if (!zlo) slab_scatter<K, 3>(buf, sv, sm_ls, tc, qq, c, cc, skip);
  __syncthreads();
  if (any_hanging) {  // hanging slots: several fine cells reach one coarse entity
    const int my_sub = (active && hs) ? sm_sub[qq] : -1;
    for (int sc = 0; sc < ti.n_sub; ++sc) {
      if (my_sub == sc) slab_scatter_hanging<K, true>(buf, sv, sm_ls, tc, qq, c, cc, hs);
      __syncthreads();
    }
  }
  {
    float* d = A.dst + ti.dof_begin;
    if (A.add)
      for (int i = threadIdx.x; i < ti.n_owned; i += nthr) d[i] += buf[swz(i)];
    else
      for (int i = threadIdx.x; i < ti.n_owned; i += nthr) d[i] = buf[swz(i)];
    const int32_t* hp = A.halo_pos + ti.foreign_begin;
    for (int i = threadIdx.x; i < ti.n_foreign; i += nthr) A.halo[hp[i]] = buf[swz(ti.n_owned + i)];
  }
}

// second pass: every DoF that other tiles contributed to adds its halo slots
// in a fixed order
// Every halo DoF has at least one slot; a thread takes HU DoFs and issues all
// their index, destination and first-slot loads before it adds (memory-level
// parallelism: the pass is a chain of dependent loads per DoF otherwise)
constexpr int HU = 8;
template <typename T>
__global__ void __launch_bounds__(BLOCK) halo_add_kernel(T* dst, const T* halo, const int32_t* dofs,
                                                         const int32_t* ptr, int nh) {
  pdl_begin();
  const int base = blockIdx.x * (BLOCK * HU) + threadIdx.x;
  int g[HU], e0[HU], e1[HU];
#pragma unroll
  for (int k = 0; k < HU; ++k) {
    const int u = base + k * BLOCK;
    g[k] = -1;
    if (u < nh) {
      g[k] = dofs[u];
      e0[k] = ptr[u];
      e1[k] = ptr[u + 1];
    }
  }
  T s[HU], f[HU];
#pragma unroll
  for (int k = 0; k < HU; ++k)
    if (g[k] >= 0) {
      s[k] = dst[g[k]];
      f[k] = halo[e0[k]];
    }
#pragma unroll
  for (int k = 0; k < HU; ++k)
    if (g[k] >= 0) {
      T a = s[k] + f[k];
      for (int e = e0[k] + 1; e < e1[k]; ++e) a += halo[e];  // the DoF's slots are contiguous, fixed order
      dst[g[k]] = a;
    }
}

// diagonal of C_m^T A_ref C_m for every mask m: virtual cells (m, column j)
// run the same pipeline on the unit vector e_j (Eq. 3 column by column,
// Eq. 4 with the constraints applied on both sides)
template <int K>
__global__ void __launch_bounds__(BLOCK) diag_table_kernel(double* out, int tc) {
  pdl_begin();
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

#ifndef GCMG_BODIES_ONLY  // host code: launchers (the device work list compiles the kernels only)
template <typename KERN>
void ensure_smem(KERN kernel, size_t bytes) {
  smem_allow(kernel, bytes);
}

// the fp32 line kernel with enough lines per thread for the level's tiles of
// at most L.tc cells
template <int K>
void launch_lines_f32(const CellLaunch& L, int n_tiles, size_t sm, cudaStream_t s, const CellArgs<float>& A) {
  constexpr int N2 = (K + 1) * (K + 1);
  constexpr int LMAX = (CHUNK * N2 + BLOCK - 1) / BLOCK;
  const int lpt = (L.tc * N2 + BLOCK - 1) / BLOCK;
  if (lpt <= 1) {
    ensure_smem(vmult_lines<K, float, 1>, sm);
    launch_pdl(vmult_lines<K, float, 1>, n_tiles, BLOCK, sm, s, A);
  } else if (lpt <= 2 && LMAX > 2) {
    ensure_smem(vmult_lines<K, float, (LMAX > 2 ? 2 : LMAX)>, sm);
    launch_pdl(vmult_lines<K, float, (LMAX > 2 ? 2 : LMAX)>, n_tiles, BLOCK, sm, s, A);
  } else {
    ensure_smem(vmult_lines<K, float, LMAX>, sm);
    launch_pdl(vmult_lines<K, float, LMAX>, n_tiles, BLOCK, sm, s, A);
  }
}

template <typename T>
void run_halo(const CellLaunch& L, T* dst, cudaStream_t s) {
  if (L.n_halo == 0) return;
  const int nb = (L.n_halo + BLOCK * HU - 1) / (BLOCK * HU);
  launch_pdl(halo_add_kernel<T>, nb, BLOCK, 0, s, dst, static_cast<const T*>(L.halo), L.halo_dofs, L.halo_ptr,
             L.n_halo);
  note_launches(1);
}

template <int K, typename T, int MODE, int NT>
void launch_cells_nt(const CellLaunch& L, CellArgs<T> A, size_t sm, cudaStream_t s) {
  ensure_smem(cell_kernel<K, T, MODE, NT>, sm);
  launch_pdl(cell_kernel<K, T, MODE, NT>, L.n_tiles, NT, sm, s, A);
  note_launches(1);
}

template <int K, typename T, int MODE>
void run_cells(const CellLaunch& L, CellArgs<T> A, cudaStream_t s) {
  if constexpr (MODE == MODE_VMULT && sizeof(T) == 8) {
    if (A.geom && L.tc <= CHUNK) {  // mapped cells, fp64 operator: double-float arithmetic on the FP32 pipe
      const size_t smm = mapped_df_smem((K + 1) * (K + 1) * (K + 1), L.tc, L.max_local);
      ensure_smem(vmult_lines_df<K, true>, smm);
      launch_pdl(vmult_lines_df<K, true>, L.n_tiles, BLOCK, smm, s, A);
      note_launches(1);
      run_halo<T>(L, A.dst, s);
      return;
    }
  }
  if (A.geom) {  // mapped cells: the chunked kernel with the quadrature-point geometry, every mode
    const size_t smm = smem_layout<T>((K + 1) * (K + 1) * (K + 1), L.tc, L.max_local, true, MODE == MODE_DIAG).total;
    launch_cells_nt<K, T, MODE, BLOCK>(L, A, smm, s);
    run_halo<T>(L, A.dst, s);
    return;
  }
  const size_t sm = smem_layout<T>((K + 1) * (K + 1) * (K + 1), L.tc, L.max_local).total;
  if constexpr (MODE == MODE_VMULT && sizeof(T) == 8) {
    // (a recorded launch list takes the BLOCK-thread line kernels: the persistent kernel has BLOCK threads)
    if (L.use_lanes && lanes_ok(L) && !dwl_recording()) {  // one lane per cell, double-float arithmetic (default)
      launch_vmult_lanes_df(L, A.src, A.dst, A.add, 0, L.n_tiles, s);
      run_halo<T>(L, A.dst, s);
      return;
    }
    if (L.tc <= CHUNK) {  // fp64 operator: double-float arithmetic on the FP32 pipe
      const size_t sm1 = sm - (size_t)L.max_local * sizeof(T);
      ensure_smem(vmult_lines_df<K>, sm1);
      launch_pdl(vmult_lines_df<K>, L.n_tiles, BLOCK, sm1, s, A);
      note_launches(1);
      run_halo<T>(L, A.dst, s);
      return;
    }
  }
  if constexpr (MODE == MODE_VMULT && sizeof(T) == 4) {
    if (L.use_lanes && lanes_ok(L) && !dwl_recording()) {  // one lane per cell (default)
      launch_vmult_lanes(L, A.src, A.dst, A.add, 0, L.n_tiles, s);
      run_halo<T>(L, A.dst, s);
      return;
    }
    if (L.tc <= CHUNK && (L.threads == BLOCK || dwl_recording())) {
      // vmult_lines keeps one tile-DoF buffer (input, then accumulator) plus K-1 <= 4 zero slots
      const size_t sm1 = sm - (size_t)L.max_local * sizeof(T) + 16;
      launch_lines_f32<K>(L, L.n_tiles, sm1, s, A);
      note_launches(1);
      run_halo<T>(L, A.dst, s);
      return;
    }
  }
  // the thread count is a tuning parameter of the fp32 operator only
  const int nt = (MODE == MODE_VMULT && sizeof(T) == 4 && !dwl_recording()) ? L.threads : BLOCK;
  if (nt == 128)
    launch_cells_nt<K, T, MODE, 128>(L, A, sm, s);
  else if (nt == 384)
    launch_cells_nt<K, T, MODE, 384>(L, A, sm, s);
  else if (nt == 512)
    launch_cells_nt<K, T, MODE, 512>(L, A, sm, s);
  else
    launch_cells_nt<K, T, MODE, BLOCK>(L, A, sm, s);
  run_halo<T>(L, A.dst, s);
}

template <int K>
void run_regs(const CellLaunch& L, CellArgs<float> A, cudaStream_t s) {
  const size_t sm = slab_smem<K>(L.tc, L.max_local);
  ensure_smem(vmult_slab<K>, sm);
  {
    launch_pdl(vmult_slab<K>, L.n_tiles, slab_warps<K>(L.tc) * 32, sm, s, A);
    note_launches(1);
  }
  run_halo<float>(L, A.dst, s);
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
  A.halo = static_cast<T*>(L.halo);
  A.halo_pos = L.halo_pos;
  A.lo = L.lo;
  A.dom = L.dom;
  A.coef = L.coef;
  A.geom = L.geom;
  A.geps = L.geps;
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

#endif  // GCMG_BODIES_ONLY
}  // namespace

#ifndef GCMG_BODIES_ONLY
size_t cell_smem_bytes(int k, bool fp64, int tc, int max_local, bool mapped) {
  const int n3 = (k + 1) * (k + 1) * (k + 1);
  return fp64 ? smem_layout<double>(n3, tc, max_local, mapped, mapped).total
              : smem_layout<float>(n3, tc, max_local, mapped, mapped).total;
}

void launch_vmult(const CellLaunch& L, bool fp64, const void* src, void* dst, int add, cudaStream_t s) {
  if (L.n_tiles == 0) return;
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
    if (L.tc > 64 || L.use_lines || L.geom || dwl_recording()) {
      dispatch<float, MODE_VMULT>(L, A, s);
      return;
    }
    switch (L.k) {
      case 1: run_regs<1>(L, A, s); break;
      case 2: run_regs<2>(L, A, s); break;
      case 3: run_regs<3>(L, A, s); break;
      case 4: run_regs<4>(L, A, s); break;
      default: break;
    }
  }
}

bool vmult_tiles_ok(const CellLaunch& L, bool fp64) {
  if (L.use_lanes && lanes_ok(L)) return true;
  return L.tc <= CHUNK && !L.geom && (fp64 || (L.use_lines && L.threads == BLOCK));
}

void launch_vmult_tiles(const CellLaunch& L, bool fp64, const void* src, void* dst, int t0, int t1, cudaStream_t s) {
  if (t1 <= t0 || !vmult_tiles_ok(L, fp64)) return;
  const int n3 = (L.k + 1) * (L.k + 1) * (L.k + 1);
  if (fp64) {
    if (L.use_lanes && lanes_ok(L)) {
      launch_vmult_lanes_df(L, static_cast<const double*>(src), static_cast<double*>(dst), 0, t0, t1, s);
      return;
    }
    CellArgs<double> A = make_args<double>(L);
    A.src = static_cast<const double*>(src);
    A.dst = static_cast<double*>(dst);
    A.tile0 = t0;
    const size_t sm = smem_layout<double>(n3, L.tc, L.max_local).total - (size_t)L.max_local * sizeof(double);
    switch (L.k) {
      case 1: ensure_smem(vmult_lines_df<1>, sm); launch_pdl(vmult_lines_df<1>, t1 - t0, BLOCK, sm, s, A); break;
      case 2: ensure_smem(vmult_lines_df<2>, sm); launch_pdl(vmult_lines_df<2>, t1 - t0, BLOCK, sm, s, A); break;
      case 3: ensure_smem(vmult_lines_df<3>, sm); launch_pdl(vmult_lines_df<3>, t1 - t0, BLOCK, sm, s, A); break;
      case 4: ensure_smem(vmult_lines_df<4>, sm); launch_pdl(vmult_lines_df<4>, t1 - t0, BLOCK, sm, s, A); break;
      default: return;
    }
  } else {
    if (L.use_lanes && lanes_ok(L)) {
      launch_vmult_lanes(L, src, dst, 0, t0, t1, s);
      return;
    }
    CellArgs<float> A = make_args<float>(L);
    A.src = static_cast<const float*>(src);
    A.dst = static_cast<float*>(dst);
    A.tile0 = t0;
    const size_t sm = smem_layout<float>(n3, L.tc, L.max_local).total - (size_t)L.max_local * sizeof(float) + 16;
    switch (L.k) {
      case 1: launch_lines_f32<1>(L, t1 - t0, sm, s, A); break;
      case 2: launch_lines_f32<2>(L, t1 - t0, sm, s, A); break;
      case 3: launch_lines_f32<3>(L, t1 - t0, sm, s, A); break;
      case 4: launch_lines_f32<4>(L, t1 - t0, sm, s, A); break;
      default: return;
    }
  }
  note_launches(1);
}

void launch_rhs(const CellLaunch& L, const RhsDesc& f, double* dst, cudaStream_t s) {
  if (L.n_tiles == 0) return;
  CellArgs<double> A = make_args<double>(L);
  A.dst = dst;
  A.fn = f;
  dispatch<double, MODE_RHS>(L, A, s);
}

void launch_rhs_lift(const CellLaunch& L, const RhsDesc& u, double* dst, cudaStream_t s) {
  if (L.n_tiles == 0) return;
  CellArgs<double> A = make_args<double>(L);
  A.dst = dst;
  A.add = 1;
  A.fn = u;
  dispatch<double, MODE_LIFT>(L, A, s);
}

void launch_diag(const CellLaunch& L, const double* diag_tab, double* dst, cudaStream_t s) {
  if (L.n_tiles == 0) return;
  CellArgs<double> A = make_args<double>(L);
  A.dst = dst;
  A.diag_tab = diag_tab;
  dispatch<double, MODE_DIAG>(L, A, s);
}

void launch_halo_add(const CellLaunch& L, bool fp64, void* dst, cudaStream_t s) {
  if (fp64)
    run_halo<double>(L, static_cast<double*>(dst), s);
  else
    run_halo<float>(L, static_cast<float*>(dst), s);
}

void launch_diag_table(int k, double* tab_out, cudaStream_t s) {
  const int n3 = (k + 1) * (k + 1) * (k + 1);
  const int tc = 32;
  const size_t sm = (((size_t)tc * 10 + 15) & ~(size_t)15) + (size_t)tc * n3 * sizeof(double);
  const int nb = (512 * n3 + tc - 1) / tc;
  switch (k) {
    case 1: { launch_pdl(diag_table_kernel<1>, nb, BLOCK, sm, s, tab_out, tc); note_launches(1); } break;
    case 2: { launch_pdl(diag_table_kernel<2>, nb, BLOCK, sm, s, tab_out, tc); note_launches(1); } break;
    case 3: { launch_pdl(diag_table_kernel<3>, nb, BLOCK, sm, s, tab_out, tc); note_launches(1); } break;
    case 4: { launch_pdl(diag_table_kernel<4>, nb, BLOCK, sm, s, tab_out, tc); note_launches(1); } break;
    default: break;
  }
}

namespace {

template <int K>
__global__ void coef_harmonic_kernel(int64_t n_cells, const double* __restrict__ nu_q, double* __restrict__ nu) {
  constexpr int N = K + 1, N3 = N * N * N;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const DevTables<double>& tb = tab<double>(K);
  double sw = 0.0, s = 0.0;
  for (int q = 0; q < N3; ++q) {
    const double w = tb.gw[q % N] * tb.gw[(q / N) % N] * tb.gw[q / (N * N)];
    sw += w;
    s += w / nu_q[c * N3 + q];
  }
  nu[c] = sw / s;
}

__global__ void check_positive_kernel(const double* __restrict__ v, int64_t n, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[i];
    if (!(x > 0.0 && x <= 1.7976931348623157e308)) *bad = 1;
  }
}

__global__ void coef_coarsen_kernel(int n_coarse, const int32_t* __restrict__ fine_of, const uint8_t* __restrict__ refined,
                                    const double* __restrict__ nu_f, double* __restrict__ nu_c) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_coarse) return;
  const int32_t f = fine_of[c];
  if (!refined[c]) {
    nu_c[c] = nu_f[f];
    return;
  }
  double s = 0.0;
  for (int q = 0; q < 8; ++q) s += nu_f[f + q];
  nu_c[c] = s / 8.0;
}

template <int K>
__global__ void quadrature_points_kernel(int64_t n_cells, const CellMeta* __restrict__ meta,
                                         const int32_t* __restrict__ ijk, double lo, double dom,
                                         double* __restrict__ xyz) {
  constexpr int N = K + 1, N3 = N * N * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_cells * N3) return;
  const int64_t c = t / N3;
  const int q = (int)(t - c * N3);
  const int qi[3] = {q % N, (q / N) % N, q / (N * N)};
  const double h = ldexp(dom, -(int)meta[c].level);
  for (int d = 0; d < 3; ++d) xyz[3 * t + d] = lo + h * ((double)ijk[3 * c + d] + tab<double>(K).gq[qi[d]]);
}

}  // namespace

void launch_coef_harmonic(int k, int64_t n_cells, const double* nu_q, double* nu, cudaStream_t s) {
  if (n_cells == 0) return;
  const int grid = (int)((n_cells + 255) / 256);
  switch (k) {
    case 1: coef_harmonic_kernel<1><<<grid, 256, 0, s>>>(n_cells, nu_q, nu); break;
    case 2: coef_harmonic_kernel<2><<<grid, 256, 0, s>>>(n_cells, nu_q, nu); break;
    case 3: coef_harmonic_kernel<3><<<grid, 256, 0, s>>>(n_cells, nu_q, nu); break;
    case 4: coef_harmonic_kernel<4><<<grid, 256, 0, s>>>(n_cells, nu_q, nu); break;
    default: return;
  }
  note_launches(1);
}

void launch_check_positive(const double* v, int64_t n, int* bad, cudaStream_t s) {
  if (n == 0) return;
  const int64_t g = std::min<int64_t>((n + 255) / 256, 152 * 8);
  check_positive_kernel<<<(int)g, 256, 0, s>>>(v, n, bad);
  note_launches(1);
}

void launch_coef_coarsen(int n_coarse, const int32_t* fine_of, const uint8_t* refined, const double* nu_f,
                         double* nu_c, cudaStream_t s) {
  if (n_coarse == 0) return;
  coef_coarsen_kernel<<<(n_coarse + 255) / 256, 256, 0, s>>>(n_coarse, fine_of, refined, nu_f, nu_c);
  note_launches(1);
}

void launch_quadrature_points(const CellLaunch& L, int64_t n_cells, double* xyz, cudaStream_t s) {
  const int n3 = (L.k + 1) * (L.k + 1) * (L.k + 1);
  const int64_t n = n_cells * n3;
  if (n == 0) return;
  const int grid = (int)((n + 255) / 256);
  switch (L.k) {
    case 1: quadrature_points_kernel<1><<<grid, 256, 0, s>>>(n_cells, L.meta, L.cell_ijk, L.lo, L.dom, xyz); break;
    case 2: quadrature_points_kernel<2><<<grid, 256, 0, s>>>(n_cells, L.meta, L.cell_ijk, L.lo, L.dom, xyz); break;
    case 3: quadrature_points_kernel<3><<<grid, 256, 0, s>>>(n_cells, L.meta, L.cell_ijk, L.lo, L.dom, xyz); break;
    case 4: quadrature_points_kernel<4><<<grid, 256, 0, s>>>(n_cells, L.meta, L.cell_ijk, L.lo, L.dom, xyz); break;
    default: return;
  }
  note_launches(1);
}

void dwl_register_cell() {
  int id = DWL_BASE_CELL;
#define GCMG_DWL_REG(fn) dwl_register(reinterpret_cast<const void*>(fn), id++, dwl_args_size(fn));
  GCMG_DWL_CELL(GCMG_DWL_REG)
#undef GCMG_DWL_REG
}

#endif  // GCMG_BODIES_ONLY
}  // namespace gcmg
