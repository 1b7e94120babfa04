// Transfer kernels between two levels (Sec. 3.5, Eqs. 5-7).
//
// Prolongation, cell loop over the coarse cells (coarse-side identification):
//   x_f += sum_e S_e^(f) W_e^(f) P_e^(f,c) C_e^(c) G_e^(c) x_c
// * G^(c), C^(c): gather the coarse cell values with the hanging-node
//   interpolation, exactly as in the operator (same tables, same mask);
// * P_e per category (Eq. 7): geometric coarsening has two categories,
//   "refined" (the element prolongation onto the 2k+1 nodes per direction of
//   the eight children, a tensor product of 1D matrices) and "not refined"
//   (identity); polynomial coarsening has one (degree k/2 -> k, 1D matrices);
// * W^(f): every fine DoF receives equal values from all cells that share it
//   (continuity of the coarse function), so the valence weighting is realised
//   as owner selection: exactly one (fine cell, slot) writes each fine DoF,
//   constrained fine DoFs are skipped.  Writes never collide: no atomics.
// Restriction is the exact transpose (R = P^T): the owner gathers the fine
// value, the transposed 1D matrices and C^T follow, and the coarse cells add
// into the coarse vector through the coarse level's tiles, colour by colour.
#include "device.cuh"
#include "kernels.h"

namespace gcmg {

#ifndef GCMG_BODIES_ONLY
GCMG_DEFINE_UPLOAD(upload_tables_transfer)
#endif

namespace {

constexpr int TP = 8;  // coarse cells expanded at a time

template <int KT, int WHICH, typename T>
__device__ __forceinline__ T pm(int i, int a) {
  return WHICH == 0 ? tab<T>(KT).Ph[i][a] : tab<T>(KT).Pp[i][a];
}

// apply the 1D matrix P along axis D: input extents (e0, e1, e2) with
// e_D = NI, output extent along D = NO.  TRANS: out[a] = sum_i P[i][a] in[i]
template <int KT, int WHICH, int NI, int NO, int D, bool TRANS, typename T>
__device__ __forceinline__ void tsweep(const T* in, T* out, int e0, int e1, int e2, int ncells, int in_cs,
                                       int out_cs, const uint8_t* act) {
  const int nl = (D == 0) ? e1 * e2 : (D == 1 ? e0 * e2 : e0 * e1);
  for (int t = threadIdx.x; t < ncells * nl; t += blockDim.x) {
    const int cell = t / nl, r = t - cell * nl;
    if (act && !act[cell]) continue;
    int ib, is, ob, os;
    if (D == 0) {
      const int y = r % e1, z = r / e1;
      ib = e0 * (y + e1 * z);
      is = 1;
      ob = NO * (y + e1 * z);
      os = 1;
    } else if (D == 1) {
      const int x = r % e0, z = r / e0;
      ib = x + e0 * e1 * z;
      is = e0;
      ob = x + e0 * NO * z;
      os = e0;
    } else {
      const int x = r % e0, y = r / e0;
      ib = x + e0 * y;
      is = e0 * e1;
      ob = ib;
      os = is;
    }
    const T* pi = in + cell * in_cs + ib;
    T* po = out + cell * out_cs + ob;
    T v[NI];
#pragma unroll
    for (int a = 0; a < NI; ++a) v[a] = pi[a * is];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      T s = 0;
#pragma unroll
      for (int a = 0; a < NI; ++a) s += (TRANS ? pm<KT, WHICH, T>(a, o) : pm<KT, WHICH, T>(o, a)) * v[a];
      po[o * os] = s;
    }
  }
}

template <typename T>
struct TArgs {
  int n_coarse;
  const int32_t* fine_of;
  const uint8_t* refined;
  const int32_t* gstart_f;
  const uint32_t* own_f;
  const int32_t* gstart_c;
  const uint16_t* mask_c;
  const T* src;
  T* dst;
  // restriction: rhs set: restrict rhs - src (the residual b - A x, the same
  // subtraction as the residual kernel) instead of src; overwrite: dst = R r
  // instead of dst += R r (before the halo pass adds the foreign slots)
  const T* rhs;
  int overwrite;
  // restriction: coarse tiles
  const TileInfo* tiles;
  T* halo;
  const int32_t* halo_pos;
  const CellMeta* meta;
  const int32_t* foreign;
  const uint16_t* subptr;
  const uint8_t* perm;
  int tc;
  int max_local;
};

// ---------------------------------------------------------------------------
// geometric (h) transfer, degree K on both levels
// ---------------------------------------------------------------------------
template <int K, typename T>
__global__ void __launch_bounds__(BLOCK) prolong_h(TArgs<T> A) {
  pdl_begin();
  constexpr int N = K + 1, N3 = N * N * N, M = 2 * K + 1, M3 = M * M * M;
  constexpr int S1 = M * N * N, S2 = M * M * N;
  constexpr int RG = 8;  // loads in flight per thread
  __shared__ uint16_t sm_mask[TP];
  __shared__ uint8_t sm_ref[TP];
  __shared__ int32_t sm_fine[TP];
  __shared__ int32_t sm_gsc[TP * NSLOT];       // coarse cells' global slot starts
  __shared__ uint32_t sm_own[TP * 8];          // ownership masks of the fine cells
#ifdef GCMG_DWL_POOL  // the persistent kernel: one pool for every kernel's largest array
  int32_t* sm_gs = reinterpret_cast<int32_t*>(GCMG_DWL_POOL);
  static_assert(TP * 8 * NSLOT * 4 <= GCMG_DWL_POOL_BYTES, "pool");
#else
  __shared__ int32_t sm_gs[TP * 8 * NSLOT];    // their global slot starts (-1: none)
#endif
  __shared__ uint16_t s_so[N3];                // per local node: entity slot | offset << 5
  __shared__ uint16_t s_e3[8 * N3];            // child q, node n -> position in the 2k+1 lattice
  extern __shared__ __align__(16) unsigned char smem[];
  T* cb = reinterpret_cast<T*>(smem);
  T* e2 = cb + TP * N3;
  T* e3 = e2 + TP * S2;
  T* e1 = e3;  // e1 is dead before the z sweep writes e3
  const int c0 = blockIdx.x * TP;
  const int nc = min(TP, A.n_coarse - c0);
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    sm_mask[c] = A.mask_c[c0 + c];
    sm_ref[c] = A.refined[c0 + c];
    sm_fine[c] = A.fine_of[c0 + c];
  }
  for (int i = threadIdx.x; i < 8 * N3; i += blockDim.x) {
    const int q = i / N3, n = i - q * N3;
    const int a = n % N, b = (n / N) % N, c = n / (N * N);
    if (q == 0) {
      int slot, off;
      node_slot<K>(a, b, c, slot, off);
      s_so[n] = (uint16_t)(slot | (off << 5));
    }
    s_e3[i] = (uint16_t)(((q & 1) * K + a) + M * ((((q >> 1) & 1) * K + b) + M * ((q >> 2) * K + c)));
  }
  for (int t = threadIdx.x; t < nc * NSLOT; t += blockDim.x) cp_async(sm_gsc + t, A.gstart_c + (size_t)c0 * NSLOT + t);
  __syncthreads();
  // the fine cells' slot starts and ownership (children of a refined cell are consecutive),
  // asynchronous copies all in flight at once
  for (int t = threadIdx.x; t < nc * 8 * NSLOT; t += blockDim.x) {
    const int jq = t / NSLOT, slot = t - jq * NSLOT, j = jq >> 3, q = jq & 7;
    const bool use = sm_fine[j] >= 0 && (sm_ref[j] || q == 0);  // fine_of < 0: no fine cells
    const int f = sm_fine[j] + q;
    if (use)
      cp_async(sm_gs + t, A.gstart_f + (size_t)f * NSLOT + slot);
    else
      sm_gs[t] = -1;
    if (slot == 0) {
      if (use)
        cp_async(sm_own + jq, A.own_f + f);
      else
        sm_own[jq] = 0u;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // G^(c): the coarse values (RG loads in flight per thread)
  for (int t0 = threadIdx.x; t0 < nc * N3; t0 += RG * BLOCK) {
    T v[RG];
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      const int t = t0 + u * BLOCK;
      v[u] = T(0);
      if (t < nc * N3) {
        const int cell = t / N3, n = t - cell * N3, so = s_so[n];
        const int32_t g = sm_gsc[cell * NSLOT + (so & 31)];
        if (g >= 0) v[u] = A.src[g + (so >> 5)];
      }
    }
#pragma unroll
    for (int u = 0; u < RG; ++u)
      if (t0 + u * BLOCK < nc * N3) cb[t0 + u * BLOCK] = v[u];
  }
  __syncthreads();
  hanging_all<K, false>(cb, sm_mask, nc);
  tsweep<K, 0, N, M, 0, false>(cb, e1, N, N, N, nc, N3, S1, sm_ref);
  __syncthreads();
  tsweep<K, 0, N, M, 1, false>(e1, e2, M, N, N, nc, S1, S2, sm_ref);
  __syncthreads();
  tsweep<K, 0, N, M, 2, false>(e2, e3, M, M, N, nc, S2, M3, sm_ref);
  __syncthreads();
  // owner-selected additions to the fine vector (RG read-modify-writes in flight)
  const int ntot = nc * 8 * N3;
  for (int t0 = threadIdx.x; t0 < ntot; t0 += RG * BLOCK) {
    int idx[RG];
    T val[RG];
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      const int t = t0 + u * BLOCK;
      idx[u] = -1;
      if (t < ntot) {
        const int j = t / (8 * N3), r = t - j * 8 * N3;  // r = q N3 + n
        const int q = r / N3, n = r - q * N3;
        const int so = s_so[n], slot = so & 31;
        if ((sm_own[j * 8 + q] >> slot) & 1u) {
          idx[u] = sm_gs[(j * 8 + q) * NSLOT + slot] + (so >> 5);
          val[u] = sm_ref[j] ? e3[j * M3 + s_e3[r]] : cb[j * N3 + n];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RG; ++u)
      if (idx[u] >= 0) atomicAdd(A.dst + idx[u], val[u]);
  }
}

// scatter the chunk's coarse cells (positions c0.. in sub-colour order) into
// the tile accumulator, sub-colour by sub-colour
template <int KC, typename T>
__device__ __forceinline__ void restrict_scatter(const TArgs<T>& A, const TileInfo& ti, const CellMeta* sm_meta,
                                                 const uint16_t* sm_cell, int c0, int np, const T* cb, T* ys) {
  constexpr int N = KC + 1, N2 = N * N, N3 = N2 * N;
  for (int s = 0; s < ti.n_sub; ++s) {
    const int q0 = max(c0, (int)A.subptr[ti.sub_begin + s]);
    const int q1 = min(c0 + np, (int)A.subptr[ti.sub_begin + s + 1]);
    if (q1 <= q0) continue;
    for (int t = threadIdx.x; t < (q1 - q0) * N2; t += blockDim.x) {
      const int j = q0 - c0 + t / N2, r = t % N2;
      const int b = r % N, c = r / N;
      const uint16_t* ls = sm_meta[sm_cell[j]].ls;
      const T* in = cb + j * N3 + N * r;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        int slot, off;
        node_slot<KC>(a, b, c, slot, off);
        const uint16_t l = ls[slot];
        if (l != LS_NONE) ys[l + off] += in[a];
      }
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void restrict_write(const TArgs<T>& A, const TileInfo& ti, const T* ys) {
  T* dst = A.dst + ti.dof_begin;
  if (A.overwrite)
    for (int i = threadIdx.x; i < ti.n_owned; i += blockDim.x) dst[i] = ys[i];
  else
    for (int i = threadIdx.x; i < ti.n_owned; i += blockDim.x) dst[i] += ys[i];
  const int32_t* hp = A.halo_pos + ti.foreign_begin;
  for (int i = threadIdx.x; i < ti.n_foreign; i += blockDim.x) A.halo[hp[i]] = ys[ti.n_owned + i];
}

// TPC coarse cells are expanded at a time: 8, or 4 on levels with many tiles
// (at k = 4, 5 instead of 3 CTAs per SM; on levels of one or two waves the
// longer chain of chunks per tile costs more than the occupancy gains)
template <int K, typename T, int TPC>
__global__ void __launch_bounds__(BLOCK) restrict_h(TArgs<T> A) {
  pdl_begin();
  constexpr int N = K + 1, N3 = N * N * N, M = 2 * K + 1, M3 = M * M * M;
  constexpr int S1 = M * N * N, S2 = M * M * N;
  __shared__ uint8_t sm_ref[TPC];
  __shared__ int32_t sm_fine[TPC];
  __shared__ uint16_t sm_mask[TPC];
  __shared__ uint16_t sm_cell[TPC];
  __shared__ uint32_t sm_own[TPC * 8];          // ownership masks of the fine cells
#ifdef GCMG_DWL_POOL
  int32_t* sm_gs = reinterpret_cast<int32_t*>(GCMG_DWL_POOL);
  static_assert(TPC * 8 * NSLOT * 4 <= GCMG_DWL_POOL_BYTES, "pool");
#else
  __shared__ int32_t sm_gs[TPC * 8 * NSLOT];    // their global slot starts (-1: none)
#endif
  __shared__ uint16_t s_so[N3];                // per local node: entity slot | offset << 5
  __shared__ uint16_t s_e3[8 * N3];            // child q, node n -> position in the 2k+1 lattice
  extern __shared__ __align__(16) unsigned char smem[];
  CellMeta* sm_meta = reinterpret_cast<CellMeta*>(smem);
  T* cb = reinterpret_cast<T*>(smem + (size_t)A.tc * sizeof(CellMeta));
  T* e2 = cb + TPC * N3;
  T* e3 = e2 + TPC * S2;
  T* e1 = e3;  // e3 is dead once the z sweep has read it
  T* ys = e3 + TPC * M3;
  const TileInfo ti = A.tiles[blockIdx.x];
  const int nc = ti.n_cells;
  {
    const uint4* g = reinterpret_cast<const uint4*>(A.meta + ti.cell_begin);
    uint4* s = reinterpret_cast<uint4*>(sm_meta);
    for (int i = threadIdx.x; i < nc * 4; i += blockDim.x) s[i] = g[i];
  }
  for (int i = threadIdx.x; i < ti.n_owned + ti.n_foreign; i += blockDim.x) ys[i] = T(0);
  for (int i = threadIdx.x; i < 8 * N3; i += blockDim.x) {
    const int q = i / N3, n = i - q * N3;
    const int a = n % N, b = (n / N) % N, c = n / (N * N);
    if (q == 0) {
      int slot, off;
      node_slot<K>(a, b, c, slot, off);
      s_so[n] = (uint16_t)(slot | (off << 5));
    }
    s_e3[i] = (uint16_t)(((q & 1) * K + a) + M * ((((q >> 1) & 1) * K + b) + M * ((q >> 2) * K + c)));
  }
  for (int c0 = 0; c0 < nc; c0 += TPC) {
    const int np = min(TPC, nc - c0);
    __syncthreads();
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
      const int cell = A.perm[ti.cell_begin + c0 + j];
      sm_cell[j] = (uint16_t)cell;
      sm_ref[j] = A.refined[ti.cell_begin + cell];
      sm_fine[j] = A.fine_of[ti.cell_begin + cell];
      sm_mask[j] = A.mask_c[ti.cell_begin + cell];
    }
    for (int i = threadIdx.x; i < np * M3; i += blockDim.x) e3[i] = T(0);
    for (int i = threadIdx.x; i < np * N3; i += blockDim.x) cb[i] = T(0);
    __syncthreads();
    // the fine cells' slot starts and ownership, coalesced (children of a
    // refined coarse cell are consecutive fine cells)
    for (int t = threadIdx.x; t < np * 8 * NSLOT; t += blockDim.x) {
      const int jq = t / NSLOT, slot = t - jq * NSLOT, j = jq >> 3, q = jq & 7;
      const bool use = sm_fine[j] >= 0 && (sm_ref[j] || q == 0);  // fine_of < 0: no fine cells
      const int f = sm_fine[j] + q;
      if (use)
        cp_async(sm_gs + t, A.gstart_f + (size_t)f * NSLOT + slot);
      else
        sm_gs[t] = -1;
      if (slot == 0) {
        if (use)
          cp_async(sm_own + jq, A.own_f + f);
        else
          sm_own[jq] = 0u;
      }
    }
    cp_async_wait_all();
    __syncthreads();
    // gather the owned fine values (RG loads in flight per thread: 16 takes the finest Q4
    // restriction from 0.199 to 0.182 ms, 32 gains nothing more)
    constexpr int RG = 16;
    const int ntot = np * 8 * N3;
    for (int t0 = threadIdx.x; t0 < ntot; t0 += RG * BLOCK) {
      T val[RG];
      int dst[RG];
#pragma unroll
      for (int u = 0; u < RG; ++u) {
        const int t = t0 + u * BLOCK;
        dst[u] = -1;
        if (t < ntot) {
          const int j = t / (8 * N3), r = t - j * 8 * N3;  // r = q N3 + n
          const int q = r / N3, n = r - q * N3;
          const int so = s_so[n], slot = so & 31;
          if ((sm_own[j * 8 + q] >> slot) & 1u) {
            const int gi = sm_gs[(j * 8 + q) * NSLOT + slot] + (so >> 5);
            val[u] = A.rhs ? A.rhs[gi] - A.src[gi] : A.src[gi];
            // refined: position in the children's 2k+1 lattice; else the
            // identity category (marked by the offset TPC M3): into cb
            dst[u] = sm_ref[j] ? j * M3 + s_e3[r] : TPC * M3 + j * N3 + n;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < RG; ++u) {
        if (dst[u] < 0) continue;
        if (dst[u] >= TPC * M3)
          cb[dst[u] - TPC * M3] = val[u];
        else
          e3[dst[u]] = val[u];
      }
    }
    __syncthreads();
    tsweep<K, 0, M, N, 2, true>(e3, e2, M, M, M, np, M3, S2, sm_ref);
    __syncthreads();
    tsweep<K, 0, M, N, 1, true>(e2, e1, M, M, N, np, S2, S1, sm_ref);
    __syncthreads();
    tsweep<K, 0, M, N, 0, true>(e1, cb, M, N, N, np, S1, N3, sm_ref);
    __syncthreads();
    hanging_all<K, true>(cb, sm_mask, np);  // C^(c)T
    restrict_scatter<K>(A, ti, sm_meta, sm_cell, c0, np, cb, ys);
  }
  __syncthreads();
  restrict_write(A, ti, ys);
}

// ---------------------------------------------------------------------------
// polynomial (p) transfer on one mesh, degree KF -> KC = KF / 2
// ---------------------------------------------------------------------------
template <int KF, typename T>
__global__ void __launch_bounds__(BLOCK) prolong_p(TArgs<T> A) {
  pdl_begin();
  constexpr int KC = KF / 2, NF = KF + 1, NC = KC + 1;
  constexpr int NC3 = NC * NC * NC, NF3 = NF * NF * NF, S1 = NF * NC * NC, S2 = NF * NF * NC;
  __shared__ uint16_t sm_mask[TP];
  extern __shared__ __align__(16) unsigned char smem[];
  T* cb = reinterpret_cast<T*>(smem);
  T* e1 = cb + TP * NC3;
  T* e2 = e1 + TP * S1;
  T* e3 = e2 + TP * S2;
  const int c0 = blockIdx.x * TP;
  const int nc = min(TP, A.n_coarse - c0);
  for (int c = threadIdx.x; c < nc; c += blockDim.x) sm_mask[c] = A.mask_c[c0 + c];
  constexpr int RG = 8;  // independent chains of loads in flight per thread
  for (int t0 = threadIdx.x; t0 < nc * NC3; t0 += RG * BLOCK) {
    T v[RG];
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      const int t = t0 + u * BLOCK;
      v[u] = T(0);
      if (t < nc * NC3) {
        const int cell = t / NC3, n = t - cell * NC3;
        int slot, off;
        node_slot<KC>(n % NC, (n / NC) % NC, n / (NC * NC), slot, off);
        const int32_t g = A.gstart_c[(size_t)(c0 + cell) * NSLOT + slot];
        if (g >= 0) v[u] = A.src[g + off];
      }
    }
#pragma unroll
    for (int u = 0; u < RG; ++u)
      if (t0 + u * BLOCK < nc * NC3) cb[t0 + u * BLOCK] = v[u];
  }
  __syncthreads();
  hanging_all<KC, false>(cb, sm_mask, nc);
  tsweep<KF, 1, NC, NF, 0, false>(cb, e1, NC, NC, NC, nc, NC3, S1, nullptr);
  __syncthreads();
  tsweep<KF, 1, NC, NF, 1, false>(e1, e2, NF, NC, NC, nc, S1, S2, nullptr);
  __syncthreads();
  tsweep<KF, 1, NC, NF, 2, false>(e2, e3, NF, NF, NC, nc, S2, NF3, nullptr);
  __syncthreads();
  // owner-selected additions (each fine DoF once: red.add gives the read-modify-write's sum)
  for (int t0 = threadIdx.x; t0 < nc * NF3; t0 += RG * BLOCK) {
    int idx[RG];
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      const int t = t0 + u * BLOCK;
      idx[u] = -1;
      if (t < nc * NF3) {
        const int cell = t / NF3, n = t - cell * NF3;
        const int f = c0 + cell;
        int slot, off;
        node_slot<KF>(n % NF, (n / NF) % NF, n / (NF * NF), slot, off);
        if ((A.own_f[f] >> slot) & 1u) idx[u] = A.gstart_f[(size_t)f * NSLOT + slot] + off;
      }
    }
#pragma unroll
    for (int u = 0; u < RG; ++u)
      if (idx[u] >= 0) atomicAdd(A.dst + idx[u], e3[t0 + u * BLOCK]);
  }
}

template <int KF, typename T>
__global__ void __launch_bounds__(BLOCK) restrict_p(TArgs<T> A) {
  pdl_begin();
  constexpr int KC = KF / 2, NF = KF + 1, NC = KC + 1;
  constexpr int NC3 = NC * NC * NC, NF3 = NF * NF * NF, S1 = NF * NC * NC, S2 = NF * NF * NC;
  __shared__ uint16_t sm_mask[TP];
  __shared__ uint16_t sm_cell[TP];
  extern __shared__ __align__(16) unsigned char smem[];
  CellMeta* sm_meta = reinterpret_cast<CellMeta*>(smem);
  T* cb = reinterpret_cast<T*>(smem + (size_t)A.tc * sizeof(CellMeta));
  T* e1 = cb + TP * NC3;
  T* e2 = e1 + TP * S1;
  T* e3 = e2 + TP * S2;
  T* ys = e3 + TP * NF3;
  const TileInfo ti = A.tiles[blockIdx.x];
  const int nc = ti.n_cells;
  {
    const uint4* g = reinterpret_cast<const uint4*>(A.meta + ti.cell_begin);
    uint4* s = reinterpret_cast<uint4*>(sm_meta);
    for (int i = threadIdx.x; i < nc * 4; i += blockDim.x) s[i] = g[i];
  }
  for (int i = threadIdx.x; i < ti.n_owned + ti.n_foreign; i += blockDim.x) ys[i] = T(0);
  for (int c0 = 0; c0 < nc; c0 += TP) {
    const int np = min(TP, nc - c0);
    __syncthreads();
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
      const int cell = A.perm[ti.cell_begin + c0 + j];
      sm_cell[j] = (uint16_t)cell;
      sm_mask[j] = A.mask_c[ti.cell_begin + cell];
    }
    __syncthreads();
    constexpr int RG = 8;  // independent chains of loads in flight per thread
    for (int t0 = threadIdx.x; t0 < np * NF3; t0 += RG * BLOCK) {
      T v[RG];
#pragma unroll
      for (int u = 0; u < RG; ++u) {
        const int t = t0 + u * BLOCK;
        v[u] = T(0);
        if (t < np * NF3) {
          const int j = t / NF3, n = t - j * NF3;
          const int f = ti.cell_begin + sm_cell[j];
          int slot, off;
          node_slot<KF>(n % NF, (n / NF) % NF, n / (NF * NF), slot, off);
          if ((A.own_f[f] >> slot) & 1u) {
            const int gi = A.gstart_f[(size_t)f * NSLOT + slot] + off;
            v[u] = A.rhs ? A.rhs[gi] - A.src[gi] : A.src[gi];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < RG; ++u)
        if (t0 + u * BLOCK < np * NF3) e3[t0 + u * BLOCK] = v[u];
    }
    __syncthreads();
    tsweep<KF, 1, NF, NC, 2, true>(e3, e2, NF, NF, NF, np, NF3, S2, nullptr);
    __syncthreads();
    tsweep<KF, 1, NF, NC, 1, true>(e2, e1, NF, NF, NC, np, S2, S1, nullptr);
    __syncthreads();
    tsweep<KF, 1, NF, NC, 0, true>(e1, cb, NF, NC, NC, np, S1, NC3, nullptr);
    __syncthreads();
    hanging_all<KC, true>(cb, sm_mask, np);
    restrict_scatter<KC>(A, ti, sm_meta, sm_cell, c0, np, cb, ys);
  }
  __syncthreads();
  restrict_write(A, ti, ys);
}

template <typename T>
TArgs<T> targs(const TransferLaunch& L) {
  TArgs<T> A{};
  A.n_coarse = L.n_coarse;
  A.fine_of = L.fine_of;
  A.refined = L.refined;
  A.gstart_f = L.gstart_f;
  A.own_f = L.own_f;
  A.gstart_c = L.gstart_c;
  A.mask_c = L.mask_c;
  A.tiles = L.coarse.tiles;
  A.halo = static_cast<T*>(L.coarse.halo);
  A.halo_pos = L.coarse.halo_pos;
  A.meta = L.coarse.meta;
  A.foreign = L.coarse.foreign;
  A.subptr = L.coarse.subptr;
  A.perm = L.coarse.perm;
  A.tc = L.coarse.tc;
  A.max_local = L.coarse.max_local;
  return A;
}

#ifndef GCMG_BODIES_ONLY  // host code: launchers (the device work list compiles the kernels only)
template <typename K_>
void set_smem(K_ kernel, size_t bytes) {
  smem_allow(kernel, bytes);
}

template <int K, typename T>
void prolong_h_run(const TransferLaunch& L, const T* src, T* dst, cudaStream_t s) {
  constexpr int N = K + 1, M = 2 * K + 1;
  const size_t sm = (size_t)TP * (N * N * N + M * M * N + M * M * M) * sizeof(T);  // cb, e2, e3 (= e1)
  set_smem(prolong_h<K, T>, sm);
  TArgs<T> A = targs<T>(L);
  A.src = src;
  A.dst = dst;
  const int nb = (L.n_coarse + TP - 1) / TP;
  { launch_pdl(prolong_h<K, T>, nb, BLOCK, sm, s, A); note_launches(1); }
}

template <int K, typename T, int TPC>
void restrict_h_launch(const TransferLaunch& L, const T* src, T* dst, const T* rhs, bool ow, cudaStream_t s) {
  constexpr int N = K + 1, M = 2 * K + 1;
  const size_t sm = (size_t)L.coarse.tc * sizeof(CellMeta) +
                    ((size_t)TPC * (N * N * N + M * M * N + M * M * M) + L.coarse.max_local) * sizeof(T);
  set_smem(restrict_h<K, T, TPC>, sm);
  TArgs<T> A = targs<T>(L);
  A.src = src;
  A.dst = dst;
  A.rhs = rhs;
  A.overwrite = ow;
  launch_pdl(restrict_h<K, T, TPC>, L.coarse.n_tiles, BLOCK, sm, s, A);
  note_launches(1);
}

template <int K, typename T>
void restrict_h_run(const TransferLaunch& L, const T* src, T* dst, const T* rhs, bool ow, cudaStream_t s) {
  // (a recorded launch list takes 4-cell chunks: less shared memory per CTA of the persistent kernel)
  if (L.coarse.chunk == 4 || dwl_recording() || (L.coarse.chunk == 0 && L.coarse.n_tiles > 4 * L.coarse.n_sm))
    restrict_h_launch<K, T, 4>(L, src, dst, rhs, ow, s);
  else
    restrict_h_launch<K, T, TP>(L, src, dst, rhs, ow, s);
  launch_halo_add(L.coarse, sizeof(T) == 8, dst, s);
}

template <int KF, typename T>
void prolong_p_run(const TransferLaunch& L, const T* src, T* dst, cudaStream_t s) {
  constexpr int NF = KF + 1, NC = KF / 2 + 1;
  const size_t sm = (size_t)TP * (NC * NC * NC + NF * NC * NC + NF * NF * NC + NF * NF * NF) * sizeof(T);
  set_smem(prolong_p<KF, T>, sm);
  TArgs<T> A = targs<T>(L);
  A.src = src;
  A.dst = dst;
  const int nb = (L.n_coarse + TP - 1) / TP;
  { launch_pdl(prolong_p<KF, T>, nb, BLOCK, sm, s, A); note_launches(1); }
}

template <int KF, typename T>
void restrict_p_run(const TransferLaunch& L, const T* src, T* dst, const T* rhs, bool ow, cudaStream_t s) {
  constexpr int NF = KF + 1, NC = KF / 2 + 1;
  const size_t sm = (size_t)L.coarse.tc * sizeof(CellMeta) +
                    ((size_t)TP * (NC * NC * NC + NF * NC * NC + NF * NF * NC + NF * NF * NF) + L.coarse.max_local) *
                        sizeof(T);
  set_smem(restrict_p<KF, T>, sm);
  TArgs<T> A = targs<T>(L);
  A.src = src;
  A.dst = dst;
  A.rhs = rhs;
  A.overwrite = ow;
  { launch_pdl(restrict_p<KF, T>, L.coarse.n_tiles, BLOCK, sm, s, A); note_launches(1); }
  launch_halo_add(L.coarse, sizeof(T) == 8, dst, s);
}

template <typename T>
void prolong_any(const TransferLaunch& L, const T* src, T* dst, cudaStream_t s) {
  if (L.kind == 0) {
    switch (L.kf) {
      case 1: prolong_h_run<1>(L, src, dst, s); break;
      case 2: prolong_h_run<2>(L, src, dst, s); break;
      case 3: prolong_h_run<3>(L, src, dst, s); break;
      case 4: prolong_h_run<4>(L, src, dst, s); break;
    }
  } else {
    switch (L.kf) {
      case 2: prolong_p_run<2>(L, src, dst, s); break;
      case 3: prolong_p_run<3>(L, src, dst, s); break;
      case 4: prolong_p_run<4>(L, src, dst, s); break;
    }
  }
}

template <typename T>
void restrict_any(const TransferLaunch& L, const T* src, T* dst, const T* rhs, bool ow, cudaStream_t s) {
  if (L.kind == 0) {
    switch (L.kf) {
      case 1: restrict_h_run<1>(L, src, dst, rhs, ow, s); break;
      case 2: restrict_h_run<2>(L, src, dst, rhs, ow, s); break;
      case 3: restrict_h_run<3>(L, src, dst, rhs, ow, s); break;
      case 4: restrict_h_run<4>(L, src, dst, rhs, ow, s); break;
    }
  } else {
    switch (L.kf) {
      case 2: restrict_p_run<2>(L, src, dst, rhs, ow, s); break;
      case 3: restrict_p_run<3>(L, src, dst, rhs, ow, s); break;
      case 4: restrict_p_run<4>(L, src, dst, rhs, ow, s); break;
    }
  }
}

#endif  // GCMG_BODIES_ONLY
}  // namespace

#ifndef GCMG_BODIES_ONLY
void launch_prolongate_add(const TransferLaunch& L, bool fp64, const void* coarse, void* fine, cudaStream_t s) {
  if (fp64)
    prolong_any<double>(L, static_cast<const double*>(coarse), static_cast<double*>(fine), s);
  else
    prolong_any<float>(L, static_cast<const float*>(coarse), static_cast<float*>(fine), s);
}

void launch_restrict_add(const TransferLaunch& L, bool fp64, const void* fine, void* coarse, cudaStream_t s) {
  if (fp64)
    restrict_any<double>(L, static_cast<const double*>(fine), static_cast<double*>(coarse), nullptr, false, s);
  else
    restrict_any<float>(L, static_cast<const float*>(fine), static_cast<float*>(coarse), nullptr, false, s);
}

void launch_restrict_residual(const TransferLaunch& L, bool fp64, const void* b, const void* Ax, void* coarse,
                              bool overwrite, cudaStream_t s) {
  if (fp64)
    restrict_any<double>(L, static_cast<const double*>(Ax), static_cast<double*>(coarse),
                         static_cast<const double*>(b), overwrite, s);
  else
    restrict_any<float>(L, static_cast<const float*>(Ax), static_cast<float*>(coarse), static_cast<const float*>(b),
                        overwrite, s);
}

void dwl_register_transfer() {
  int id = DWL_BASE_TRANSFER;
#define GCMG_DWL_REG(fn) dwl_register(reinterpret_cast<const void*>(fn), id++, dwl_args_size(fn));
  GCMG_DWL_TRANSFER(GCMG_DWL_REG)
#undef GCMG_DWL_REG
}

#endif  // GCMG_BODIES_ONLY
}  // namespace gcmg
