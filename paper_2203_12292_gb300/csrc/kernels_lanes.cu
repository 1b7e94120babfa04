// fp32 tile kernel of the cell loop of Eq. 2 with one lane per cell:
//   v = sum_e G_e^T C_e^T S_e^T Q_e S_e C_e G_e x
//
// A tile holds at most 32 consecutive (Morton-ordered) cells; lane j of every
// warp works on cell j, and the k+1 warps of the CTA share the (k+1)^2 1D
// lines of each direction.  All lanes of a warp therefore touch the same
// local node of 32 different cells at once, so
//   * the cell buffer is node-major (node n of cell j at n * 32 + j): every
//     access to it, in every direction, reads or writes 32 consecutive words
//     (no bank conflicts), and all indexing except the DoF gather/scatter is
//     uniform across the warp;
//   * the entity starts of the tile are stored transposed (slot s of cell j
//     at s * 32 + j), read conflict-free.
// The sweeps apply the fast-diagonalisation form of the Cartesian cell matrix
// h (K x M x M + M x K x M + M x M x K) = h B^T(x3) diag(lam_a+lam_b+lam_c) B(x3)
// with the even-odd split of B (rows of B are symmetric or antisymmetric
// under x -> 1 - x).
//
// Accumulation without atomics and in a fixed order.  Two local nodes of
// different cells can be the same DoF only if, along every axis, their
// coordinates are equal or both lie on the cell boundary (0 or k); the same
// holds through hanging faces and edges, whose slots point to the coarse
// entity with the same local offsets.
//   * fp32, tiles without hanging cells: warp w keeps the z-plane c = w of
//     its lane's cell in registers (gather, x and y sweeps forward; the z
//     phase through the cell buffer; y and x sweeps backward and the scatter).
//     The cell buffer and the tile's DoF buffer share one shared-memory
//     region (gathers finish before the cell buffer is written, the
//     accumulator is cleared after its last read; the tiles with hanging
//     cells hold their x-lines in registers across those points), so 8
//     blocks of 48 registers fit an SM at k = 4.
//     Planes c = 0 and c = k are the only ones that meet, so warp k adds after
//     warp 0 (a named barrier); a warp adds its nodes in program order.
//   * tiles with hanging cells, and the double-float kernel: the x-lines
//     (b, c) are grouped into classes by (b or "boundary", c or "boundary");
//     each class is given to one warp, so two warps never add to the same
//     DoF.  Within one instruction two lanes add to the same DoF only through
//     hanging slots (siblings behind one coarse face or edge), added one lane
//     after another in lane order.  These tiles apply C_e and C_e^T (Sec. 3.2,
//     direction by direction) between separate passes.
// The sums are therefore reproducible bit for bit.
#include <algorithm>
#include <map>
#include <vector>

#include "device.cuh"
#include "kernels.h"

namespace gcmg {

GCMG_DEFINE_UPLOAD(upload_tables_lanes_1d)

namespace {

constexpr int LW = 8;  // table entries of x-lines per warp

// x-line r = b + N c of degree K: slot of node (0, b, c) | byte offset of the
// node in its entity << 8 | byte offset of node (1, b, c) in the slot after it
// << 16; per warp the x-lines it gathers and scatters (-1: none),
// class-partitioned
struct LaneLines {
  uint32_t line[KMAX + 1][NMAX * NMAX];
  int8_t xw[KMAX + 1][NMAX][LW];
  int32_t nx[KMAX + 1][NMAX];  // x-lines of each warp
};
__constant__ LaneLines c_ll;

template <typename T>
struct LaneArgsT {
  const TileInfo* tiles;
  const LaneTile* lt;
  const LaneHang* lh;    // per tile: hanging lines and slots of every lane
  const int32_t* order;  // tile of block b: order[b] (null: tile0 + b)
  const TileInfo* tiles_lo;  // with order: block b's TileInfo, LaneTile, LaneHang at [b]
  const LaneTile* lt_lo;
  const LaneHang* lh_lo;
  int n_hang;            // with order: blocks below n_hang have tiles with hanging cells
  const int32_t* foreign;
  const int32_t* halo_pos;
  const T* src;
  T* dst;
  T* halo;
  const double* coef;  // per cell nu_e, null: 1
  double dom;
  int add;
  int tile0;
};
using LaneArgs = LaneArgsT<float>;

// child-side interpolation I_p (TRANS: its transpose) on one line in
// registers.  I_1[a][b] = I_0[k-a][k-b] (Gauss-Lobatto points and Lagrange
// basis are symmetric under x -> 1 - x), so p = 1 reverses the line, applies
// I_0 and reverses back: one set of constant-operand multiply-adds
template <int K, bool TRANS>
__device__ __forceinline__ void interp_line_reg(float* v, int p) {
  constexpr int N = K + 1;
  const DevTables<float>& tb = tab<float>(K);
  float x[N], y[N];
#pragma unroll
  for (int a = 0; a < N; ++a) x[a] = p ? v[K - a] : v[a];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < N; ++a) s += (TRANS ? tb.I[0][a][r] : tb.I[0][r][a]) * x[a];
    y[r] = s;
  }
#pragma unroll
  for (int a = 0; a < N; ++a) v[a] = p ? y[K - a] : y[a];
}

// one direction D of C_e (TRANS: C_e^T) on the lines of warp w: line
// q = i + N w has the other coordinates (u, v) = (q % N, q / N) in increasing
// axis order; lane j interpolates when the line lies on a hanging face or edge
// of its cell.  SWEEP (D = 2 only): the z sweep follows (forward after C_z) or
// precedes (backward before C_z^T) the interpolation on the same lines.
template <int K, int D, bool TRANS, bool SWEEP = false>
__device__ __forceinline__ void hang_pass(float* cb, uint16_t m, uint32_t hlD, int w, int lane) {
  constexpr int N = K + 1, N2 = N * N;
  constexpr int S = (D == 0 ? 1 : (D == 1 ? N : N2)) * 32;
  const DevTables<float>& tb = tab<float>(K);
  const int p = (m >> D) & 1;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int u = i, v = w;  // line (u, v): the other two coordinates
    const bool hl = (hlD >> (u + N * v)) & 1u;
    if (!SWEEP && !hl) continue;
    const int base = D == 0 ? N * u + N2 * v : (D == 1 ? u + N2 * v : u + N * v);
    float* ptr = cb + base * 32 + lane;
    float x[N];
#pragma unroll
    for (int a = 0; a < N; ++a) x[a] = ptr[a * S];
    if (SWEEP && TRANS) eo_backward<N, 0, 1>(x, tb.Be);
    if (hl) interp_line_reg<K, TRANS>(x, p);
    if (SWEEP && !TRANS) eo_forward<N, 0, 1>(x, tb.Be);
#pragma unroll
    for (int a = 0; a < N; ++a) ptr[a * S] = x[a];
  }
}

// *x += v where lanes with the same address (siblings behind one hanging face
// or edge) add one after another in lane order; absent DoFs (the zero region)
// add nothing.  Only lanes whose slot hangs can share an address within one
// instruction: without such a lane (hang_any = 0) the plain addition is exact.
__device__ __noinline__ void add_ordered_slow(float* x, float v, bool real, int lane) {
  const unsigned key = real ? (unsigned)__cvta_generic_to_shared(x) : ~(unsigned)lane;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int rank = __popc(peers & ((1u << lane) - 1u));
  const int most = __reduce_max_sync(0xffffffffu, (unsigned)__popc(peers));
  for (int q = 0; q < most; ++q) {
    if (real && rank == q) *x += v;
    __syncwarp();
  }
}

// (the ordered path out of line: the unrolled scatter of the tiles with hanging cells calls it
// at every node, and inlined it would multiply that code)
__device__ __forceinline__ void add_ordered(float* x, float v, bool real, int lane, bool hang_any) {
  if (!hang_any)
    *x += v;
  else
    add_ordered_slow(x, v, real, lane);
}

// zero the accumulator (n floats from the 16-byte aligned x0)
__device__ __forceinline__ void clear_acc(float* x0, int n, int nt) {
  float4* z4 = reinterpret_cast<float4*>(x0);
  for (int i = threadIdx.x; i < (n + 3) / 4; i += nt) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// named barrier `id` of n threads: producers arrive, consumers wait
__device__ __forceinline__ void named_bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// the three gather/scatter addresses of x-line r of the cell in this lane:
// node (0, b, c), first interior node (1, b, c), node (k, b, c)
template <int K>
__device__ __forceinline__ void xline_ptrs(const LaneTile* st, char* xb, int r, int lane, float*& p0, float*& p1,
                                           float*& p2) {
  const uint32_t li = c_ll.line[K][r];
  const int s0 = li & 0xff, o0 = (li >> 8) & 0xff, o1 = li >> 16;
  p0 = reinterpret_cast<float*>(xb + st->ls[s0][lane] + o0);
  p1 = reinterpret_cast<float*>(xb + st->ls[s0 + 1][lane] + o1);
  p2 = reinterpret_cast<float*>(xb + st->ls[s0 + 2][lane] + o0);
}

// y sweep on the lines (a, c) = (i, w) of warp w
template <int K, bool FWD>
__device__ __forceinline__ void sweep_y(float* cb, int w, int lane) {
  constexpr int N = K + 1, N2 = N * N;
  const DevTables<float>& tb = tab<float>(K);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float* p = cb + (i + N2 * w) * 32 + lane;
    float v[N];
#pragma unroll
    for (int b = 0; b < N; ++b) v[b] = p[b * N * 32];
    if (FWD)
      eo_forward<N, 0, 1>(v, tb.Be);
    else
      eo_backward<N, 0, 1>(v, tb.Be);
#pragma unroll
    for (int b = 0; b < N; ++b) p[b * N * 32] = v[b];
  }
}

template <int K>
__global__ void __launch_bounds__((K + 1) * 32, K == 4 ? 8 : 1) vmult_lanes(LaneArgs A) {
  pdl_begin();
  constexpr int N = K + 1, N2 = N * N, N3 = N2 * N, NT = N * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  LaneTile* st = reinterpret_cast<LaneTile*>(smem);
  LaneHang* hg = reinterpret_cast<LaneHang*>(smem + sizeof(LaneTile));
  // the cell buffer and the tile's DoF buffer (input, then accumulator) share one region: the
  // DoFs are gathered into registers before the cell buffer is written, and the accumulator
  // is cleared after the cell buffer's last read (8 instead of 7 blocks per SM at k = 4)
  float* cb = reinterpret_cast<float*>(smem + sizeof(LaneTile) + sizeof(LaneHang));
  float* xs0 = cb;  // 16-byte aligned
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // block b's tile: records in launch order at [b] (no dependent load of the tile index) or tile0 + b
  const int bx = blockIdx.x, tl = A.tile0 + bx;
  const LaneTile* ltp = A.order ? A.lt_lo + bx : A.lt + tl;
  const LaneHang* lhp = A.order ? A.lh_lo + bx : A.lh + tl;
  const TileInfo ti = A.order ? A.tiles_lo[bx] : A.tiles[tl];
  const int nloc = ti.n_owned + ti.n_foreign;
  // tile DoF i at xs[i] (then the zero region; later the accumulator): xs + i is 16-byte aligned
  // exactly where src + dof_begin + i is, so the owned range moves in 16-byte pieces
  const float* so = A.src + ti.dof_begin;
  const int sh = (int)((reinterpret_cast<uintptr_t>(so) >> 2) & 3);
  float* xs = xs0 + sh;
  const int h0 = min((4 - sh) & 3, ti.n_owned), nv = (ti.n_owned - h0) >> 2;
  {  // asynchronous copies of the lane metadata and the tile's DoFs, all in flight at once
    const uint4* g = reinterpret_cast<const uint4*>(ltp);
    uint4* s = reinterpret_cast<uint4*>(st);
    for (int i = threadIdx.x; i < (int)(sizeof(LaneTile) / 16); i += NT) cp_async16(s + i, g + i);
    if (!A.order || (int)blockIdx.x < A.n_hang) {  // the tile has hanging cells (or may have)
      const uint4* gh = reinterpret_cast<const uint4*>(lhp);
      uint4* shh = reinterpret_cast<uint4*>(hg);
      for (int i = threadIdx.x; i < (int)(sizeof(LaneHang) / 16); i += NT) cp_async16(shh + i, gh + i);
    }
    if (threadIdx.x < h0) cp_async(xs + threadIdx.x, so + threadIdx.x);
#pragma unroll 4
    for (int j = threadIdx.x; j < nv; j += NT) cp_async16(xs + h0 + 4 * j, so + h0 + 4 * j);
    for (int i = h0 + 4 * nv + threadIdx.x; i < ti.n_owned; i += NT) cp_async(xs + i, so + i);
    const int32_t* fl = A.foreign + ti.foreign_begin;
    float* xf = xs + ti.n_owned;
    for (int i0 = threadIdx.x; i0 < ti.n_foreign; i0 += 4 * NT) {
      int idx[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) idx[u] = (i0 + u * NT < ti.n_foreign) ? fl[i0 + u * NT] : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (idx[u] >= 0) cp_async(xf + i0 + u * NT, A.src + idx[u]);
    }
  }
  if (threadIdx.x < LANE_ZERO) xs[nloc + threadIdx.x] = 0.f;
  cp_async_wait_all();
  __syncthreads();

  const DevTables<float>& tb = tab<float>(K);
  const uint16_t m = st->mask[lane];
  const bool hang = st->hang != 0;  // uniform over the CTA
  float h;
  {
    const int c = ti.cell_begin + min(lane, ti.n_cells - 1);
    const double hd = ldexp(A.dom, -(int)st->level[lane]);
    h = (float)(A.coef ? hd * A.coef[c] : hd);
  }
  char* xb = reinterpret_cast<char*>(xs);
  const int nxl = c_ll.nx[K][w];

  if (!hang) {
    // Warp w holds the plane c = w of its cell in registers: G_e, the x and y
    // sweeps forward; the z phase through the cell buffer; the y and x sweeps
    // backward and G_e^T, again on the plane in registers.
    //   Plane x-lines (b, w): node (0, b, w) lies in slot 9 cls(w) + 3 cls(b),
    // nodes (1..k-1, b, w) in the slot after it, node (k, b, w) two after it;
    // their offsets in the entities are the same for b = 0 and b = k and grow
    // by one x-step (node (0, .)) or one x-line of the entity (node (1, .)) per
    // interior b (entity DoFs lexicographic over the interior axes).
    const uint32_t l0 = c_ll.line[K][N * w], l1 = c_ll.line[K][(K > 1 ? 1 : 0) + N * w];
    const uint16_t* lsw = &st->ls[l0 & 0xff][lane];
    const char* xA0 = xb + ((l0 >> 8) & 0xff);  // node (0, b, w), b = 0 or k
    const char* xA1 = xb + (l0 >> 16);          // node (1, b, w), b = 0 or k
    const char* xB0 = xb + ((l1 >> 8) & 0xff);  // node (0, 1, w)
    const char* xB1 = xb + (l1 >> 16);          // node (1, 1, w)
    float u[N2];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      const bool in = b > 0 && b < K;
      const int sb = b == 0 ? 0 : (b == K ? 6 : 3);
      const int q0 = lsw[(sb + 0) * 32], q1 = lsw[(sb + 1) * 32], q2 = lsw[(sb + 2) * 32];
      const float* p0 = reinterpret_cast<const float*>((in ? xB0 : xA0) + q0) + (in ? b - 1 : 0);
      const float* p1 = reinterpret_cast<const float*>((in ? xB1 : xA1) + q1) + (in ? (b - 1) * (K - 1) : 0);
      const float* p2 = reinterpret_cast<const float*>((in ? xB0 : xA0) + q2) + (in ? b - 1 : 0);
      u[N * b] = *p0;
#pragma unroll
      for (int a = 1; a < K; ++a) u[N * b + a] = p1[a - 1];
      u[N * b + K] = *p2;
    }
    __syncthreads();  // every plane gathered: the DoF buffer is dead
#pragma unroll
    for (int b = 0; b < N; ++b) eo_forward<N, 0, 1>(u + N * b, tb.Be);  // x-lines of the plane
#pragma unroll
    for (int a = 0; a < N; ++a) eo_forward<N, 0, N>(u + a, tb.Be);  // y-lines
    {
      float* p = cb + (N2 * w) * 32 + lane;
#pragma unroll
      for (int n = 0; n < N2; ++n) p[n * 32] = u[n];
    }
    __syncthreads();
    // z: forward sweep, h (lam_a + lam_b + lam_c) in mode order, backward sweep (lines (a, b) = (i, w))
    {
      const float hb = h * tb.lame[w];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float* p = cb + (i + N * w) * 32 + lane;
        float v[N];
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = p[c * N2 * 32];
        eo_forward<N, 0, 1>(v, tb.Be);
        const float hab = fmaf(h, tb.lame[i], hb);
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] *= fmaf(h, tb.lame[c], hab);
        eo_backward<N, 0, 1>(v, tb.Be);
#pragma unroll
        for (int c = 0; c < N; ++c) p[c * N2 * 32] = v[c];
      }
    }
    __syncthreads();
    {
      const float* p = cb + (N2 * w) * 32 + lane;
#pragma unroll
      for (int n = 0; n < N2; ++n) u[n] = p[n * 32];
    }
#pragma unroll
    for (int a = 0; a < N; ++a) eo_backward<N, 0, N>(u + a, tb.Be);
#pragma unroll
    for (int b = 0; b < N; ++b) eo_backward<N, 0, 1>(u + N * b, tb.Be);
    __syncthreads();  // every plane loaded: the cell buffer is dead
    clear_acc(xs0, sh + nloc, NT);
    __syncthreads();
    // G_e^T.  Nodes of two cells are one DoF only where every coordinate is
    // equal or both lie on the cell boundary: between planes only c = 0 and
    // c = k meet, so warp k adds after warp 0 (named barrier 1); within a
    // plane the x-lines and their nodes add in program order.
    if (w == K) named_bar_sync(1, 64);
#pragma unroll
    for (int b = 0; b < N; ++b) {
      const bool in = b > 0 && b < K;
      const int sb = b == 0 ? 0 : (b == K ? 6 : 3);
      const int q0 = lsw[(sb + 0) * 32], q1 = lsw[(sb + 1) * 32], q2 = lsw[(sb + 2) * 32];
      float* p0 = reinterpret_cast<float*>(const_cast<char*>(in ? xB0 : xA0) + q0) + (in ? b - 1 : 0);
      float* p1 = reinterpret_cast<float*>(const_cast<char*>(in ? xB1 : xA1) + q1) + (in ? (b - 1) * (K - 1) : 0);
      float* p2 = reinterpret_cast<float*>(const_cast<char*>(in ? xB0 : xA0) + q2) + (in ? b - 1 : 0);
      *p0 += u[N * b];
#pragma unroll
      for (int a = 1; a < K; ++a) p1[a - 1] += u[N * b + a];
      *p2 += u[N * b + K];
    }
    if (w == 0) named_bar_arrive(1, 64);
  } else {
    // G_e and C_x on the warp's x-lines, all gathered before the cell buffer is written
    constexpr int NXW = K <= 2 ? 4 : N;  // x-lines per warp at most
    float v[NXW][N];
#pragma unroll
    for (int i = 0; i < NXW; ++i)
      if (i < nxl) {
        const int r = c_ll.xw[K][w][i];
        float *p0, *p1, *p2;
        xline_ptrs<K>(st, xb, r, lane, p0, p1, p2);
        v[i][0] = *p0;
#pragma unroll
        for (int a = 1; a < K; ++a) v[i][a] = p1[a - 1];
        v[i][K] = *p2;
        if ((hg->hl[0][lane] >> r) & 1u) interp_line_reg<K, false>(v[i], m & 1);
      }
    __syncthreads();  // the DoF buffer is dead
#pragma unroll
    for (int i = 0; i < NXW; ++i)
      if (i < nxl) {
        float* p = cb + N * c_ll.xw[K][w][i] * 32 + lane;
#pragma unroll
        for (int a = 0; a < N; ++a) p[a * 32] = v[i][a];
      }
    __syncthreads();
    hang_pass<K, 1, false>(cb, m, hg->hl[1][lane], w, lane);  // C_y
    __syncthreads();
    hang_pass<K, 2, false, true>(cb, m, hg->hl[2][lane], w, lane);  // C_z, forward z sweep
    __syncthreads();
    sweep_y<K, true>(cb, w, lane);
    __syncthreads();
    // x: forward sweep, h (lam_a + lam_b + lam_c) in mode order, backward sweep (lines (b, c) = (i, w))
    {
      const float hc = h * tb.lame[w];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float* p = cb + N * (i + N * w) * 32 + lane;
        float v[N];
#pragma unroll
        for (int a = 0; a < N; ++a) v[a] = p[a * 32];
        eo_forward<N, 0, 1>(v, tb.Be);
        const float hbc = fmaf(h, tb.lame[i], hc);
#pragma unroll
        for (int a = 0; a < N; ++a) v[a] *= fmaf(h, tb.lame[a], hbc);
        eo_backward<N, 0, 1>(v, tb.Be);
#pragma unroll
        for (int a = 0; a < N; ++a) p[a * 32] = v[a];
      }
    }
    __syncthreads();
    sweep_y<K, false>(cb, w, lane);
    __syncthreads();
    hang_pass<K, 2, true, true>(cb, m, hg->hl[2][lane], w, lane);  // backward z sweep, C_z^T
    __syncthreads();
    hang_pass<K, 1, true>(cb, m, hg->hl[1][lane], w, lane);  // C_y^T
    __syncthreads();
    // C_x^T and G_e^T on the warp's class of x-lines: all lines read before the accumulator
    // (the same region) is cleared
#pragma unroll
    for (int i = 0; i < NXW; ++i)
      if (i < nxl) {
        const float* p = cb + N * c_ll.xw[K][w][i] * 32 + lane;
#pragma unroll
        for (int a = 0; a < N; ++a) v[i][a] = p[a * 32];
      }
    __syncthreads();  // the cell buffer is dead
    clear_acc(xs0, sh + nloc, NT);
    __syncthreads();
    const uint32_t hs = hg->hs[lane];
    const int zb = nloc * 4;  // byte offset of the zero region
#pragma unroll
    for (int i = 0; i < NXW; ++i) {
      if (i >= nxl) break;
      const int r = c_ll.xw[K][w][i];
      if ((hg->hl[0][lane] >> r) & 1u) interp_line_reg<K, true>(v[i], m & 1);
      const uint32_t li = c_ll.line[K][r];
      const int s0 = li & 0xff, o0 = (li >> 8) & 0xff, o1 = li >> 16;
      const int b0 = st->ls[s0][lane], b1 = st->ls[s0 + 1][lane], b2 = st->ls[s0 + 2][lane];
      float* p0 = reinterpret_cast<float*>(xb + b0 + o0);
      float* p1 = reinterpret_cast<float*>(xb + b1 + o1);
      float* p2 = reinterpret_cast<float*>(xb + b2 + o0);
      const bool h0 = __any_sync(0xffffffffu, (hs >> s0) & 1u), h1 = __any_sync(0xffffffffu, (hs >> (s0 + 1)) & 1u),
                 h2 = __any_sync(0xffffffffu, (hs >> (s0 + 2)) & 1u);
      add_ordered(p0, v[i][0], b0 != zb, lane, h0);
#pragma unroll
      for (int a = 1; a < K; ++a) add_ordered(p1 + a - 1, v[i][a], b1 != zb, lane, h1);
      add_ordered(p2, v[i][K], b2 != zb, lane, h2);
    }
  }
  __syncthreads();
  // owned DoFs: plain stores (or additions), 16 bytes at a time where src and dst are aligned
  // alike; foreign DoFs: into their halo slots
  float* d = A.dst + ti.dof_begin;
  if ((int)((reinterpret_cast<uintptr_t>(d) >> 2) & 3) == sh) {
    if (threadIdx.x < h0) d[threadIdx.x] = A.add ? d[threadIdx.x] + xs[threadIdx.x] : xs[threadIdx.x];
    for (int j = threadIdx.x; j < nv; j += NT) {
      float4 x4 = *reinterpret_cast<const float4*>(xs + h0 + 4 * j);
      float4* d4 = reinterpret_cast<float4*>(d + h0 + 4 * j);
      if (A.add) {
        const float4 o = *d4;
        x4 = make_float4(o.x + x4.x, o.y + x4.y, o.z + x4.z, o.w + x4.w);
      }
      *d4 = x4;
    }
    for (int i = h0 + 4 * nv + threadIdx.x; i < ti.n_owned; i += NT) d[i] = A.add ? d[i] + xs[i] : xs[i];
  } else {
    for (int i = threadIdx.x; i < ti.n_owned; i += NT) d[i] = A.add ? d[i] + xs[i] : xs[i];
  }
  const int32_t* hp = A.halo_pos + ti.foreign_begin;
  for (int i = threadIdx.x; i < ti.n_foreign; i += NT) A.halo[hp[i]] = xs[ti.n_owned + i];
}

// ---------------------------------------------------------------------------
// fp64 operator (the CG operator of the mixed solve and every level of the
// fp64 multigrid) with the same lane-per-cell structure: fp64 vectors in and
// out, all arithmetic in double-float (hi + lo floats, about 48 significand
// bits: error-free two-sum and fused product error, the fp64 tables split
// into high and low parts), on the FP32 pipe, which GB300 has many times
// wider than its FP64 pipe.  Values are converted once on entry to and once
// on exit from the tile; the cell buffer and the accumulator hold df pairs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ df df_sel(bool p, df a, df b) { return df{p ? a.hi : b.hi, p ? a.lo : b.lo}; }

// sum_j x_j c_j over T double-float values and double-float constants
// (ch + cl) with one normalisation: the high products p_j = x_j.hi ch_j carry
// their exact rounding errors (fused multiply-add), the p_j are summed by
// error-free two-sums, and the low-order terms (product errors, cross terms
// x.hi cl and x.lo ch, two-sum errors) go into one fp32 sum; 12 T - 5
// operations instead of 18 T - 11 for a chain of df_fma
template <int T>
__device__ __forceinline__ df df_dot(const df* x, const float* ch, const float* cl) {
  float S = __fmul_rn(x[0].hi, ch[0]);
  float L = __fmaf_rn(x[0].hi, cl[0], __fmaf_rn(x[0].lo, ch[0], __fmaf_rn(x[0].hi, ch[0], -S)));
#pragma unroll
  for (int j = 1; j < T; ++j) {
    const float p = __fmul_rn(x[j].hi, ch[j]);
    const float l = __fmaf_rn(x[j].hi, cl[j], __fmaf_rn(x[j].lo, ch[j], __fmaf_rn(x[j].hi, ch[j], -p)));
    const float s = __fadd_rn(S, p);
    const float z = __fsub_rn(s, S);
    const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(s, z)), __fsub_rn(p, z));
    S = s;
    L = __fadd_rn(L, __fadd_rn(l, t));
  }
  return df_norm(S, L);
}

// even-odd forward transform with B (nodal -> modes in mode order) and its
// backward transform, in double-float, rows as df_dot
template <int K>
__device__ __forceinline__ void df_eo_fwd_fast(df* u) {
  constexpr int N = K + 1, NH = N / 2, NE = (N + 1) / 2;
  const float(&Bh)[NMAX][NMAX] = c_tf[K].Be;
  const float(&Bl)[NMAX][NMAX] = c_tflo[K].Be;
  df e[NE], o[NH > 0 ? NH : 1];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    e[j] = df_add(u[j], u[N - 1 - j]);
    o[j] = df_sub(u[j], u[N - 1 - j]);
  }
  if (N % 2) e[NH] = u[NH];
#pragma unroll
  for (int r = 0; r < NE; ++r) u[r] = df_dot<NE>(e, Bh[r], Bl[r]);
#pragma unroll
  for (int r = 0; r < NH; ++r) u[NE + r] = df_dot<NH>(o, Bh[NE + r], Bl[NE + r]);
}

template <int K>
__device__ __forceinline__ void df_eo_bwd_fast(df* u) {
  constexpr int N = K + 1, NH = N / 2, NE = (N + 1) / 2;
  df E[NE], O[NH > 0 ? NH : 1];
  float ch[NMAX], cl[NMAX];
#pragma unroll
  for (int j = 0; j < NE; ++j) {
#pragma unroll
    for (int r = 0; r < NE; ++r) {
      ch[r] = c_tf[K].Be[r][j];
      cl[r] = c_tflo[K].Be[r][j];
    }
    E[j] = df_dot<NE>(u, ch, cl);
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) {
#pragma unroll
    for (int r = 0; r < NH; ++r) {
      ch[r] = c_tf[K].Be[NE + r][j];
      cl[r] = c_tflo[K].Be[NE + r][j];
    }
    O[j] = df_dot<NH>(u + NE, ch, cl);
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    u[j] = df_add(E[j], O[j]);
    u[N - 1 - j] = df_sub(E[j], O[j]);
  }
  if (N % 2) u[NH] = E[NH];
}

// I_p (TRANS: transposed) on one df line, by the mirror identity of interp_line_reg
template <int K, bool TRANS>
__device__ __forceinline__ void interp_line_df(df* v, int p) {
  constexpr int N = K + 1;
  const float(&Ih)[NMAX][NMAX] = c_tf[K].I[0];
  const float(&Il)[NMAX][NMAX] = c_tflo[K].I[0];
  df x[N], y[N];
#pragma unroll
  for (int a = 0; a < N; ++a) x[a] = df_sel(p, v[K - a], v[a]);
  float ch[NMAX], cl[NMAX];
#pragma unroll
  for (int r = 0; r < N; ++r) {
#pragma unroll
    for (int a = 0; a < N; ++a) {
      ch[a] = TRANS ? Ih[a][r] : Ih[r][a];
      cl[a] = TRANS ? Il[a][r] : Il[r][a];
    }
    y[r] = df_dot<N>(x, ch, cl);
  }
#pragma unroll
  for (int a = 0; a < N; ++a) v[a] = df_sel(p, y[K - a], y[a]);
}

template <int K, int D, bool TRANS, bool SWEEP = false>
__device__ __forceinline__ void hang_pass_df(df* cb, uint16_t m, uint32_t hlD, int w, int lane) {
  constexpr int N = K + 1, N2 = N * N;
  constexpr int S = (D == 0 ? 1 : (D == 1 ? N : N2)) * 32;
  const int p = (m >> D) & 1;
#pragma unroll 1
  for (int i = 0; i < N; ++i) {
    const int u = i, v = w;  // line (u, v): the other two coordinates
    const bool hl = (hlD >> (u + N * v)) & 1u;
    if (!SWEEP && !hl) continue;
    const int base = D == 0 ? N * u + N2 * v : (D == 1 ? u + N2 * v : u + N * v);
    df* ptr = cb + base * 32 + lane;
    df x[N];
#pragma unroll
    for (int a = 0; a < N; ++a) x[a] = ptr[a * S];
    if (SWEEP && TRANS) df_eo_bwd_fast<K>(x);
    if (hl) interp_line_df<K, TRANS>(x, p);
    if (SWEEP && !TRANS) df_eo_fwd_fast<K>(x);
#pragma unroll
    for (int a = 0; a < N; ++a) ptr[a * S] = x[a];
  }
}

template <int K, bool FWD>
__device__ __forceinline__ void sweep_y_df(df* cb, int w, int lane) {
  constexpr int N = K + 1, N2 = N * N;
#pragma unroll 1
  for (int i = 0; i < N; ++i) {
    df* p = cb + (i + N2 * w) * 32 + lane;
    df v[N];
#pragma unroll
    for (int b = 0; b < N; ++b) v[b] = p[b * N * 32];
    if (FWD)
      df_eo_fwd_fast<K>(v);
    else
      df_eo_bwd_fast<K>(v);
#pragma unroll
    for (int b = 0; b < N; ++b) p[b * N * 32] = v[b];
  }
}

// forward sweep, h (lam_a + lam_b + lam_c) in mode order, backward sweep on the
// lines along direction D (2: z-lines (a, b) = (i, w); 0: x-lines (b, c) = (i, w))
template <int K, int D>
__device__ __forceinline__ void sweep_scale_df(df* cb, int w, int lane, df h) {
  constexpr int N = K + 1, N2 = N * N;
  constexpr int S = (D == 0 ? 1 : N2) * 32;
#pragma unroll 1
  for (int i = 0; i < N; ++i) {
    df* p = cb + (D == 0 ? N * (i + N * w) : i + N * w) * 32 + lane;
    df v[N];
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = p[c * S];
    df_eo_fwd_fast<K>(v);
#pragma unroll
    for (int c = 0; c < N; ++c) {
      // mode index of the node: along D the line index c, the others (i, w)
      const int idx = D == 0 ? c + N * i + N2 * w : i + N * w + N2 * c;
      v[c] = df_mul(v[c], df_mul(df{c_tf[K].lam3[idx], c_tflo[K].lam3[idx]}, h));
    }
    df_eo_bwd_fast<K>(v);
#pragma unroll
    for (int c = 0; c < N; ++c) p[c * S] = v[c];
  }
}

__device__ __forceinline__ void add_ordered_df(df* x, df v, bool real, int lane, bool hang_any) {
  if (!hang_any) {
    *x = df_add(*x, v);
    return;
  }
  const unsigned key = real ? (unsigned)__cvta_generic_to_shared(x) : ~(unsigned)lane;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int rank = __popc(peers & ((1u << lane) - 1u));
  const int most = __reduce_max_sync(0xffffffffu, (unsigned)__popc(peers));
  for (int q = 0; q < most; ++q) {
    if (real && rank == q) *x = df_add(*x, v);
    __syncwarp();
  }
}

template <int K>
__global__ void __launch_bounds__((K + 1) * 32) vmult_lanes_df(LaneArgsT<double> A) {
  pdl_begin();
  constexpr int N = K + 1, N3 = N * N * N, NT = N * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  LaneTile* st = reinterpret_cast<LaneTile*>(smem);
  LaneHang* hg = reinterpret_cast<LaneHang*>(smem + sizeof(LaneTile));
  df* cb = reinterpret_cast<df*>(smem + sizeof(LaneTile) + sizeof(LaneHang));
  double* xd0 = reinterpret_cast<double*>(cb + N3 * 32);  // 16-byte aligned
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // block b's tile: records in launch order at [b] (no dependent load of the tile index) or tile0 + b
  const int bx = blockIdx.x, tl = A.tile0 + bx;
  const LaneTile* ltp = A.order ? A.lt_lo + bx : A.lt + tl;
  const LaneHang* lhp = A.order ? A.lh_lo + bx : A.lh + tl;
  const TileInfo ti = A.order ? A.tiles_lo[bx] : A.tiles[tl];
  const int nloc = ti.n_owned + ti.n_foreign;
  // tile DoF i at xd[i] (fp64 on arrival, then df in place; the zero region after it)
  const double* so = A.src + ti.dof_begin;
  const int sh = (int)((reinterpret_cast<uintptr_t>(so) >> 3) & 1);
  double* xd = xd0 + sh;
  df* xs = reinterpret_cast<df*>(xd);
  const int h0 = min(sh, ti.n_owned), nv = (ti.n_owned - h0) >> 1;
  {
    const uint4* g = reinterpret_cast<const uint4*>(ltp);
    uint4* s = reinterpret_cast<uint4*>(st);
    for (int i = threadIdx.x; i < (int)(sizeof(LaneTile) / 16); i += NT) cp_async16(s + i, g + i);
    if (!A.order || (int)blockIdx.x < A.n_hang) {  // the tile has hanging cells (or may have)
      const uint4* gh = reinterpret_cast<const uint4*>(lhp);
      uint4* shh = reinterpret_cast<uint4*>(hg);
      for (int i = threadIdx.x; i < (int)(sizeof(LaneHang) / 16); i += NT) cp_async16(shh + i, gh + i);
    }
    if (threadIdx.x < h0) cp_async(xd + threadIdx.x, so + threadIdx.x);
#pragma unroll 4
    for (int j = threadIdx.x; j < nv; j += NT) cp_async16(xd + h0 + 2 * j, so + h0 + 2 * j);
    for (int i = h0 + 2 * nv + threadIdx.x; i < ti.n_owned; i += NT) cp_async(xd + i, so + i);
    const int32_t* fl = A.foreign + ti.foreign_begin;
    double* xf = xd + ti.n_owned;
    for (int i0 = threadIdx.x; i0 < ti.n_foreign; i0 += 4 * NT) {
      int idx[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) idx[u] = (i0 + u * NT < ti.n_foreign) ? fl[i0 + u * NT] : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (idx[u] >= 0) cp_async(xf + i0 + u * NT, A.src + idx[u]);
    }
  }
  if (threadIdx.x < LANE_ZERO) xs[nloc + threadIdx.x] = df{0.f, 0.f};
  cp_async_wait_all();
  __syncthreads();
  for (int i = threadIdx.x; i < nloc; i += NT) xs[i] = df_from(xd[i]);  // one thread per element: in place
  const uint16_t m = st->mask[lane];
  const bool hang = st->hang != 0;
  df h;
  {
    const int c = ti.cell_begin + min(lane, ti.n_cells - 1);
    const double hd = ldexp(A.dom, -(int)st->level[lane]);
    h = df_from(A.coef ? hd * A.coef[c] : hd);
  }
  char* xb = reinterpret_cast<char*>(xs);
  const int nxl = c_ll.nx[K][w];
  __syncthreads();

  // G_e (+ C_x on hanging tiles, else the forward x sweep)
#pragma unroll 1
  for (int i = 0; i < nxl; ++i) {
    const int r = c_ll.xw[K][w][i];
    const uint32_t li = c_ll.line[K][r];
    const int s0 = li & 0xff, o0 = (li >> 8) & 0xff, o1 = li >> 16;
    const df* p0 = reinterpret_cast<const df*>(xb + 2 * (st->ls[s0][lane] + o0));
    const df* p1 = reinterpret_cast<const df*>(xb + 2 * (st->ls[s0 + 1][lane] + o1));
    const df* p2 = reinterpret_cast<const df*>(xb + 2 * (st->ls[s0 + 2][lane] + o0));
    df v[N];
    v[0] = *p0;
#pragma unroll
    for (int a = 1; a < K; ++a) v[a] = p1[a - 1];
    v[K] = *p2;
    if (!hang)
      df_eo_fwd_fast<K>(v);
    else if ((hg->hl[0][lane] >> r) & 1u)
      interp_line_df<K, false>(v, m & 1);
    df* p = cb + N * r * 32 + lane;
#pragma unroll
    for (int a = 0; a < N; ++a) p[a * 32] = v[a];
  }
  __syncthreads();
  if (hang) {
    hang_pass_df<K, 1, false>(cb, m, hg->hl[1][lane], w, lane);  // C_y
    __syncthreads();
    hang_pass_df<K, 2, false, true>(cb, m, hg->hl[2][lane], w, lane);  // C_z, forward z sweep
    __syncthreads();
  }
  {  // the tile DoFs are dead: clear the accumulator
    float4* z4 = reinterpret_cast<float4*>(xd0);
    for (int i = threadIdx.x; i < (sh + nloc + 1) / 2; i += NT) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  sweep_y_df<K, true>(cb, w, lane);
  __syncthreads();
  if (!hang)
    sweep_scale_df<K, 2>(cb, w, lane, h);
  else
    sweep_scale_df<K, 0>(cb, w, lane, h);
  __syncthreads();
  sweep_y_df<K, false>(cb, w, lane);
  __syncthreads();
  if (hang) {
    hang_pass_df<K, 2, true, true>(cb, m, hg->hl[2][lane], w, lane);  // backward z sweep, C_z^T
    __syncthreads();
    hang_pass_df<K, 1, true>(cb, m, hg->hl[1][lane], w, lane);  // C_y^T
    __syncthreads();
  }
  // backward x sweep (tiles without hanging cells) or C_x^T, then G_e^T on the warp's class of x-lines
  const uint32_t hs = hang ? hg->hs[lane] : 0u;
  const int zb = nloc * 4;
#pragma unroll 1
  for (int i = 0; i < nxl; ++i) {
    const int r = c_ll.xw[K][w][i];
    const df* p = cb + N * r * 32 + lane;
    df v[N];
#pragma unroll
    for (int a = 0; a < N; ++a) v[a] = p[a * 32];
    if (!hang)
      df_eo_bwd_fast<K>(v);
    else if ((hg->hl[0][lane] >> r) & 1u)
      interp_line_df<K, true>(v, m & 1);
    const uint32_t li = c_ll.line[K][r];
    const int s0 = li & 0xff, o0 = (li >> 8) & 0xff, o1 = li >> 16;
    const int b0 = st->ls[s0][lane], b1 = st->ls[s0 + 1][lane], b2 = st->ls[s0 + 2][lane];
    df* q0 = reinterpret_cast<df*>(xb + 2 * (b0 + o0));
    df* q1 = reinterpret_cast<df*>(xb + 2 * (b1 + o1));
    df* q2 = reinterpret_cast<df*>(xb + 2 * (b2 + o0));
    if (!hang) {
      *q0 = df_add(*q0, v[0]);
#pragma unroll
      for (int a = 1; a < K; ++a) q1[a - 1] = df_add(q1[a - 1], v[a]);
      *q2 = df_add(*q2, v[K]);
    } else {
      const bool g0 = __any_sync(0xffffffffu, (hs >> s0) & 1u), g1 = __any_sync(0xffffffffu, (hs >> (s0 + 1)) & 1u),
                 g2 = __any_sync(0xffffffffu, (hs >> (s0 + 2)) & 1u);
      add_ordered_df(q0, v[0], b0 != zb, lane, g0);
#pragma unroll
      for (int a = 1; a < K; ++a) add_ordered_df(q1 + a - 1, v[a], b1 != zb, lane, g1);
      add_ordered_df(q2, v[K], b2 != zb, lane, g2);
    }
  }
  __syncthreads();
  double* d = A.dst + ti.dof_begin;
  if (A.add)
    for (int i = threadIdx.x; i < ti.n_owned; i += NT) d[i] += df_to(xs[i]);
  else
    for (int i = threadIdx.x; i < ti.n_owned; i += NT) d[i] = df_to(xs[i]);
  const int32_t* hp = A.halo_pos + ti.foreign_begin;
  for (int i = threadIdx.x; i < ti.n_foreign; i += NT) A.halo[hp[i]] = df_to(xs[ti.n_owned + i]);
}

// host: entity slot and offset of local node (a, b, c) of a degree-k cell
// (the numbering of the level set-up: slot cx + 3 cy + 9 cz, DoFs of an
// entity lexicographic over its interior axes)
void host_node_slot(int k, int a, int b, int c, int& slot, int& off) {
  const int ca = a == 0 ? 0 : (a == k ? 2 : 1), cbb = b == 0 ? 0 : (b == k ? 2 : 1),
            cc = c == 0 ? 0 : (c == k ? 2 : 1);
  slot = ca + 3 * cbb + 9 * cc;
  int o = 0, mul = 1;
  if (ca == 1) {
    o += a - 1;
    mul *= k - 1;
  }
  if (cbb == 1) {
    o += (b - 1) * mul;
    mul *= k - 1;
  }
  if (cc == 1) o += (c - 1) * mul;
  off = o;
}

// x-line tables: slots and offsets per line; the line classes (lines whose
// nodes can share DoFs between cells) dealt to the k+1 warps, largest class
// first to the least loaded warp
void fill_lane_lines(LaneLines& t) {
  t = LaneLines{};
  for (int k = 0; k <= KMAX; ++k)
    for (int w = 0; w < NMAX; ++w)
      for (int i = 0; i < LW; ++i) t.xw[k][w][i] = -1;
  for (int k = 1; k <= KMAX; ++k) {
    const int n = k + 1;
    for (int c = 0; c < n; ++c)
      for (int b = 0; b < n; ++b) {
        int s0, o0, s1, o1 = 0;
        host_node_slot(k, 0, b, c, s0, o0);
        if (k > 1) host_node_slot(k, 1, b, c, s1, o1);
        t.line[k][b + n * c] = (uint32_t)s0 | ((uint32_t)(4 * o0) << 8) | ((uint32_t)(4 * o1) << 16);
      }
    auto cls = [&](int x) { return (x == 0 || x == k) ? -1 : x; };
    std::map<std::pair<int, int>, std::vector<int>> classes;
    for (int c = 0; c < n; ++c)
      for (int b = 0; b < n; ++b) classes[{cls(b), cls(c)}].push_back(b + n * c);
    std::vector<std::vector<int>> cl;
    for (auto& kv : classes) cl.push_back(kv.second);
    std::stable_sort(cl.begin(), cl.end(), [](const std::vector<int>& x, const std::vector<int>& y) {
      return x.size() > y.size();
    });
    std::vector<int> load(n, 0);
    for (const auto& c : cl) {
      int w = 0;
      for (int u = 1; u < n; ++u)
        if (load[u] < load[w]) w = u;
      for (int r : c) {
        if (load[w] >= LW) throw std::runtime_error("lane line table overflow");
        t.xw[k][w][load[w]++] = (int8_t)r;
      }
    }
    for (int w = 0; w < n; ++w) t.nx[k][w] = load[w];
  }
}

template <int K>
size_t lanes_smem(int max_local) {
  constexpr int N3 = (K + 1) * (K + 1) * (K + 1);
  // one region for the cell buffer and the tile DoFs (shifted by up to 3 for the 16-byte
  // copies, the zero region, and the float4 clearing)
  return sizeof(LaneTile) + sizeof(LaneHang) +
         std::max((size_t)N3 * 32, (size_t)max_local + LANE_ZERO + 8) * sizeof(float);
}

template <int K>
size_t lanes_df_smem(int max_local) {
  constexpr int N3 = (K + 1) * (K + 1) * (K + 1);
  return sizeof(LaneTile) + sizeof(LaneHang) + ((size_t)N3 * 32 + (size_t)max_local + LANE_ZERO + 4) * sizeof(double);
}

template <int K>
cudaError_t run_lanes_df(const CellLaunch& L, const LaneArgsT<double>& A, int n_tiles, cudaStream_t s) {
  const size_t sm = lanes_df_smem<K>(L.max_local);
  cudaError_t e = smem_allow(vmult_lanes_df<K>, sm);
  if (e != cudaSuccess) return e;
  e = launch_pdl(vmult_lanes_df<K>, n_tiles, (K + 1) * 32, sm, s, A);
  note_launches(1);
  return e;
}

template <int K>
cudaError_t run_lanes(const CellLaunch& L, const LaneArgs& A, int n_tiles, cudaStream_t s) {
  const size_t sm = lanes_smem<K>(L.max_local);
  cudaError_t e = smem_allow(vmult_lanes<K>, sm);
  if (e != cudaSuccess) return e;
  e = launch_pdl(vmult_lanes<K>, n_tiles, (K + 1) * 32, sm, s, A);
  note_launches(1);
  return e;
}

}  // namespace

void upload_tables_lanes() {
  upload_tables_lanes_1d();
  static LaneLines t;
  fill_lane_lines(t);
  cudaMemcpyToSymbol(c_ll, &t, sizeof(t));
}

bool lanes_ok(const CellLaunch& L) { return L.lane_tiles && L.tc <= 32 && !L.geom && L.k >= 1 && L.k <= KMAX; }

void launch_vmult_lanes_df(const CellLaunch& L, const double* src, double* dst, int add, int t0, int t1,
                           cudaStream_t s) {
  if (t1 <= t0 || !lanes_ok(L)) return;
  LaneArgsT<double> A{};
  A.tiles = L.tiles;
  A.lt = static_cast<const LaneTile*>(L.lane_tiles);
  A.lh = static_cast<const LaneHang*>(L.lane_hang);
  A.n_hang = L.n_hang_tiles;
  A.order = (t0 == 0 && t1 == L.n_tiles) ? L.lane_order : nullptr;
  A.tiles_lo = L.tiles_lo;
  A.lt_lo = static_cast<const LaneTile*>(L.lane_tiles_lo);
  A.lh_lo = static_cast<const LaneHang*>(L.lane_hang_lo);
  A.foreign = L.foreign;
  A.halo_pos = L.halo_pos;
  A.src = src;
  A.dst = dst;
  A.halo = static_cast<double*>(L.halo);
  A.coef = L.coef;
  A.dom = L.dom;
  A.add = add;
  A.tile0 = t0;
  switch (L.k) {
    case 1: run_lanes_df<1>(L, A, t1 - t0, s); break;
    case 2: run_lanes_df<2>(L, A, t1 - t0, s); break;
    case 3: run_lanes_df<3>(L, A, t1 - t0, s); break;
    case 4: run_lanes_df<4>(L, A, t1 - t0, s); break;
    default: break;
  }
}

void launch_vmult_lanes(const CellLaunch& L, const void* src, void* dst, int add, int t0, int t1, cudaStream_t s) {
  if (t1 <= t0 || !lanes_ok(L)) return;
  LaneArgs A{};
  A.tiles = L.tiles;
  A.lt = static_cast<const LaneTile*>(L.lane_tiles);
  A.lh = static_cast<const LaneHang*>(L.lane_hang);
  A.n_hang = L.n_hang_tiles;
  // a whole level: tiles with hanging cells first (their longer code path then
  // runs mostly on its own instead of interleaved with the regular tiles')
  A.order = (t0 == 0 && t1 == L.n_tiles) ? L.lane_order : nullptr;
  A.tiles_lo = L.tiles_lo;
  A.lt_lo = static_cast<const LaneTile*>(L.lane_tiles_lo);
  A.lh_lo = static_cast<const LaneHang*>(L.lane_hang_lo);
  A.foreign = L.foreign;
  A.halo_pos = L.halo_pos;
  A.src = static_cast<const float*>(src);
  A.dst = static_cast<float*>(dst);
  A.halo = static_cast<float*>(L.halo);
  A.coef = L.coef;
  A.dom = L.dom;
  A.add = add;
  A.tile0 = t0;
  switch (L.k) {
    case 1: run_lanes<1>(L, A, t1 - t0, s); break;
    case 2: run_lanes<2>(L, A, t1 - t0, s); break;
    case 3: run_lanes<3>(L, A, t1 - t0, s); break;
    case 4: run_lanes<4>(L, A, t1 - t0, s); break;
    default: break;
  }
}

}  // namespace gcmg
