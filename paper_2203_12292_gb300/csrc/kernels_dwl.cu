// Persistent kernel of the device work list: every problem of a batch runs its
// recorded launch sequence (CG prologue, the body of one CG iteration, the
// epilogue; dwl.h) inside one cooperative launch.
//
// The kernels of kernels_cell.cu, kernels_transfer.cu and kernels_vec.cu are
// compiled here once more as device functions (the host code of those files
// is left out), with blockIdx and gridDim read from shared variables that
// hold the virtual block of the current item.  Each CTA (BLOCK threads) runs
// whole items, so the bodies' block barriers hold as in a launch.
//
// Schedule, in lockstep: every active problem has a current operation; the
// items of all current operations are numbered problem by problem and CTA c
// runs items c, c + G, ... (G CTAs); a grid barrier follows; then every
// problem moves to its next operation (after the CG loop test: to the loop
// body again or to the epilogue).  Every CTA keeps the same copy of the
// problems' positions and advances it from the same data, so no further
// synchronisation is needed.  The grid barrier's waits are bounded: a wait
// that gives up records an error and the kernel returns; so does a schedule
// longer than its bound.
#include <cuda_runtime.h>

#include <utility>

#include "device.cuh"
#include "dwl.h"
#include "kernels.h"

namespace gcmg {
namespace dwl_virtual {
__shared__ uint3 vb;  // virtual blockIdx of the current item
__shared__ uint3 vg;  // virtual gridDim of the current operation
constexpr int POOL_BYTES = 8 * 8 * 27 * 4;
__shared__ __align__(16) unsigned char pool[POOL_BYTES];  // shared by the bodies (one runs at a time)
}  // namespace dwl_virtual
}  // namespace gcmg

#pragma push_macro("__global__")
#pragma push_macro("__launch_bounds__")
#undef __global__
// each body a function of its own (not inlined into one dispatcher), so that
// the registers are those of the largest body, not of all of them together
#define __global__ __device__ __noinline__
#undef __launch_bounds__
#define __launch_bounds__(...)
#define blockIdx (::gcmg::dwl_virtual::vb)
#define gridDim (::gcmg::dwl_virtual::vg)
// the data of one operation is written by earlier operations of the same
// launch: no read-only (non-coherent) loads
#define __ldg(p) (*(p))
#define __restrict__
#define GCMG_BODIES_ONLY
#define GCMG_DWL_POOL (::gcmg::dwl_virtual::pool)
#define GCMG_DWL_POOL_BYTES (::gcmg::dwl_virtual::POOL_BYTES)
#include "kernels_cell.cu"
#include "kernels_transfer.cu"
#include "kernels_vec.cu"
#undef GCMG_DWL_POOL_BYTES
#undef GCMG_DWL_POOL
#undef GCMG_BODIES_ONLY
#undef __restrict__
#undef __ldg
#undef gridDim
#undef blockIdx
#pragma pop_macro("__launch_bounds__")
#pragma pop_macro("__global__")

namespace gcmg {

GCMG_DEFINE_UPLOAD(upload_tables_dwl)

namespace {

template <typename... KArgs, size_t... I>
__device__ __forceinline__ void dwl_call(void (*fn)(KArgs...), const unsigned char* buf, std::index_sequence<I...>) {
  fn(*reinterpret_cast<const KArgs*>(buf + dwl_offset<KArgs...>(I))...);
}
template <typename... KArgs>
__device__ __forceinline__ void dwl_call(void (*fn)(KArgs...), const unsigned char* buf) {
  dwl_call(fn, buf, std::index_sequence_for<KArgs...>{});
}

// one item of a registered operation (ids in the order of the registries)
__device__ void dwl_run(const DwlOp& op) {
  int id = 0;
#define GCMG_DWL_CASE(fn)      \
  if (op.type == id++) {       \
    dwl_call(fn, op.args);     \
    return;                    \
  }
  GCMG_DWL_CELL(GCMG_DWL_CASE)
  GCMG_DWL_TRANSFER(GCMG_DWL_CASE)
  GCMG_DWL_VEC(GCMG_DWL_CASE)
  GCMG_DWL_VEC_SERIAL(GCMG_DWL_CASE)
#undef GCMG_DWL_CASE
}

// the CG loop test of cg_check_kernel, its flag kept per problem
__device__ void dwl_check(const DwlOp& op, int* go) {
  using H = cudaGraphConditionalHandle;
  double* scal = *reinterpret_cast<double* const*>(op.args + dwl_offset<H, double*, int, double>(1));
  const int maxit = *reinterpret_cast<const int*>(op.args + dwl_offset<H, double*, int, double>(2));
  const double rtol2 = *reinterpret_cast<const double*>(op.args + dwl_offset<H, double*, int, double>(3));
  const double it = scal[8] + 1.0;
  scal[8] = it;
  const double rr = scal[2], nb2 = scal[7], pq = scal[1];
  go[op.prob] = ((it < (double)maxit) && (rr > rtol2 * nb2) && (pq > 0.0)) ? 1 : 0;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// grid barrier (all CTAs resident: cooperative launch); false after a bounded wait
__device__ bool dwl_grid_sync(unsigned* bar, unsigned& gen, int* ok_sh, unsigned spin_limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = gen;
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], g + 1);
    }
    // every CTA, the last to arrive included, ends with an acquire load of the
    // generation, so that its later loads see what the other CTAs wrote
    unsigned it = 0;
    while (ld_acquire(&bar[1]) == g) {
      if (++it > spin_limit) {
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    gen = g + 1;
    *ok_sh = ok;
  }
  __syncthreads();
  return *ok_sh != 0;
}

__global__ void __launch_bounds__(BLOCK, 2) dwl_kernel(DwlParams P) {
  __shared__ int s_pc[DWL_MAX_PROBS];
  __shared__ int s_pref[DWL_MAX_PROBS + 1];
  __shared__ int s_wsum[BLOCK / 32];
  __shared__ int s_ok;
  const int np = P.np;
  for (int p = threadIdx.x; p < np; p += BLOCK) s_pc[p] = P.probs[p].pro < P.probs[p].end ? P.probs[p].pro : -1;
  unsigned gen = 0;
  for (long long step = 0; step < P.max_steps; ++step) {
    __syncthreads();
    // items of the current operations, numbered problem by problem (exclusive
    // scan; thread t holds problems per t .. per t + per - 1)
    {
      const int per = (np + BLOCK - 1) / BLOCK;  // <= DWL_MAX_PROBS / BLOCK
      int cnt[DWL_MAX_PROBS / BLOCK];
      int sum = 0;
#pragma unroll
      for (int j = 0; j < DWL_MAX_PROBS / BLOCK; ++j) {
        const int p = threadIdx.x * per + j;
        cnt[j] = (j < per && p < np && s_pc[p] >= 0) ? P.ops[s_pc[p]].items : 0;
        sum += cnt[j];
      }
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (lane == 31) s_wsum[warp] = incl;
      __syncthreads();
      int base = 0;
      for (int w = 0; w < warp; ++w) base += s_wsum[w];
      int run = base + incl - sum;
#pragma unroll
      for (int j = 0; j < DWL_MAX_PROBS / BLOCK; ++j) {
        const int p = threadIdx.x * per + j;
        if (j < per && p < np) s_pref[p] = run;
        run += cnt[j];
      }
      if (threadIdx.x == BLOCK - 1) s_pref[np] = run;
    }
    __syncthreads();
    const int total = s_pref[np];
    if (total == 0) {  // every problem finished (the same in every CTA)
      if (blockIdx.x == 0 && threadIdx.x == 0) P.status[1] = (int)step;
      return;
    }
    for (int g = blockIdx.x; g < total; g += gridDim.x) {
      int lo = 0, hi = np;  // the problem p with s_pref[p] <= g < s_pref[p + 1]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_pref[mid] <= g) lo = mid; else hi = mid;
      }
      const DwlOp& op = P.ops[s_pc[lo]];
      if (threadIdx.x == 0) {
        dwl_virtual::vb = make_uint3((unsigned)(g - s_pref[lo]), 0u, 0u);
        dwl_virtual::vg = make_uint3((unsigned)op.items, 1u, 1u);
      }
      __syncthreads();
      if (op.type == DWL_OP_CHECK) {
        if (threadIdx.x == 0) dwl_check(op, P.go);
      } else if (op.block < BLOCK) {
        if ((int)threadIdx.x < op.block) dwl_run(op);  // serial operations: no block barrier inside
      } else {
        dwl_run(op);
      }
      __syncthreads();  // the next item reuses the shared memory
    }
    if (step == 0 && (int)blockIdx.x == P.absent_cta) return;  // its peers' waits run out
    if (!dwl_grid_sync(P.bar, gen, &s_ok, P.spin_limit)) {
      if (threadIdx.x == 0) atomicExch(&P.status[0], 1);
      return;
    }
    for (int p = threadIdx.x; p < np; p += BLOCK) {
      int pc = s_pc[p];
      if (pc < 0) continue;
      const DwlProb& pr = P.probs[p];
      if (P.ops[pc].type == DWL_OP_CHECK)
        pc = P.go[p] ? pr.body : pr.epi;
      else
        ++pc;
      s_pc[p] = pc < pr.end ? pc : -1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&P.status[0], 2);
}

}  // namespace

int dwl_grid(size_t smem, int n_sm) {
  const cudaError_t e = smem_allow(dwl_kernel, smem);
  if (e != cudaSuccess) return -1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dwl_kernel, BLOCK, smem) != cudaSuccess || per_sm < 1)
    return -1;
  return per_sm * n_sm;
}

cudaError_t launch_dwl(const DwlParams& P, int grid, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(BLOCK);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, dwl_kernel, P);
  note_launch_error(e);
  if (e == cudaSuccess) note_launches(1);
  return e;
}

}  // namespace gcmg
