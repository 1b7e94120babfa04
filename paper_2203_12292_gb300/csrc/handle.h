// Internal state of a libgcmg handle (levels, transfers, timers, graphs)
// and the orchestration steps shared by the C ABI translation units.
#pragma once

#include <memory>
#include <vector>

#include "gcmg.h"
#include "host.h"
#include "internal.h"
#include "kernels.h"
#include "mlp_net.h"

namespace gcmg {

struct LevelDev {
  LevelHost host;
  bool fp32 = true;
  DevBuf tiles, meta, foreign, subptr, perm, cell_ijk, gstart, own, mask, lane_tiles, lane_order, lane_hang, tiles_lo,
      lane_tiles_lo, lane_hang_lo;
  DevBuf halo, halo_dofs, halo_ptr, halo_src, halo_pos;
  DevBuf diag64, dinv64, dinv32;
  DevBuf x, b, d, t;        // V-cycle vectors in level precision
  DevBuf w64a, w64b, w64c;  // fp64 work vectors (set-up, fp64 smoothing through the API)
  DevBuf w32a, w32b;        // fp32 work vectors (fp32 smoothing through the API)
  CellLaunch cl{};
  double lam = 1.0;
  // learned smoother: kind, parameter copy, bf16 diagonal features per cell
  int smoother = GCMG_SMOOTHER_CHEBYSHEV;
  DevBuf mlp_image, dfeat;  // packed bf16 weights of the fused kernel, bf16 diagonal features
  DevBuf mlp_dproj;         // diagonal part of the first layer per cell (the smoother's network)
  DevBuf mlp_image_call, mlp_dproj_call;  // the same for gcmg_mlp_correct calls
  uint64_t mlp_call_version = 0;          // network version they were built from
  DevBuf coef;              // per cell coefficient nu_e (allocated once one is set)
  // local smoothing: refinement-edge DoFs; Algorithm 1's copy pairs (active DoF, level DoF)
  DevBuf edge_idx, cp_g, cp_idx;
  int64_t n_edge = 0, n_cp = 0;
  int64_t n() const { return host.n_free; }
};

struct TransferDev {
  TransferHost host;
  DevBuf fine_of, refined;
  TransferLaunch tl{};
};


// CUDA-event timers per (level, stage): the per-level, per-stage profile of
// a V-cycle (presmoothing, residual, restriction, coarse solve, prolongation,
// postsmoothing) plus operator applications and CG vector work.
struct Profiler {
  bool on = false;
  struct Rec {
    cudaEvent_t a = nullptr, b = nullptr;
    int level = 0, stage = 0;
  };
  std::vector<Rec> pool;
  size_t used = 0;
  std::vector<double> ms;
  std::vector<int64_t> cnt;
  int nlev = 0;
  ~Profiler() {
    for (auto& r : pool) {
      if (r.a) cudaEventDestroy(r.a);
      if (r.b) cudaEventDestroy(r.b);
    }
  }
};
constexpr int NSTAGE = 10;

// CUDA graphs of the V-cycle and of the operator half of a CG iteration;
// captured once per handle (re-captured when smoother parameters or the
// profiling state change).  Timers captured into a graph are event-record
// nodes, read after each replay.
struct GraphRec {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;  // kernel launches per replay
  std::vector<Profiler::Rec> recs;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (auto& r : recs) {
      if (r.a) cudaEventDestroy(r.a);
      if (r.b) cudaEventDestroy(r.b);
    }
    recs.clear();
  }
  ~GraphRec() { reset(); }
};

struct Handle {
  cudaStream_t stream = nullptr;
  int n_sm = 152;               // multiprocessors of the handle's device (set-up)
  bool stop_after_cgc = false;  // finest level: return after the prolongation
  bool ls = false;              // local smoothing: lev[0..top_mg] refinement levels, lev.back() the active mesh
  int top_mg = 0;               // finest multigrid level (lev.size() - 1 for global coarsening)
  bool in_batch = false;        // owned by a batch, whose graph holds the kernels' arguments
  cudaStream_t cap_stream = nullptr;
  bool use_graphs = true;
  GraphRec* capturing = nullptr;
  GraphRec g_core, g_a;
  Profiler prof;
  gcmg_config cfg{};
  std::vector<std::unique_ptr<LevelDev>> lev;
  std::vector<std::unique_ptr<TransferDev>> tr;  // tr[l]: between levels l and l-1
  DevBuf diag_tab[KMAX + 1];
  DevBuf Ainv;
  int n0 = 0;
  DevBuf scratch, scal, modes;
  DevBuf cg_r, cg_p, cg_q, cg_z, cg_x;
  DevBuf lscratch;     // inner products of the learned step's Galerkin step length
  // host-buffer operator: the input copy in DoF order on its own stream, overlapped with the tiles
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> pipe_ev;
  // operator on several host vectors: two device input and output buffers,
  // the output copies on a stream of their own, events per buffer pair
  cudaStream_t out_stream = nullptr;
  DevBuf many_in[2], many_out[2];
  cudaEvent_t many_ev[7] = {};  // in[2], comp[2], out[2], start
  ~Handle() {
    g_core.reset();
    g_a.reset();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (cudaEvent_t e : pipe_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : many_ev)
      if (e) cudaEventDestroy(e);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    if (out_stream) cudaStreamDestroy(out_stream);
  }
};

// set-up of all levels, transfers, diagonals, coarse factor and eigenvalue
// estimates of one problem (Sec. 5 set-up); throws Error
void setup_handle(Handle& H, const std::vector<Octree>& meshes, int lmax, const gcmg_config& cfg);
// the operator-dependent parts of the set-up: Jacobi diagonals, coarse
// inverse, Chebyshev eigenvalue estimates (after a change of coefficient)
void setup_numerics(Handle& H);
void upload_all_tables();
void check_config(const gcmg_config* cfg);
void check_level(const Handle& h, int level);
int prof_begin(Handle& H, int level, int stage);
void prof_end(Handle& H, int rec);
void vmult(Handle& H, int l, bool fp64, const void* src, void* dst, int stage = GCMG_STAGE_VMULT);
void vcycle_level(Handle& H, int l);
bool any_learned(const Handle& H);

}  // namespace gcmg

struct gcmg_mesh {
  std::vector<gcmg::Octree> levels;  // coarsest (one cell) first
  int lmax = 0;
};

struct gcmg_handle {
  gcmg::Handle h;
};
