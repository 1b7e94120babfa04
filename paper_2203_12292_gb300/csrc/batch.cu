// Batches of independent Poisson problems solved by one CUDA-graph launch,
// and the autotuner of the operator's tile size and thread mapping per
// polynomial degree.  The paper solves one problem per run; batching many
// uneven problems on one GPU is an extension.
//
// Every problem keeps its own handle (levels, transfers, vectors).  One
// graph holds, for every problem, the CG prologue, a conditional WHILE node
// whose body is one CG iteration (V-cycle, beta, p update, operator, alpha,
// x/r update, convergence check), and an epilogue; the check kernel of each
// iteration sets the node's condition on the device, so the whole batch
// runs to convergence without a host round trip.  Problems are independent
// branches of the graph and run concurrently.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dwl.h"
#include "handle.h"

// the device work list of a batch: every problem's recorded prologue, CG
// iteration and epilogue, run by one persistent cooperative kernel
struct DwlState {
  gcmg::DevBuf ops, probs, go, ctl;  // ctl: barrier (2 unsigned) and status (2 int)
  int np = 0, grid = 0;
  size_t smem = 0;
  long long max_steps = 0, n_ops = 0;
  cudaGraphExec_t exec = nullptr;  // the launch captured in a graph (null: launched directly)
  int steps = 0;
  std::vector<const double*> key_b;
  std::vector<double*> key_x;
  double key_rtol = -1.0;
  int key_maxit = -1;
  ~DwlState() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

struct gcmg_batch {
  std::vector<std::unique_ptr<gcmg_handle>> probs;
  std::unique_ptr<DwlState> dwl;
  // test of the persistent kernel's bounded waits (gcmg_batch_persistent_wait_test)
  int absent_cta = -1;
  unsigned spin_limit = 1u << 25;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  // the graph is specific to its arguments
  std::vector<const double*> key_b;
  std::vector<double*> key_x;
  double key_rtol = -1.0;
  int key_maxit = -1;
  gcmg::DevBuf stats;  // per problem: iterations, rr, |b|^2, status
  std::vector<long long> pro_kernels, body_kernels;
  ~gcmg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace gcmg {

long long launch_counter();

DwlRecorder*& dwl_recorder() {
  thread_local DwlRecorder* r = nullptr;
  return r;
}

namespace {
struct DwlEntry {
  int id;
  size_t bytes;
  int coarsen;
  bool serial;
};
std::mutex g_dwl_mu;
std::unordered_map<const void*, DwlEntry> g_dwl_reg;
}  // namespace

void dwl_register(const void* kernel, int id, size_t arg_bytes) {
  std::lock_guard<std::mutex> lock(g_dwl_mu);
  g_dwl_reg[kernel] = DwlEntry{id, arg_bytes, 1, false};
}

void dwl_set_coarsen(const void* kernel, int factor) {
  std::lock_guard<std::mutex> lock(g_dwl_mu);
  const auto it = g_dwl_reg.find(kernel);
  if (it != g_dwl_reg.end() && factor >= 1) it->second.coarsen = factor;
}

void dwl_set_serial(const void* kernel) {
  std::lock_guard<std::mutex> lock(g_dwl_mu);
  const auto it = g_dwl_reg.find(kernel);
  if (it != g_dwl_reg.end()) it->second.serial = true;
}

int dwl_lookup(const void* kernel, size_t* bytes, int* coarsen, bool* serial) {
  std::lock_guard<std::mutex> lock(g_dwl_mu);
  const auto it = g_dwl_reg.find(kernel);
  if (it == g_dwl_reg.end()) return -1;
  *bytes = it->second.bytes;
  *coarsen = it->second.coarsen;
  *serial = it->second.serial;
  return it->second.id;
}

void dwl_register_all() {
  static std::once_flag once;
  std::call_once(once, [] {
    dwl_register_cell();
    dwl_register_transfer();
    dwl_register_vec();
  });
}

namespace {

struct CgVecs {
  int64_t n;
  double *x, *r, *p, *q, *z, *S, *scratch;
};

CgVecs vecs(Handle& H) {
  const int top = (int)H.lev.size() - 1;
  return CgVecs{H.lev[top]->n(),        H.cg_x.as<double>(), H.cg_r.as<double>(), H.cg_p.as<double>(),
                H.cg_q.as<double>(),    H.cg_z.as<double>(), H.scal.as<double>(), H.scratch.as<double>()};
}

// V-cycle of Algorithms 1-2 as plain kernel launches (captured by the caller)
void vcycle_kernels(Handle& H, const double* b, double* x) {
  const int top = (int)H.lev.size() - 1;
  LevelDev& F = *H.lev[top];
  if (F.fp32)
    launch_cast(false, b, F.b.p, F.n(), H.stream);
  else
    launch_copy(b, F.b.as<double>(), F.n(), H.stream);
  vcycle_level(H, top);
  if (F.fp32)
    launch_cast(true, F.x.p, x, F.n(), H.stream);
  else
    launch_copy(F.x.as<double>(), x, F.n(), H.stream);
}

// q = A p, alpha = rz / pq, x += alpha p, r -= alpha q, rr
void op_half(Handle& H, const CgVecs& v) {
  vmult(H, (int)H.lev.size() - 1, true, v.p, v.q, GCMG_STAGE_CG_VMULT);
  launch_dot(v.p, v.q, v.n, v.scratch, v.S, 0, DOT_ALPHA, H.stream);
  launch_cg_update_xr(v.x, v.r, v.p, v.q, v.S, v.n, v.scratch, v.S, H.stream);
}

void cg_prologue(Handle& H, const double* b, double rtol2, int maxit, cudaGraphConditionalHandle hc) {
  const CgVecs v = vecs(H);
  launch_zero(true, v.x, v.n, H.stream);
  launch_copy(b, v.r, v.n, H.stream);
  launch_dot(v.r, v.r, v.n, v.scratch, v.S, 7, DOT_STORE, H.stream);
  launch_scalar_set(v.S, 8, 0.0, H.stream);
  vcycle_kernels(H, v.r, v.z);
  launch_dot(v.r, v.z, v.n, v.scratch, v.S, 0, DOT_STORE, H.stream);
  launch_copy(v.z, v.p, v.n, H.stream);
  op_half(H, v);
  launch_cg_check(hc, v.S, maxit, rtol2, H.stream);
}

void cg_body(Handle& H, double rtol2, int maxit, cudaGraphConditionalHandle hc) {
  const CgVecs v = vecs(H);
  const bool flexible = any_learned(H);
  if (flexible) launch_dot(v.r, v.z, v.n, v.scratch, v.S, 6, DOT_STORE, H.stream);
  vcycle_kernels(H, v.r, v.z);
  launch_dot(v.r, v.z, v.n, v.scratch, v.S, 0, flexible ? DOT_BETA_FLEX : DOT_BETA, H.stream);
  launch_cg_update_p(v.p, v.z, v.S, v.n, H.stream);
  op_half(H, v);
  launch_cg_check(hc, v.S, maxit, rtol2, H.stream);
}

// capture of launches on stream cs; returns the number of kernels recorded
template <typename F>
long long record(Handle& H, cudaStream_t cs, F&& body) {
  cudaStream_t saved = H.stream;
  const bool prof = H.prof.on;
  H.stream = cs;
  H.prof.on = false;  // event nodes are not allowed inside conditional bodies
  const long long before = launch_counter();
  try {
    body();
  } catch (...) {
    H.stream = saved;
    H.prof.on = prof;
    throw;
  }
  H.stream = saved;
  H.prof.on = prof;
  const long long k = launch_counter() - before;
  note_launches((int)-k);  // recorded, not run
  return k;
}

void build_graph(gcmg_batch& B, const double* const* b, double* const* x, double rtol, int maxit) {
  if (B.exec) cudaGraphExecDestroy(B.exec);
  B.exec = nullptr;
  const int np = (int)B.probs.size();
  const double rtol2 = rtol * rtol;
  cudaStream_t cs = B.cap;
  cudaGraph_t G = nullptr;
  ck(cudaGraphCreate(&G, 0), "graph create");
  B.pro_kernels.assign(np, 0);
  B.body_kernels.assign(np, 0);
  double* stats = B.stats.as<double>();
  try {
    for (int i = 0; i < np; ++i) {
      Handle& H = B.probs[i]->h;
      const CgVecs v = vecs(H);
      cudaGraph_t body = nullptr;
      cudaGraphConditionalHandle hc = 0;
      ck(cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "capture");
      if (v.n == 0) {
        B.pro_kernels[i] = record(H, cs, [&] {
          launch_scalar_set(v.S, 7, 0.0, cs);
          launch_scalar_set(v.S, 8, 0.0, cs);
          launch_cg_stats(v.S, rtol2, stats + 4 * i, cs);
        });
      } else {
        ck(cudaGraphConditionalHandleCreate(&hc, G, 0, 0), "conditional handle");
        B.pro_kernels[i] = record(H, cs, [&] { cg_prologue(H, b[i], rtol2, maxit, hc); });
        // the WHILE node after the prologue, then the epilogue after it
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* edges = nullptr;
        size_t nd = 0;
        ck(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, &edges, &nd), "capture info");
        cudaGraphNodeParams prm = {};
        prm.type = cudaGraphNodeTypeConditional;
        prm.conditional.handle = hc;
        prm.conditional.type = cudaGraphCondTypeWhile;
        prm.conditional.size = 1;
        cudaGraphNode_t wn;
        ck(cudaGraphAddNode(&wn, G, deps, edges, nd, &prm), "while node");
        body = prm.conditional.phGraph_out[0];
        ck(cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1, cudaStreamSetCaptureDependencies),
           "capture dependencies");
        B.pro_kernels[i] += record(H, cs, [&] {
          launch_copy(v.x, x[i], v.n, cs);
          launch_cg_stats(v.S, rtol2, stats + 4 * i, cs);
        });
      }
      cudaGraph_t g_out = nullptr;
      ck(cudaStreamEndCapture(cs, &g_out), "end capture");
      if (body) {
        ck(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "capture");
        B.body_kernels[i] = record(H, cs, [&] { cg_body(H, rtol2, maxit, hc); });
        ck(cudaStreamEndCapture(cs, &g_out), "end capture");
      }
    }
  } catch (...) {
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(cs, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(cs, &g);
    }
    cudaGraphDestroy(G);
    throw;
  }
  const cudaError_t e = cudaGraphInstantiate(&B.exec, G, 0);
  cudaGraphDestroy(G);
  ck(e, "graph instantiate");
}

// ---------------------------------------------------------------------------
// device work list
// ---------------------------------------------------------------------------

// the launches of f recorded (not run) as device-work-list operations
template <typename F>
std::vector<DwlOp> record_ops(Handle& H, F&& f) {
  DwlRecorder rec;
  const bool prof = H.prof.on;
  H.prof.on = false;
  const long long before = launch_counter();
  g_launch_err = cudaSuccess;
  dwl_recorder() = &rec;
  try {
    f();
  } catch (...) {
    dwl_recorder() = nullptr;
    H.prof.on = prof;
    note_launches((int)-(launch_counter() - before));
    throw;
  }
  dwl_recorder() = nullptr;
  H.prof.on = prof;
  note_launches((int)-(launch_counter() - before));  // recorded, not run
  if (g_launch_err != cudaSuccess) {
    g_launch_err = cudaSuccess;
    throw Error(GCMG_ERR_ARG, "the persistent batch runs the line-parallel operators and the kernels of the "
                              "plain V-cycle and CG only (a launch of this problem has no device-work-list form)");
  }
  return std::move(rec.ops);
}

void build_dwl(gcmg_batch& B, const double* const* b, double* const* x, double rtol, int maxit) {
  const int np = (int)B.probs.size();
  if (np > DWL_MAX_PROBS) throw Error(GCMG_ERR_ARG, "the persistent batch takes at most 1024 problems");
  dwl_register_all();
  const double rtol2 = rtol * rtol;
  std::vector<DwlOp> all;
  std::vector<DwlProb> pr(np);
  long long longest = 0;
  auto append = [&](std::vector<DwlOp>&& v, int prob) {
    for (auto& op : v) {
      if (op.type == DWL_OP_CHECK) op.prob = prob;
      all.push_back(op);
    }
  };
  for (int i = 0; i < np; ++i) {
    Handle& H = B.probs[i]->h;
    const CgVecs v = vecs(H);
    DwlProb q{};
    q.pro = (int32_t)all.size();
    if (v.n == 0) {
      append(record_ops(H, [&] {
               launch_scalar_set(v.S, 7, 0.0, H.stream);
               launch_scalar_set(v.S, 8, 0.0, H.stream);
               launch_cg_stats(v.S, rtol2, B.stats.as<double>() + 4 * i, H.stream);
             }),
             i);
      q.body = q.epi = q.end = (int32_t)all.size();
    } else {
      append(record_ops(H, [&] { cg_prologue(H, b[i], rtol2, maxit, 0); }), i);
      q.body = (int32_t)all.size();
      append(record_ops(H, [&] { cg_body(H, rtol2, maxit, 0); }), i);
      q.epi = (int32_t)all.size();
      append(record_ops(H, [&] {
               launch_copy(v.x, x[i], v.n, H.stream);
               launch_cg_stats(v.S, rtol2, B.stats.as<double>() + 4 * i, H.stream);
             }),
             i);
      q.end = (int32_t)all.size();
      if (q.body == q.pro || all[q.body - 1].type != DWL_OP_CHECK || q.epi == q.body ||
          all[q.epi - 1].type != DWL_OP_CHECK)
        throw Error(GCMG_ERR_INTERNAL, "recorded CG without its loop test");
    }
    pr[i] = q;
    longest = std::max(longest, (long long)(q.body - q.pro) + (long long)maxit * (q.epi - q.body) + (q.end - q.epi));
  }
  auto D = std::make_unique<DwlState>();
  D->np = np;
  D->n_ops = (long long)all.size();
  D->max_steps = longest + 8;
  for (const auto& op : all) D->smem = std::max(D->smem, (size_t)op.smem);
  D->grid = dwl_grid(D->smem, B.probs.empty() ? 152 : B.probs[0]->h.n_sm);
  if (D->grid < 1) throw Error(GCMG_ERR_CUDA, "the persistent batch kernel does not fit on this device");
  D->ops.upload(all, B.stream);
  D->probs.upload(pr, B.stream);
  D->go.alloc((size_t)std::max(np, 1) * sizeof(int));
  D->ctl.alloc(4 * sizeof(unsigned));
  ck(cudaStreamSynchronize(B.stream), "upload");
  // one launch of the persistent kernel, captured in a graph with the reset of its barrier
  DwlParams P{D->ops.as<DwlOp>(), D->probs.as<DwlProb>(), np, D->go.as<int>(), D->ctl.as<unsigned>(),
              D->ctl.as<int>() + 2, D->max_steps, B.spin_limit, B.absent_cta};
  cudaGraph_t G = nullptr;
  ck(cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeRelaxed), "capture");
  cudaError_t e = cudaMemsetAsync(D->ctl.p, 0, 4 * sizeof(unsigned), B.cap);
  if (e == cudaSuccess) e = launch_dwl(P, D->grid, D->smem, B.cap);
  const cudaError_t e2 = cudaStreamEndCapture(B.cap, &G);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&D->exec, G, 0);
  if (G) cudaGraphDestroy(G);
  g_launch_err = cudaSuccess;
  note_launches(-1);  // captured, not run
  ck(e, "persistent batch graph");
  D->key_b.assign(b, b + np);
  D->key_x.assign(x, x + np);
  D->key_rtol = rtol;
  D->key_maxit = maxit;
  B.dwl = std::move(D);
}

// fp32 (or fp64) operator of the finest level: GDoF/s over `reps` applications
double time_vmult(Handle& H, bool fp64, int reps) {
  const int top = (int)H.lev.size() - 1;
  LevelDev& F = *H.lev[top];
  const int64_t n = F.n();
  if (n == 0) return 0.0;
  DevBuf x, y;
  x.alloc(n * (fp64 ? 8 : 4));
  y.alloc(n * (fp64 ? 8 : 4));
  ck(cudaMemsetAsync(x.p, 0, x.bytes, H.stream), "memset");
  for (int i = 0; i < 3; ++i) vmult(H, top, fp64, x.p, y.p);
  cudaEvent_t a, b;
  ck(cudaEventCreate(&a), "event");
  ck(cudaEventCreate(&b), "event");
  ck(cudaEventRecord(a, H.stream), "event");
  for (int i = 0; i < reps; ++i) vmult(H, top, fp64, x.p, y.p);
  ck(cudaEventRecord(b, H.stream), "event");
  ck(cudaEventSynchronize(b), "event");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (double)n * reps / (ms * 1e6);
}

}  // namespace
}  // namespace gcmg

using namespace gcmg;

extern "C" {

int gcmg_autotune(const gcmg_mesh* probe, int degree, int mg_fp32, int reps, void* stream, gcmg_tuning* best,
                  gcmg_tuning* all, int* n_all) {
  return guarded([&] {
    if (!probe || !best || degree < 1 || degree > KMAX || reps < 1) throw Error(GCMG_ERR_ARG, "bad arguments");
    upload_all_tables();
    // candidates (tile cells, kernel, threads): the default (one lane per cell on 32-cell tiles), one lane
    // per cell on 8/16-cell tiles, one thread per line on 8..128-cell tiles (lines per thread follow
    // from the tile size; 256 or 512 threads for the chunked kernel of tiles above 32 cells), slab
    // threads on 16..64-cell tiles (fp32 only).  The probe's finest level must keep every size
    // (at least 2 x SMs x 128 cells).
    // (one lane per cell on 32-cell tiles is the default's finest-level kernel; forcing it onto the
    // coarse levels' smaller tiles as well is slower there, which this probe does not time)
    static const int c32[][3] = {{32, 0, 0},   {8, 3, 0},   {16, 3, 0},   {8, 1, 0},     {16, 1, 0},
                                 {32, 1, 0},   {64, 1, 256}, {64, 1, 512}, {128, 1, 256}, {128, 1, 512},
                                 {16, 2, 0},   {32, 2, 0},   {64, 2, 0}};
    static const int c64[][3] = {{32, 0, 0}, {8, 1, 0}, {16, 1, 0}, {32, 1, 0}, {64, 1, 0}, {128, 1, 0}};
    const int nc = mg_fp32 ? (int)(sizeof(c32) / sizeof(c32[0])) : (int)(sizeof(c64) / sizeof(c64[0]));
    static_assert(sizeof(c32) / sizeof(c32[0]) <= GCMG_AUTOTUNE_MAX, "candidate list");
    const int (*list)[3] = mg_fp32 ? c32 : c64;
    gcmg_tuning top{degree, 0, 0, 0, -1.0};
    for (int c = 0; c < nc; ++c) {
      gcmg_config cfg;
      gcmg_config_default(&cfg);
      cfg.degree = degree;
      cfg.mg_fp32 = mg_fp32;
      cfg.tile_cells = list[c][0];
      cfg.cell_kernel = list[c][1];
      cfg.cell_threads = list[c][2];
      Handle H;
      H.stream = static_cast<cudaStream_t>(stream);
      setup_handle(H, probe->levels, probe->lmax, cfg);
      const gcmg_tuning t{degree, cfg.tile_cells, cfg.cell_kernel, cfg.cell_threads, time_vmult(H, mg_fp32 == 0, reps)};
      if (all) all[c] = t;
      if (t.gdofs > top.gdofs) top = t;
    }
    if (n_all) *n_all = nc;
    *best = top;
  });
}

int gcmg_batch_create(int n, const gcmg_mesh* const* meshes, const gcmg_config* cfgs, int n_threads, void* stream,
                      gcmg_batch** out) {
  return guarded([&] {
    if (n <= 0 || !meshes || !cfgs || !out) throw Error(GCMG_ERR_ARG, "bad arguments");
    for (int i = 0; i < n; ++i) {
      if (!meshes[i]) throw Error(GCMG_ERR_ARG, "null mesh");
      check_config(&cfgs[i]);
      if (cfgs[i].local_smoothing) throw Error(GCMG_ERR_ARG, "the batch runs global coarsening only");
    }
    upload_all_tables();
    int dev = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    auto B = std::make_unique<gcmg_batch>();
    B->stream = static_cast<cudaStream_t>(stream);
    B->probs.resize(n);
    const int nt = std::max(1, std::min(n_threads > 0 ? n_threads : 16, n));
    std::atomic<int> next{0};
    std::vector<int> codes(nt, GCMG_OK);
    std::vector<std::string> msgs(nt);
    // host set-up of the problems in parallel; every worker queues its device
    // work on a stream of its own
    auto worker = [&](int t) {
      cudaStream_t s = nullptr;
      try {
        ck(cudaSetDevice(dev), "cudaSetDevice");
        ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
        for (int i; (i = next.fetch_add(1)) < n;) {
          auto h = std::make_unique<gcmg_handle>();
          h->h.stream = s;
          h->h.in_batch = true;
          setup_handle(h->h, meshes[i]->levels, meshes[i]->lmax, cfgs[i]);
          B->probs[i] = std::move(h);
        }
        ck(cudaStreamSynchronize(s), "setup");
      } catch (const Error& e) {
        codes[t] = e.code;
        msgs[t] = e.what();
        next.store(n);
      } catch (const std::exception& e) {
        codes[t] = GCMG_ERR_INTERNAL;
        msgs[t] = e.what();
        next.store(n);
      }
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(worker, t);
    worker(0);
    for (auto& t : th) t.join();
    for (int t = 0; t < nt; ++t)
      if (codes[t] != GCMG_OK) throw Error(codes[t], msgs[t]);
    for (auto& h : B->probs) h->h.stream = B->stream;
    ck(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking), "stream");
    B->stats.alloc((size_t)n * 4 * sizeof(double));
    *out = B.release();
  });
}

void gcmg_batch_destroy(gcmg_batch* b) { delete b; }

int gcmg_batch_size(const gcmg_batch* b, int* n) {
  return guarded([&] {
    if (!b || !n) throw Error(GCMG_ERR_ARG, "null argument");
    *n = (int)b->probs.size();
  });
}

int gcmg_batch_handle(gcmg_batch* b, int i, gcmg_handle** h) {
  return guarded([&] {
    if (!b || !h || i < 0 || i >= (int)b->probs.size()) throw Error(GCMG_ERR_ARG, "bad arguments");
    *h = b->probs[i].get();
  });
}

int gcmg_batch_cg_solve(gcmg_batch* b, const double* const* rhs, double* const* x, double rtol, int maxit,
                        gcmg_solve_stats* stats) {
  return guarded([&] {
    if (!b || !rhs || !x || !(rtol > 0) || maxit < 1) throw Error(GCMG_ERR_ARG, "bad arguments");
    const int np = (int)b->probs.size();
    for (int i = 0; i < np; ++i) {
      if (b->probs[i]->h.lev.back()->n() && (!rhs[i] || !x[i])) throw Error(GCMG_ERR_ARG, "bad vectors");
      b->probs[i]->h.stream = b->stream;
    }
    const bool same = b->exec && b->key_rtol == rtol && b->key_maxit == maxit &&
                      std::equal(b->key_b.begin(), b->key_b.end(), rhs) && std::equal(b->key_x.begin(), b->key_x.end(), x);
    if (!same) {
      build_graph(*b, rhs, x, rtol, maxit);
      b->key_b.assign(rhs, rhs + np);
      b->key_x.assign(x, x + np);
      b->key_rtol = rtol;
      b->key_maxit = maxit;
    }
    ck(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    std::vector<double> h((size_t)np * 4);
    ck(cudaMemcpyAsync(h.data(), b->stats.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "stats");
    ck(cudaStreamSynchronize(b->stream), "batch solve");
    long long kernels = 0;
    for (int i = 0; i < np; ++i) {
      const int it = (int)h[4 * i];
      kernels += b->pro_kernels[i] + (it > 1 ? (long long)(it - 1) * b->body_kernels[i] : 0);
      if (stats) {
        const double nb2 = h[4 * i + 2];
        stats[i] = gcmg_solve_stats{it, std::sqrt(nb2), nb2 > 0 ? std::sqrt(h[4 * i + 1] / nb2) : 0.0,
                                    (int)h[4 * i + 3]};
      }
    }
    note_launches((int)std::min<long long>(kernels, 1LL << 30));
  });
}

int gcmg_batch_cg_solve_persistent(gcmg_batch* b, const double* const* rhs, double* const* x, double rtol, int maxit,
                                   gcmg_solve_stats* stats) {
  return guarded([&] {
    if (!b || !rhs || !x || !(rtol > 0) || maxit < 1) throw Error(GCMG_ERR_ARG, "bad arguments");
    const int np = (int)b->probs.size();
    for (int i = 0; i < np; ++i) {
      if (b->probs[i]->h.lev.back()->n() && (!rhs[i] || !x[i])) throw Error(GCMG_ERR_ARG, "bad vectors");
      b->probs[i]->h.stream = b->stream;
    }
    DwlState* D = b->dwl.get();
    const bool same = D && D->key_rtol == rtol && D->key_maxit == maxit &&
                      std::equal(D->key_b.begin(), D->key_b.end(), rhs) && std::equal(D->key_x.begin(), D->key_x.end(), x);
    if (!same) {
      build_dwl(*b, rhs, x, rtol, maxit);
      D = b->dwl.get();
    }
    ck(cudaGraphLaunch(D->exec, b->stream), "graph launch");
    note_launches(1);
    std::vector<double> h((size_t)np * 4);
    int st[2] = {0, 0};
    ck(cudaMemcpyAsync(h.data(), b->stats.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "stats");
    ck(cudaMemcpyAsync(st, D->ctl.as<int>() + 2, sizeof(st), cudaMemcpyDeviceToHost, b->stream), "status");
    ck(cudaStreamSynchronize(b->stream), "batch solve");
    if (st[0] == 1) throw Error(GCMG_ERR_INTERNAL, "persistent batch: a grid-barrier wait gave up");
    if (st[0] == 2) throw Error(GCMG_ERR_INTERNAL, "persistent batch: the schedule exceeded its bound");
    D->steps = st[1];
    for (int i = 0; i < np && stats; ++i) {
      const double nb2 = h[4 * i + 2];
      stats[i] = gcmg_solve_stats{(int)h[4 * i], std::sqrt(nb2), nb2 > 0 ? std::sqrt(h[4 * i + 1] / nb2) : 0.0,
                                  (int)h[4 * i + 3]};
    }
  });
}

int gcmg_batch_persistent_wait_test(gcmg_batch* b, int absent_cta, unsigned spin_limit) {
  return guarded([&] {
    if (!b || spin_limit < 1) throw Error(GCMG_ERR_ARG, "bad arguments");
    b->absent_cta = absent_cta;
    b->spin_limit = spin_limit;
    b->dwl.reset();  // the next persistent solve rebuilds its launch with these parameters
  });
}

int gcmg_batch_persistent_info(const gcmg_batch* b, gcmg_persistent_info* info) {
  return guarded([&] {
    if (!b || !info) throw Error(GCMG_ERR_ARG, "null argument");
    const DwlState* D = b->dwl.get();
    if (!D) throw Error(GCMG_ERR_ARG, "no persistent solve yet");
    *info = gcmg_persistent_info{D->grid, (int)D->smem, D->n_ops, D->steps, D->exec ? 1 : 0};
  });
}

}  // extern "C"
