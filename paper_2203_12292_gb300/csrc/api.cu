// C ABI of libgcmg: set-up of the multigrid levels and the orchestration of
// the V-cycle (Algorithms 1-2) and of the preconditioned CG (Sec. 2).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "dwl.h"
#include "handle.h"
#include "splitmix.h"

namespace gcmg {

void upload_tables_cell();
void upload_tables_transfer();
void upload_tables_mlp();

static std::atomic<long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_counter() { return g_launches.load(); }


// cells per tile of a level: the configured size (default 32, the
// autotuner's choice for every degree on GB300), halved while the level would
// give fewer than two tiles per SM (at least 8 cells per tile): small levels
// are latency-bound and finish sooner with more, shorter tiles
int tile_cells_for(int configured, size_t n_cells, int n_sm) {
  int tc = configured ? configured : 32;
  while (tc > 8 && n_cells < (size_t)2 * n_sm * tc) tc /= 2;
  return tc;
}

// multiprocessors of the current device, queried on every call (no cached
// process-wide value: host threads and devices may differ); without a usable
// device the host-only mesh checks assume a GB300 (152 SMs)
int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n <= 0) {
    cudaGetLastError();
    return 152;
  }
  return n;
}

void check_level(const Handle& h, int level) {
  if (level < 0 || level >= (int)h.lev.size()) throw Error(GCMG_ERR_ARG, "level out of range");
}

void prof_flush(Handle& H) {
  Profiler& P = H.prof;
  if (!P.used) return;
  ck(cudaEventSynchronize(P.pool[P.used - 1].b), "profile");
  for (size_t i = 0; i < P.used; ++i) {
    float t = 0.f;
    ck(cudaEventElapsedTime(&t, P.pool[i].a, P.pool[i].b), "profile");
    const size_t idx = (size_t)P.pool[i].level * NSTAGE + P.pool[i].stage;
    P.ms[idx] += t;
    P.cnt[idx] += 1;
  }
  P.used = 0;
}

// returns a record index, or -1 when profiling is off (<= -2: a record of the
// graph being captured)
int prof_begin(Handle& H, int level, int stage) {
  Profiler& P = H.prof;
  if (!P.on) return -1;
  if (H.capturing) {
    Profiler::Rec r;
    ck(cudaEventCreate(&r.a), "event");
    ck(cudaEventCreate(&r.b), "event");
    r.level = level;
    r.stage = stage;
    ck(cudaEventRecordWithFlags(r.a, H.stream, cudaEventRecordExternal), "event");
    H.capturing->recs.push_back(r);
    return -2 - (int)(H.capturing->recs.size() - 1);
  }
  if (P.used == P.pool.size()) {
    if (P.pool.size() >= 8192) prof_flush(H);
    if (P.used == P.pool.size()) {
      Profiler::Rec r;
      ck(cudaEventCreate(&r.a), "event");
      ck(cudaEventCreate(&r.b), "event");
      P.pool.push_back(r);
    }
  }
  Profiler::Rec& r = P.pool[P.used];
  r.level = level;
  r.stage = stage;
  ck(cudaEventRecord(r.a, H.stream), "event");
  return (int)P.used++;
}

void prof_end(Handle& H, int rec) {
  if (rec == -1) return;
  if (rec <= -2) {
    ck(cudaEventRecordWithFlags(H.capturing->recs[-2 - rec].b, H.stream, cudaEventRecordExternal), "event");
    return;
  }
  ck(cudaEventRecord(H.prof.pool[rec].b, H.stream), "event");
}

// after a replay of g has completed: add its timers
void prof_graph(Handle& H, GraphRec& g) {
  Profiler& P = H.prof;
  if (!P.on || g.recs.empty()) return;
  for (auto& r : g.recs) {
    float t = 0.f;
    ck(cudaEventElapsedTime(&t, r.a, r.b), "profile");
    const size_t idx = (size_t)r.level * NSTAGE + r.stage;
    P.ms[idx] += t;
    P.cnt[idx] += 1;
  }
}

void vmult(Handle& H, int l, bool fp64, const void* src, void* dst, int stage) {
  LevelDev& L = *H.lev[l];
  if (L.n() == 0) return;
  const int r = prof_begin(H, l, stage);
  launch_vmult(L.cl, fp64, src, dst, 0, H.stream);
  prof_end(H, r);
}

double dot_host(Handle& H, const double* x, const double* y, int64_t n) {
  if (n == 0) return 0.0;
  launch_dot(x, y, n, H.scratch.as<double>(), H.scal.as<double>(), 8, DOT_STORE, H.stream);
  double v = 0;
  ck(cudaMemcpyAsync(&v, H.scal.as<double>() + 8, sizeof(double), cudaMemcpyDeviceToHost, H.stream), "dot");
  ck(cudaStreamSynchronize(H.stream), "sync");
  return v;
}

// largest eigenvalue of a symmetric tridiagonal matrix by Sturm bisection
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double q = a[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
      if (q == 0.0) q = 1e-300;
      q = a[i] - x - b[i - 1] * b[i - 1] / q;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= m)
      hi = mid;
    else
      lo = mid;
  }
  return hi;
}

// lambda_max of D^{-1} A from the Lanczos tridiagonal matrix of
// Jacobi-preconditioned CG on A y = 1 (set-up; fp64)
double estimate_lambda(Handle& H, int l) {
  LevelDev& L = *H.lev[l];
  const int64_t n = L.n();
  if (n == 0) return 1.0;
  double* r = L.w64a.as<double>();
  double* p = L.w64b.as<double>();
  double* q = L.w64c.as<double>();
  double* z = L.w64c.as<double>();  // z and q are never live together
  {  // start vector: all ones plus a seeded position-keyed perturbation
    std::vector<double> s0(n);
    const double* xyz = L.host.dof_xyz_cache.data();
    for (int64_t i = 0; i < n; ++i) s0[i] = 1.0 + point_value(xyz + 3 * i, LANCZOS_START_SEED);
    ck(cudaMemcpyAsync(r, s0.data(), n * sizeof(double), cudaMemcpyHostToDevice, H.stream), "upload");
    ck(cudaStreamSynchronize(H.stream), "upload");  // s0 is freed on return
  }
  launch_pmul(z, L.dinv64.as<double>(), r, n, H.stream);
  ck(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
  double rz = dot_host(H, r, z, n);
  const double rz0 = rz;
  std::vector<double> alpha, beta;
  for (int it = 0; it < H.cfg.eig_steps; ++it) {
    vmult(H, l, true, p, q);
    const double pq = dot_host(H, p, q, n);
    if (!(pq > 0.0)) break;
    const double a = rz / pq;
    alpha.push_back(a);
    launch_axpy(true, r, q, -a, n, H.stream);
    launch_pmul(z, L.dinv64.as<double>(), r, n, H.stream);
    const double rz_new = dot_host(H, r, z, n);
    if (!(rz_new > 1e-30 * rz0)) break;  // Krylov space exhausted
    const double bt = rz_new / rz;
    beta.push_back(bt);
    launch_xpby(p, z, bt, n, H.stream);
    rz = rz_new;
  }
  const int m = (int)alpha.size();
  if (m == 0) return 1.0;
  std::vector<double> da(m), ob(std::max(m - 1, 0));
  for (int i = 0; i < m; ++i) {
    da[i] = 1.0 / alpha[i] + (i > 0 ? beta[i - 1] / alpha[i - 1] : 0.0);
    if (i + 1 < m) ob[i] = std::sqrt(beta[i]) / alpha[i];
  }
  return tridiag_max_eig(da, ob);
}

void setup_coarse(Handle& H) {
  LevelDev& L = *H.lev[0];
  const int n = (int)L.n();
  H.n0 = n;
  if (n == 0) return;
  std::vector<double> A((size_t)n * n), col(n);
  double* e = L.w64a.as<double>();
  double* y = L.w64b.as<double>();
  for (int j = 0; j < n; ++j) {
    std::vector<double> ej(n, 0.0);
    ej[j] = 1.0;
    ck(cudaMemcpyAsync(e, ej.data(), n * sizeof(double), cudaMemcpyHostToDevice, H.stream), "coarse");
    vmult(H, 0, true, e, y);
    ck(cudaMemcpyAsync(col.data(), y, n * sizeof(double), cudaMemcpyDeviceToHost, H.stream), "coarse");
    ck(cudaStreamSynchronize(H.stream), "sync");
    for (int i = 0; i < n; ++i) A[(size_t)i * n + j] = col[i];
  }
  // Cholesky A = L L^T and the explicit inverse (n <= (k-1)^3)
  std::vector<double> Lc((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      for (int m = 0; m < j; ++m) s -= Lc[(size_t)i * n + m] * Lc[(size_t)j * n + m];
      if (i == j) {
        if (!(s > 0)) throw Error(GCMG_ERR_INTERNAL, "level-0 matrix not positive definite");
        Lc[(size_t)i * n + i] = std::sqrt(s);
      } else {
        Lc[(size_t)i * n + j] = s / Lc[(size_t)j * n + j];
      }
    }
  std::vector<double> inv((size_t)n * n);
  for (int c = 0; c < n; ++c) {
    std::vector<double> v(n, 0.0);
    v[c] = 1.0;
    for (int i = 0; i < n; ++i) {
      double s = v[i];
      for (int m = 0; m < i; ++m) s -= Lc[(size_t)i * n + m] * v[m];
      v[i] = s / Lc[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = v[i];
      for (int m = i + 1; m < n; ++m) s -= Lc[(size_t)m * n + i] * v[m];
      v[i] = s / Lc[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = v[i];
  }
  H.Ainv.upload(inv, H.stream);
}

// Chebyshev coefficients of step `it` (Saad, Iterative Methods, Alg. 12.1)
struct ChebCoef {
  double c1, c2;
};
std::vector<ChebCoef> cheb_coefs(double lam_max, double range, int degree) {
  const double lmin = lam_max / range;
  const double theta = 0.5 * (lam_max + lmin), delta = 0.5 * (lam_max - lmin);
  std::vector<ChebCoef> c;
  double rho = delta / theta;
  c.push_back({0.0, 1.0 / theta});
  for (int it = 1; it < degree; ++it) {
    const double rn = 1.0 / (2.0 * theta / delta - rho);
    c.push_back({rn * rho, 2.0 * rn / delta});
    rho = rn;
  }
  return c;
}

// Chebyshev smoother on level l with vectors x, b, d, t (precision fp64)
void smooth(Handle& H, int l, bool fp64, void* x, const void* b, void* d, void* t, const void* dinv, bool zero_init) {
  LevelDev& L = *H.lev[l];
  const int64_t n = L.n();
  if (n == 0) return;
  const auto c = cheb_coefs(L.lam, H.cfg.smoothing_range, H.cfg.cheb_degree);
  size_t it = 0;
  if (zero_init) {
    launch_cheb_init(fp64, x, d, b, dinv, c[0].c2, n, H.stream);
    it = 1;
  }
  for (; it < c.size(); ++it) {
    vmult(H, l, fp64, x, t);
    launch_cheb_step(fp64, x, d, b, t, dinv, c[it].c1, c[it].c2, n, H.stream);
  }
}

// a_k: mean diagonal entry of the unit-cell Laplace matrix, from the 1D
// matrices: diag(K x M x M + M x K x M + M x M x K) averages to 3 tr K (tr M)^2 / n^3
double mean_ref_diag(int k) {
  const Basis1D& b = basis(k);
  double tk = 0, tm = 0;
  for (int i = 0; i <= k; ++i) {
    tk += b.K[i][i];
    tm += b.M[i][i];
  }
  const double n = k + 1;
  return 3.0 * tk * tm * tm / (n * n * n);
}

// bf16 diagonal features of every cell of level l (once per level)
void ensure_dfeat(Handle& H, int l) {
  LevelDev& L = *H.lev[l];
  if (L.dfeat.p) return;
  const int k = L.host.k, n3 = (k + 1) * (k + 1) * (k + 1);
  const int64_t nc = (int64_t)L.host.cells.size();
  DevBuf tmp;
  tmp.alloc((size_t)nc * n3 * sizeof(double));
  launch_cell_gather(k, L.diag64.as<double>(), nullptr, nc, L.gstart.as<int32_t>(), L.meta.as<CellMeta>(),
                     tmp.as<double>(), H.stream);
  L.dfeat.alloc((size_t)nc * MLP_DF * sizeof(uint16_t));
  launch_mlp_dfeat(tmp.as<double>(), nc, n3, L.meta.as<CellMeta>(), L.cl.dom, mean_ref_diag(k), L.dfeat.p, H.stream);
  ck(cudaStreamSynchronize(H.stream), "diagonal features");
}

// weight image and per-cell diagonal projection of a Q4 network for level l
void mlp_prepare(Handle& H, int l, const gcmg_mlp* net, DevBuf& image, DevBuf& dproj) {
  LevelDev& L = *H.lev[l];
  ensure_dfeat(H, l);
  if (!image.p) image.alloc(mlp_image_bytes());
  if (!dproj.p) dproj.alloc(L.host.cells.size() * 128 * sizeof(float));
  launch_mlp_prepare(net->net.params.as<float>(), L.dfeat.as<uint16_t>(), (int64_t)L.host.cells.size(), image.p,
                     dproj.as<float>(), H.stream);
}

void mlp_correct(Handle& H, int l, const void* image, const float* dproj, bool fp64, const void* r, void* x) {
  LevelDev& L = *H.lev[l];
  MlpFused P{image,
             dproj,
             L.gstart.as<int32_t>(),
             L.own.as<uint32_t>(),
             L.meta.as<CellMeta>(),
             (int64_t)L.host.cells.size(),
             L.cl.dom,
             mean_ref_diag(L.host.k)};
  ck(launch_mlp_correct(P, fp64, r, x, H.stream), "learned correction");
}

// residual r of level l into t, the learned correction c into d, then
// x += om c with the Galerkin step length om = (r.c) / (c.A c): the energy
// norm of the error cannot grow, whatever the network returns
void learned_step(Handle& H, int l) {
  LevelDev& L = *H.lev[l];
  const bool f64 = !L.fp32;
  const int r = prof_begin(H, l, GCMG_STAGE_LEARNED);
  vmult(H, l, f64, L.x.p, L.t.p);
  launch_residual(f64, L.t.p, L.b.p, L.t.p, L.n(), H.stream);
  launch_zero(f64, L.d.p, L.n(), H.stream);
  mlp_correct(H, l, L.mlp_image.p, L.mlp_dproj.as<float>(), f64, L.t.p, L.d.p);
  void* w = f64 ? L.w64a.p : L.w32a.p;
  vmult(H, l, f64, L.d.p, w);
  if (!H.lscratch.p) throw Error(GCMG_ERR_INTERNAL, "learned step without its scratch");
  launch_galerkin_step(f64, L.t.p, L.d.p, w, L.x.p, L.n(), H.lscratch.as<double>(), H.stream);
  prof_end(H, r);
}

bool any_learned(const Handle& H) {
  for (const auto& L : H.lev)
    if (L->smoother != GCMG_SMOOTHER_CHEBYSHEV) return true;
  return false;
}

void vcycle_level(Handle& H, int l) {
  LevelDev& L = *H.lev[l];
  const bool f64 = !L.fp32;
  if (l == 0) {
    const int r = prof_begin(H, 0, GCMG_STAGE_COARSE);
    if (H.n0) launch_coarse_solve(f64, H.Ainv.as<double>(), H.n0, L.b.p, L.x.p, H.stream);
    prof_end(H, r);
    return;
  }
  const void* dinv = f64 ? L.dinv64.p : L.dinv32.p;
  int r = prof_begin(H, l, GCMG_STAGE_PRESMOOTH);
  smooth(H, l, f64, L.x.p, L.b.p, L.d.p, L.t.p, dinv, true);  // presmoothing
  prof_end(H, r);
  r = prof_begin(H, l, GCMG_STAGE_RESIDUAL);
  vmult(H, l, f64, L.x.p, L.t.p);  // A x for the residual
  prof_end(H, r);
  LevelDev& C = *H.lev[l - 1];
  r = prof_begin(H, l, GCMG_STAGE_RESTRICT);
  // the residual r = b - A x is formed in the restriction's gather; global coarsening:
  // b^(l-1) = R r; local smoothing: b^(l-1) += R (r_S, r_E) on top of the values Algorithm 1
  // copied to level l-1 (r_E = -A_ES x_S: b_E is zero on level l)
  if (C.n()) launch_restrict_residual(H.tr[l]->tl, f64, L.b.p, L.t.p, C.b.p, !H.ls, H.stream);
  prof_end(H, r);
  vcycle_level(H, l - 1);
  r = prof_begin(H, l, GCMG_STAGE_PROLONGATE);
  if (C.n()) launch_prolongate_add(H.tr[l]->tl, f64, C.x.p, L.x.p, H.stream);  // prolongation
  prof_end(H, r);
  if (H.stop_after_cgc && l == (int)H.lev.size() - 1) return;
  if (L.smoother == GCMG_SMOOTHER_MLP_REPLACE) {
    learned_step(H, l);  // learned correction instead of postsmoothing
    return;
  }
  r = prof_begin(H, l, GCMG_STAGE_POSTSMOOTH);
  smooth(H, l, f64, L.x.p, L.b.p, L.d.p, L.t.p, dinv, false);  // postsmoothing
  prof_end(H, r);
  if (L.smoother == GCMG_SMOOTHER_MLP_AUGMENT) learned_step(H, l);
}


template <typename F>
void capture(Handle& H, GraphRec& g, F&& body) {
  g.reset();
  if (!H.cap_stream) ck(cudaStreamCreateWithFlags(&H.cap_stream, cudaStreamNonBlocking), "stream");
  cudaStream_t saved = H.stream;
  H.stream = H.cap_stream;
  H.capturing = &g;
  cudaGraph_t graph = nullptr;
  const long long before = g_launches.load();
  cudaError_t e = cudaStreamBeginCapture(H.stream, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(H.stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      H.stream = saved;
      H.capturing = nullptr;
      throw;
    }
    e = cudaStreamEndCapture(H.stream, &graph);
  }
  H.stream = saved;
  H.capturing = nullptr;
  g.kernels = g_launches.load() - before;  // recorded, not run: count them at every replay
  g_launches.fetch_sub(g.kernels);
  ck(e, "graph capture");
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  ck(e, "graph instantiate");
}

// local smoothing, Algorithm 1: the fp64 active vector A.w64a to every level
// (each active DoF to the coarsest level among its active cells, edge entries
// zero), the V-cycle from the finest refinement level, the levels' solutions
// back to A.w64b
void vcycle_ls_body(Handle& H) {
  LevelDev& A = *H.lev.back();
  for (int l = 0; l <= H.top_mg; ++l) {
    LevelDev& L = *H.lev[l];
    launch_zero(!L.fp32, L.b.p, L.n(), H.stream);
    launch_copy_to_level(!L.fp32, A.w64a.as<double>(), L.cp_g.as<int32_t>(), L.cp_idx.as<int32_t>(), L.n_cp, L.b.p,
                         H.stream);
  }
  vcycle_level(H, H.top_mg);
  for (int l = 0; l <= H.top_mg; ++l) {
    LevelDev& L = *H.lev[l];
    launch_copy_from_level(!L.fp32, L.x.p, L.cp_g.as<int32_t>(), L.cp_idx.as<int32_t>(), L.n_cp, A.w64b.as<double>(),
                           H.stream);
  }
}

// the V-cycle on the level vectors (b -> x of the finest level)
void vcycle_core(Handle& H) {
  const int top = H.top_mg;
  auto body = [&] {
    if (H.ls)
      vcycle_ls_body(H);
    else
      vcycle_level(H, top);
  };
  if (!H.use_graphs) {
    body();
    return;
  }
  if (!H.g_core.exec) capture(H, H.g_core, body);
  ck(cudaGraphLaunch(H.g_core.exec, H.stream), "graph launch");
  note_launches((int)H.g_core.kernels);
}

void vcycle(Handle& H, const double* b, double* x) {
  const int top = (int)H.lev.size() - 1;
  if (H.ls) {
    LevelDev& A = *H.lev[top];
    ck(cudaMemcpyAsync(A.w64a.p, b, A.n() * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
    vcycle_core(H);
    ck(cudaMemcpyAsync(x, A.w64b.p, A.n() * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
    return;
  }
  LevelDev& F = *H.lev[top];
  int r = prof_begin(H, top, GCMG_STAGE_CG_VECTOR);
  if (F.fp32)
    launch_cast(false, b, F.b.p, F.n(), H.stream);
  else
    ck(cudaMemcpyAsync(F.b.p, b, F.n() * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
  prof_end(H, r);
  vcycle_core(H);
  r = prof_begin(H, top, GCMG_STAGE_CG_VECTOR);
  if (F.fp32)
    launch_cast(true, F.x.p, x, F.n(), H.stream);
  else
    ck(cudaMemcpyAsync(x, F.x.p, F.n() * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
  prof_end(H, r);
}


void check_config(const gcmg_config* cfg) {
  if (cfg->degree < 1 || cfg->degree > KMAX) throw Error(GCMG_ERR_ARG, "degree must be 1..4");
  if (cfg->cheb_degree < 1 || !(cfg->smoothing_range > 1.0) || cfg->eig_steps < 1)
    throw Error(GCMG_ERR_ARG, "bad smoother parameters");
  if (cfg->tile_cells < 0 || cfg->tile_cells > 255) throw Error(GCMG_ERR_ARG, "tile_cells must be 0..255");
  if (cfg->cell_kernel < 0 || cfg->cell_kernel > 3) throw Error(GCMG_ERR_ARG, "cell_kernel must be 0, 1, 2 or 3");
  if (cfg->transfer_chunk != 0 && cfg->transfer_chunk != 4 && cfg->transfer_chunk != 8)
    throw Error(GCMG_ERR_ARG, "transfer_chunk must be 0, 4 or 8");
  if (cfg->cell_threads != 0 && cfg->cell_threads != 128 && cfg->cell_threads != 256 && cfg->cell_threads != 384 &&
      cfg->cell_threads != 512)
    throw Error(GCMG_ERR_ARG, "cell_threads must be 0, 128, 256, 384 or 512");
  if (cfg->local_smoothing != 0 && cfg->local_smoothing != 1) throw Error(GCMG_ERR_ARG, "local_smoothing must be 0 or 1");
  if (cfg->local_smoothing && cfg->p_coarsening)
    throw Error(GCMG_ERR_ARG, "local smoothing uses the refinement levels (no polynomial coarsening)");
}

// the per-degree constant tables of every translation unit, once per device
void upload_all_tables() {
  static std::mutex mu;
  static std::vector<char> done;
  int dev = 0;
  ck(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lock(mu);
  if ((int)done.size() <= dev) done.resize(dev + 1, 0);
  if (done[dev]) return;
  upload_tables_cell();
  upload_tables_lanes();
  upload_tables_transfer();
  upload_tables_mlp();
  upload_tables_dwl();
  ck(cudaDeviceSynchronize(), "upload tables");
  done[dev] = 1;
}

void setup_numerics(Handle& H) {
  const int nl = (int)H.lev.size();
  // Jacobi diagonals (Eqs. 3-4)
  for (int l = 0; l < nl; ++l) {
    const int k = H.lev[l]->cl.k;
    if (!H.diag_tab[k].p) {
      const int n3 = (k + 1) * (k + 1) * (k + 1);
      H.diag_tab[k].alloc((size_t)512 * n3 * sizeof(double));
      launch_diag_table(k, H.diag_tab[k].as<double>(), H.stream);
    }
    LevelDev& L = *H.lev[l];
    if (L.n() == 0) continue;
    launch_diag(L.cl, H.diag_tab[k].as<double>(), L.diag64.as<double>(), H.stream);
    launch_invert(L.diag64.as<double>(), L.dinv64.as<double>(), L.dinv32.as<float>(), L.n(), H.stream);
    // local smoothing: the smoother sees A_SS only, edge values stay as they are
    if (L.n_edge) launch_zero_at(L.edge_idx.as<int32_t>(), L.n_edge, L.dinv64.as<double>(), L.dinv32.as<float>(), H.stream);
  }
  ck_launches("diagonal");
  ck(cudaStreamSynchronize(H.stream), "diagonal");
  setup_coarse(H);
  ck_launches("coarse matrix");
  for (int l = 1; l <= H.top_mg; ++l) {
    H.lev[l]->lam = H.cfg.eig_safety * estimate_lambda(H, l);
    ck_launches("eigenvalue estimate");
  }
  H.g_core.reset();
  H.g_a.reset();
}

void setup_handle(Handle& H, const std::vector<Octree>& gc_meshes, int lmax, const gcmg_config& cfg) {
  H.cfg = cfg;
  H.n_sm = device_sm_count();
  H.ls = cfg.local_smoothing != 0;
  // local smoothing: the refinement levels 0..L of the finest mesh, then the active mesh itself
  std::vector<Octree> ls_meshes;
  if (H.ls) {
    const Octree& fine = gc_meshes.back();
    const int L = fine.max_level();
    for (int l = 0; l <= L; ++l) ls_meshes.push_back(refinement_level(fine, l));
    ls_meshes.push_back(fine);
  }
  const std::vector<Octree>& meshes = H.ls ? ls_meshes : gc_meshes;
  // level list: (mesh index, degree), coarsest first
  std::vector<std::pair<int, int>> spec;
  const int nm = (int)meshes.size();
  if (cfg.p_coarsening) {
    for (int m = 0; m + 1 < nm; ++m) spec.push_back({m, 1});
    std::vector<int> degs{cfg.degree};
    while (degs.back() > 1) degs.push_back(degs.back() / 2);
    for (auto it = degs.rbegin(); it != degs.rend(); ++it) spec.push_back({nm - 1, *it});
  } else {
    for (int m = 0; m < nm; ++m) spec.push_back({m, cfg.degree});
  }
  const int nl = (int)spec.size();
  for (int l = 0; l < nl; ++l) {
    auto L = std::make_unique<LevelDev>();
    const int k = spec[l].second;
    const int tc = tile_cells_for(cfg.tile_cells, meshes[spec[l].first].leaves.size(), H.n_sm);
    build_level(meshes[spec[l].first], k, tc, lmax, L->host);
    L->fp32 = cfg.mg_fp32 != 0;
    L->cl.use_lines = cfg.cell_kernel != 2;
    L->cl.use_lanes = (cfg.cell_kernel == 0 && tc == 32) || cfg.cell_kernel == 3;
    L->cl.threads = cfg.cell_threads ? cfg.cell_threads : 256;
    LevelHost& lh = L->host;
    L->tiles.upload(lh.tiles, H.stream);
    L->halo.alloc(lh.foreign.size() * sizeof(double));
    L->halo_dofs.upload(lh.halo_dofs, H.stream);
    L->halo_ptr.upload(lh.halo_ptr, H.stream);
    L->halo_src.upload(lh.halo_src, H.stream);
    L->halo_pos.upload(lh.halo_pos, H.stream);
    L->meta.upload(lh.meta, H.stream);
    L->foreign.upload(lh.foreign, H.stream);
    L->subptr.upload(lh.subptr, H.stream);
    L->perm.upload(lh.perm, H.stream);
    L->lane_tiles.upload(lh.lane, H.stream);
    L->lane_order.upload(lh.lane_order, H.stream);
    L->lane_hang.upload(lh.lane_hang, H.stream);
    {  // the lane kernels' records in launch order
      std::vector<TileInfo> ti_lo;
      std::vector<LaneTile> lt_lo;
      std::vector<LaneHang> lh_lo;
      for (size_t b = 0; b < lh.lane_order.size(); ++b) {
        const int32_t t = lh.lane_order[b];
        ti_lo.push_back(lh.tiles[t]);
        lt_lo.push_back(lh.lane[t]);
        if ((int)b < lh.n_hang_tiles) lh_lo.push_back(lh.lane_hang[t]);
      }
      L->tiles_lo.upload(ti_lo, H.stream);
      L->lane_tiles_lo.upload(lt_lo, H.stream);
      L->lane_hang_lo.upload(lh_lo, H.stream);
    }
    std::vector<int32_t> ijk(lh.cells.size() * 3);
    for (size_t c = 0; c < lh.cells.size(); ++c) {
      ijk[3 * c] = lh.cells[c].i;
      ijk[3 * c + 1] = lh.cells[c].j;
      ijk[3 * c + 2] = lh.cells[c].k;
    }
    L->cell_ijk.upload(ijk, H.stream);
    L->gstart.upload(lh.gstart, H.stream);
    L->own.upload(lh.own, H.stream);
    L->mask.upload(lh.mask, H.stream);
    CellLaunch& c = L->cl;
    c.tiles = L->tiles.as<TileInfo>();
    c.n_tiles = (int)lh.tiles.size();
    c.halo = L->halo.p;
    c.halo_dofs = L->halo_dofs.as<int32_t>();
    c.halo_ptr = L->halo_ptr.as<int32_t>();
    c.halo_src = L->halo_src.as<int32_t>();
    c.halo_pos = L->halo_pos.as<int32_t>();
    c.n_halo = (int)lh.halo_dofs.size();
    c.meta = L->meta.as<CellMeta>();
    c.foreign = L->foreign.as<int32_t>();
    c.subptr = L->subptr.as<uint16_t>();
    c.perm = L->perm.as<uint8_t>();
    c.lane_tiles = lh.lane.empty() ? nullptr : L->lane_tiles.p;
    c.lane_order = lh.lane.empty() ? nullptr : L->lane_order.as<int32_t>();
    c.lane_hang = lh.lane.empty() ? nullptr : L->lane_hang.p;
    c.tiles_lo = lh.lane.empty() ? nullptr : L->tiles_lo.as<TileInfo>();
    c.lane_tiles_lo = lh.lane.empty() ? nullptr : L->lane_tiles_lo.p;
    c.lane_hang_lo = lh.lane.empty() ? nullptr : L->lane_hang_lo.p;
    c.n_hang_tiles = lh.n_hang_tiles;
    c.cell_ijk = L->cell_ijk.as<int32_t>();
    c.k = k;
    c.tc = tc;
    c.n_sm = H.n_sm;
    c.chunk = cfg.transfer_chunk;
    c.max_local = lh.max_local;
    c.lo = lh.lo;
    c.dom = lh.hi - lh.lo;
    const int64_t n = lh.n_free;
    const size_t vb = L->fp32 ? sizeof(float) : sizeof(double);
    L->x.alloc(n * vb);
    L->b.alloc(n * vb);
    L->d.alloc(n * vb);
    L->t.alloc(n * vb);
    L->w64a.alloc(n * sizeof(double));
    L->w64b.alloc(n * sizeof(double));
    L->w64c.alloc(n * sizeof(double));
    L->w32a.alloc(n * sizeof(float));
    L->w32b.alloc(n * sizeof(float));
    L->diag64.alloc(n * sizeof(double));
    L->dinv64.alloc(n * sizeof(double));
    L->dinv32.alloc(n * sizeof(float));
    H.lev.push_back(std::move(L));
  }
  H.top_mg = H.ls ? nl - 2 : nl - 1;
  H.tr.resize(nl);
  for (int l = 1; l <= H.top_mg; ++l) {
    auto T = std::make_unique<TransferDev>();
    LevelHost& fh = H.lev[l]->host;
    LevelHost& ch = H.lev[l - 1]->host;
    if (spec[l].first == spec[l - 1].first)
      build_transfer_p(fh, ch, T->host);
    else
      build_transfer_h(fh, ch, T->host, H.ls);
    T->fine_of.upload(T->host.fine_of, H.stream);
    T->refined.upload(T->host.refined, H.stream);
    TransferLaunch& t = T->tl;
    t.kind = T->host.kind;
    t.kf = fh.k;
    t.kc = ch.k;
    t.n_coarse = (int)ch.cells.size();
    t.fine_of = T->fine_of.as<int32_t>();
    t.refined = T->refined.as<uint8_t>();
    t.gstart_f = H.lev[l]->gstart.as<int32_t>();
    t.own_f = H.lev[l]->own.as<uint32_t>();
    t.gstart_c = H.lev[l - 1]->gstart.as<int32_t>();
    t.mask_c = H.lev[l - 1]->mask.as<uint16_t>();
    t.coarse = H.lev[l - 1]->cl;
    H.tr[l] = std::move(T);
  }
  if (H.ls) {
    // refinement edges of every level, Algorithm 1's copy pairs
    std::vector<const LevelHost*> hosts;
    for (int l = 0; l <= H.top_mg; ++l) {
      LevelDev& L = *H.lev[l];
      const std::vector<int32_t> e = refinement_edge_dofs(L.host, meshes[l]);
      if (l == 0 && !e.empty()) throw Error(GCMG_ERR_INTERNAL, "level 0 does not cover the domain");
      L.n_edge = (int64_t)e.size();
      if (L.n_edge) L.edge_idx.upload(e, H.stream);
      hosts.push_back(&L.host);
    }
    std::vector<std::vector<int32_t>> cg, ci;
    local_copy_map(H.lev.back()->host, hosts, cg, ci);
    for (int l = 0; l <= H.top_mg; ++l) {
      LevelDev& L = *H.lev[l];
      L.n_cp = (int64_t)cg[l].size();
      if (L.n_cp) {
        L.cp_g.upload(cg[l], H.stream);
        L.cp_idx.upload(ci[l], H.stream);
      }
    }
    ck(cudaStreamSynchronize(H.stream), "upload");  // the host vectors are freed on return
  }
  H.scratch.alloc(DOT_BLOCKS * sizeof(double));
  H.scal.alloc(16 * sizeof(double));
  ck(cudaMemsetAsync(H.scal.p, 0, 16 * sizeof(double), H.stream), "memset");
  setup_numerics(H);
  const int64_t nf = H.lev.back()->n();
  H.cg_r.alloc(nf * sizeof(double));
  H.cg_p.alloc(nf * sizeof(double));
  H.cg_q.alloc(nf * sizeof(double));
  H.cg_z.alloc(nf * sizeof(double));
  H.cg_x.alloc(nf * sizeof(double));
  ck(cudaStreamSynchronize(H.stream), "setup");
  ck_launches("setup");
}

}  // namespace gcmg

using namespace gcmg;

extern "C" {

const char* gcmg_last_error(void) { return g_err.c_str(); }

int64_t gcmg_launch_count(void) { return (int64_t)g_launches.load(); }

int gcmg_mesh_create(double lo, double hi, int n_steps, const gcmg_refine_step* steps, gcmg_mesh** out) {
  return guarded([&] {
    if (!out || (n_steps > 0 && !steps) || !(hi > lo) || n_steps < 0) throw Error(GCMG_ERR_ARG, "bad mesh arguments");
    auto m = std::make_unique<gcmg_mesh>();
    Octree t;
    t.lo = lo;
    t.hi = hi;
    t.leaves.insert(cell_key(0, 0, 0, 0));
    for (int i = 0; i < n_steps; ++i) {
      if (steps[i].pred < 0 || steps[i].pred > 4) throw Error(GCMG_ERR_ARG, "unknown refinement predicate");
      t.refine_step(RefineStep{steps[i].pred, steps[i].a, steps[i].b, steps[i].c, steps[i].d});
      if (t.max_level() > 17) throw Error(GCMG_ERR_ARG, "mesh deeper than 17 levels");
    }
    m->lmax = t.max_level();
    std::vector<Octree> lv{t};
    while (lv.back().leaves.size() > 1) lv.push_back(coarsen_global(lv.back()));
    std::reverse(lv.begin(), lv.end());
    m->levels = std::move(lv);
    *out = m.release();
  });
}

void gcmg_mesh_destroy(gcmg_mesh* mesh) { delete mesh; }

int gcmg_mesh_num_levels(const gcmg_mesh* mesh, int* n) {
  return guarded([&] {
    if (!mesh || !n) throw Error(GCMG_ERR_ARG, "null argument");
    *n = (int)mesh->levels.size();
  });
}

int gcmg_mesh_level_cells(const gcmg_mesh* mesh, int level, int64_t* n_cells) {
  return guarded([&] {
    if (!mesh || !n_cells || level < 0 || level >= (int)mesh->levels.size()) throw Error(GCMG_ERR_ARG, "bad level");
    *n_cells = (int64_t)mesh->levels[level].leaves.size();
  });
}

int gcmg_mesh_dof_coords(const gcmg_mesh* mesh, int level, int degree, int tile_cells, int64_t* n_free, double* xyz) {
  return guarded([&] {
    if (!mesh || !n_free || level < 0 || level >= (int)mesh->levels.size()) throw Error(GCMG_ERR_ARG, "bad level");
    if (degree < 1 || degree > KMAX) throw Error(GCMG_ERR_ARG, "degree must be 1..4");
    if (tile_cells < 0 || tile_cells > 255) throw Error(GCMG_ERR_ARG, "tile_cells must be 0..255");
    LevelHost L;
    build_level(mesh->levels[level], degree, tile_cells_for(tile_cells, mesh->levels[level].leaves.size(), device_sm_count()),
                mesh->lmax, L);
    *n_free = L.n_free;
    if (xyz) std::memcpy(xyz, L.dof_xyz_cache.data(), L.dof_xyz_cache.size() * sizeof(double));
  });
}

int gcmg_mesh_check_level(const gcmg_mesh* mesh, int level, int degree, int tile_cells) {
  return guarded([&] {
    if (!mesh || level < 0 || level >= (int)mesh->levels.size()) throw Error(GCMG_ERR_ARG, "bad level");
    if (degree < 1 || degree > KMAX) throw Error(GCMG_ERR_ARG, "degree must be 1..4");
    if (tile_cells < 0 || tile_cells > 255) throw Error(GCMG_ERR_ARG, "tile_cells must be 0..255");
    LevelHost L;
    build_level(mesh->levels[level], degree, tile_cells_for(tile_cells, mesh->levels[level].leaves.size(), device_sm_count()),
                mesh->lmax, L);
    try {
      validate_level(L);
    } catch (const std::exception& e) {
      throw Error(GCMG_ERR_INTERNAL, e.what());
    }
  });
}

int gcmg_config_default(gcmg_config* cfg) {
  return guarded([&] {
    if (!cfg) throw Error(GCMG_ERR_ARG, "null config");
    cfg->degree = 1;
    cfg->p_coarsening = 0;
    cfg->mg_fp32 = 1;
    cfg->cheb_degree = 3;
    cfg->smoothing_range = 20.0;
    cfg->eig_steps = 12;
    cfg->eig_safety = 1.2;
    cfg->tile_cells = 0;
    cfg->cell_kernel = 0;
    cfg->cell_threads = 0;
    cfg->local_smoothing = 0;
    cfg->transfer_chunk = 0;
  });
}

int gcmg_setup(const gcmg_mesh* mesh, const gcmg_config* cfg, void* stream, gcmg_handle** out) {
  return guarded([&] {
    if (!mesh || !cfg || !out) throw Error(GCMG_ERR_ARG, "null argument");
    check_config(cfg);
    upload_all_tables();
    auto hh = std::make_unique<gcmg_handle>();
    hh->h.stream = static_cast<cudaStream_t>(stream);
    setup_handle(hh->h, mesh->levels, mesh->lmax, *cfg);
    *out = hh.release();
  });
}

void gcmg_destroy(gcmg_handle* h) { delete h; }

int gcmg_set_stream(gcmg_handle* h, void* stream) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    h->h.stream = static_cast<cudaStream_t>(stream);
  });
}

int gcmg_num_levels(const gcmg_handle* h, int* n) {
  return guarded([&] {
    if (!h || !n) throw Error(GCMG_ERR_ARG, "null argument");
    *n = (int)h->h.lev.size();
  });
}

int gcmg_get_level_info(const gcmg_handle* h, int level, gcmg_level_info* info) {
  return guarded([&] {
    if (!h || !info) throw Error(GCMG_ERR_ARG, "null argument");
    check_level(h->h, level);
    const LevelDev& L = *h->h.lev[level];
    info->n_free = L.host.n_free;
    info->n_cells = (int64_t)L.host.cells.size();
    info->degree = L.host.k;
    info->n_tiles = (int)L.host.tiles.size();
    info->n_halo = (int64_t)L.host.halo_dofs.size();
    info->tile_cells = L.host.tile_cells;
    info->max_local = L.host.max_local;
    info->fp32 = L.fp32 ? 1 : 0;
  });
}

int gcmg_level_dof_coords(const gcmg_handle* h, int level, double* xyz) {
  return guarded([&] {
    if (!h || !xyz) throw Error(GCMG_ERR_ARG, "null argument");
    check_level(h->h, level);
    const auto& v = h->h.lev[level]->host.dof_xyz_cache;
    std::memcpy(xyz, v.data(), v.size() * sizeof(double));
  });
}

int gcmg_level_edge_dofs(const gcmg_handle* h, int level, int64_t* n, int32_t* idx) {
  return guarded([&] {
    if (!h || !n) throw Error(GCMG_ERR_ARG, "null argument");
    check_level(h->h, level);
    const LevelDev& L = *h->h.lev[level];
    *n = L.n_edge;
    if (idx && L.n_edge)
      ck(cudaMemcpy(idx, L.edge_idx.p, L.n_edge * sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
  });
}

int gcmg_set_profiling(gcmg_handle* h, int on) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    Profiler& P = h->h.prof;
    prof_flush(h->h);
    P.on = on != 0;
    h->h.g_core.reset();
    h->h.g_a.reset();
    P.nlev = (int)h->h.lev.size();
    P.ms.assign((size_t)P.nlev * NSTAGE, 0.0);
    P.cnt.assign((size_t)P.nlev * NSTAGE, 0);
  });
}

int gcmg_get_profile(gcmg_handle* h, int level, int stage, int64_t* count, double* ms) {
  return guarded([&] {
    if (!h || !count || !ms || stage < 0 || stage >= NSTAGE) throw Error(GCMG_ERR_ARG, "bad arguments");
    check_level(h->h, level);
    prof_flush(h->h);
    Profiler& P = h->h.prof;
    if (P.ms.empty()) {
      *count = 0;
      *ms = 0.0;
      return;
    }
    *count = P.cnt[(size_t)level * NSTAGE + stage];
    *ms = P.ms[(size_t)level * NSTAGE + stage];
  });
}

int gcmg_dot(gcmg_handle* h, const double* x, const double* y, int64_t n, double* result) {
  return guarded([&] {
    if (!h || !result || n < 0 || (n > 0 && (!x || !y))) throw Error(GCMG_ERR_ARG, "bad arguments");
    Handle& H = h->h;
    if (n == 0) {
      ck(cudaMemsetAsync(result, 0, sizeof(double), H.stream), "memset");
      return;
    }
    launch_dot(x, y, n, H.scratch.as<double>(), result, 0, DOT_STORE, H.stream);
    ck_launches("dot");
  });
}

int gcmg_dot_noalloc(const double* x, const double* y, int64_t n, double* result, void* stream) {
  return guarded([&] {
    if (!result || n < 0 || (n > 0 && (!x || !y))) throw Error(GCMG_ERR_ARG, "bad arguments");
    if (n > dot_noalloc_max_n())
      throw Error(GCMG_ERR_ARG, "gcmg_dot_noalloc: n = " + std::to_string(n) + " exceeds the maximum " +
                                    std::to_string(dot_noalloc_max_n()) + " (fixed partial-sum array)");
    ck(launch_dot_noalloc(x, y, n, result, static_cast<cudaStream_t>(stream)), "gcmg_dot_noalloc");
  });
}

int gcmg_vmult_host_many(gcmg_handle* h, int level, int fp64, int n, const void* const* src, void* const* dst) {
  return guarded([&] {
    if (!h || n < 0 || (n > 0 && (!src || !dst))) throw Error(GCMG_ERR_ARG, "bad arguments");
    check_level(h->h, level);
    Handle& H = h->h;
    LevelDev& L = *H.lev[level];
    if (L.n() == 0 || n == 0) return;
    for (int i = 0; i < n; ++i)
      if (!src[i] || !dst[i]) throw Error(GCMG_ERR_ARG, "bad vectors");
    const bool f64 = fp64 != 0;
    const size_t bytes = L.n() * (f64 ? sizeof(double) : sizeof(float));
    if (!H.copy_stream) ck(cudaStreamCreateWithFlags(&H.copy_stream, cudaStreamNonBlocking), "stream");
    if (!H.out_stream) ck(cudaStreamCreateWithFlags(&H.out_stream, cudaStreamNonBlocking), "stream");
    for (cudaEvent_t& e : H.many_ev)
      if (!e) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    for (int k = 0; k < 2; ++k) {
      if (H.many_in[k].bytes < bytes) H.many_in[k].alloc(bytes);
      if (H.many_out[k].bytes < bytes) H.many_out[k].alloc(bytes);
    }
    cudaEvent_t* ev_in = H.many_ev;
    cudaEvent_t* ev_comp = H.many_ev + 2;
    cudaEvent_t* ev_out = H.many_ev + 4;
    // everything queued on the handle's stream before comes first
    ck(cudaEventRecord(H.many_ev[6], H.stream), "event");
    ck(cudaStreamWaitEvent(H.copy_stream, H.many_ev[6], 0), "wait");
    ck(cudaStreamWaitEvent(H.out_stream, H.many_ev[6], 0), "wait");
    // vector i uses buffer pair k = i % 2: its input copy waits for the operator of vector i - 2
    // (the last reader of in[k]), its operator for the output copy of vector i - 2 (the last
    // reader of out[k]); so copies in, operators and copies out of neighbouring vectors overlap
    for (int i = 0; i < n; ++i) {
      const int k = i & 1;
      if (i >= 2) ck(cudaStreamWaitEvent(H.copy_stream, ev_comp[k], 0), "wait");
      ck(cudaMemcpyAsync(H.many_in[k].p, src[i], bytes, cudaMemcpyHostToDevice, H.copy_stream), "copy in");
      ck(cudaEventRecord(ev_in[k], H.copy_stream), "event");
      ck(cudaStreamWaitEvent(H.stream, ev_in[k], 0), "wait");
      if (i >= 2) ck(cudaStreamWaitEvent(H.stream, ev_out[k], 0), "wait");
      vmult(H, level, f64, H.many_in[k].p, H.many_out[k].p);
      ck(cudaEventRecord(ev_comp[k], H.stream), "event");
      ck(cudaStreamWaitEvent(H.out_stream, ev_comp[k], 0), "wait");
      ck(cudaMemcpyAsync(dst[i], H.many_out[k].p, bytes, cudaMemcpyDeviceToHost, H.out_stream), "copy out");
      ck(cudaEventRecord(ev_out[k], H.out_stream), "event");
    }
    ck(cudaStreamSynchronize(H.out_stream), "vmult_host_many");
    ck(cudaStreamSynchronize(H.copy_stream), "vmult_host_many");
    ck(cudaStreamSynchronize(H.stream), "vmult_host_many");
  });
}

int gcmg_vmult_host(gcmg_handle* h, int level, int fp64, const void* src, void* dst) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    Handle& H = h->h;
    LevelDev& L = *H.lev[level];
    if (L.n() == 0) return;
    if (!src || !dst) throw Error(GCMG_ERR_ARG, "bad vectors");
    const bool f64 = fp64 != 0;
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    const size_t bytes = L.n() * es;
    char* a = static_cast<char*>(f64 ? L.w64a.p : L.w32a.p);
    void* b = f64 ? L.w64b.p : L.w32b.p;
    const int nt = L.cl.n_tiles;
    constexpr int K = 8;  // tile groups
    if (vmult_tiles_ok(L.cl, f64) && nt >= K) {
      // the input arrives in DoF order on a second stream; tile group g starts once the DoFs
      // below the end of its owned range are in (a tile reads no DoF above that)
      if (!H.copy_stream) ck(cudaStreamCreateWithFlags(&H.copy_stream, cudaStreamNonBlocking), "stream");
      while (H.pipe_ev.size() < K + 1) {
        cudaEvent_t e;
        ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        H.pipe_ev.push_back(e);
      }
      ck(cudaEventRecord(H.pipe_ev[K], H.stream), "event");
      ck(cudaStreamWaitEvent(H.copy_stream, H.pipe_ev[K], 0), "wait");
      const char* sp = static_cast<const char*>(src);
      int64_t done = 0;
      for (int g = 0; g < K; ++g) {
        const int t0 = (int)((int64_t)g * nt / K), t1 = (int)((int64_t)(g + 1) * nt / K);
        const TileInfo& last = L.host.tiles[t1 - 1];
        const int64_t end = (g == K - 1) ? L.n() : (int64_t)last.dof_begin + last.n_owned;
        if (end > done)
          ck(cudaMemcpyAsync(a + done * es, sp + done * es, (end - done) * es, cudaMemcpyHostToDevice, H.copy_stream),
             "copy in");
        done = std::max(done, end);
        ck(cudaEventRecord(H.pipe_ev[g], H.copy_stream), "event");
        ck(cudaStreamWaitEvent(H.stream, H.pipe_ev[g], 0), "wait");
        launch_vmult_tiles(L.cl, f64, a, b, t0, t1, H.stream);
      }
      launch_halo_add(L.cl, f64, b, H.stream);
    } else {
      ck(cudaMemcpyAsync(a, src, bytes, cudaMemcpyHostToDevice, H.stream), "copy in");
      vmult(H, level, f64, a, b);
    }
    ck(cudaMemcpyAsync(dst, b, bytes, cudaMemcpyDeviceToHost, H.stream), "copy out");
    ck(cudaStreamSynchronize(H.stream), "vmult_host");
  });
}

int gcmg_vmult(gcmg_handle* h, int level, int fp64, const void* src, void* dst) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    if (h->h.lev[level]->n() == 0) return;
    if (!src || !dst || src == dst) throw Error(GCMG_ERR_ARG, "bad vectors");
    vmult(h->h, level, fp64 != 0, src, dst);
    ck_launches("vmult");
  });
}

int gcmg_residual(gcmg_handle* h, int level, int fp64, const void* b, const void* x, void* r) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    const int64_t n = h->h.lev[level]->n();
    if (n == 0) return;
    if (!b || !x || !r || x == r) throw Error(GCMG_ERR_ARG, "bad vectors");
    vmult(h->h, level, fp64 != 0, x, r);
    launch_residual(fp64 != 0, r, b, r, n, h->h.stream);
    ck_launches("residual");
  });
}

int gcmg_vcycle_cgc(gcmg_handle* h, const double* b, double* x) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    Handle& H = h->h;
    if (H.ls) throw Error(GCMG_ERR_ARG, "not available with local smoothing");
    const int top = (int)H.lev.size() - 1;
    LevelDev& F = *H.lev[top];
    if (F.n() == 0) return;
    if (!b || !x) throw Error(GCMG_ERR_ARG, "bad vectors");
    if (F.fp32)
      launch_cast(false, b, F.b.p, F.n(), H.stream);
    else
      ck(cudaMemcpyAsync(F.b.p, b, F.n() * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
    H.stop_after_cgc = true;  // plain launches: the captured graph holds the full cycle
    try {
      vcycle_level(H, top);
    } catch (...) {
      H.stop_after_cgc = false;
      throw;
    }
    H.stop_after_cgc = false;
    if (F.fp32)
      launch_cast(true, F.x.p, x, F.n(), H.stream);
    else
      ck(cudaMemcpyAsync(x, F.x.p, F.n() * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
    ck_launches("vcycle");
  });
}

int gcmg_diagonal(gcmg_handle* h, int level, double* dst) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    LevelDev& L = *h->h.lev[level];
    if (L.n() && !dst) throw Error(GCMG_ERR_ARG, "bad vector");
    if (L.n())
      ck(cudaMemcpyAsync(dst, L.diag64.p, L.n() * sizeof(double), cudaMemcpyDeviceToDevice, h->h.stream), "copy");
  });
}

int gcmg_rhs(gcmg_handle* h, int n_modes, const double* modes, double amp, double* b) {
  return guarded([&] {
    if (!h || n_modes < 0 || (n_modes > 0 && !modes)) throw Error(GCMG_ERR_ARG, "bad arguments");
    Handle& H = h->h;
    LevelDev& L = *H.lev.back();
    if (L.n() && !b) throw Error(GCMG_ERR_ARG, "bad vector");
    if (n_modes > 0) {
      std::vector<double> v(modes, modes + 4 * n_modes);
      H.modes.upload(v, H.stream);
    }
    RhsDesc f{n_modes ? FUNC_FOURIER : FUNC_ONE, n_modes ? H.modes.as<double>() : nullptr, n_modes, amp};
    if (L.n()) launch_rhs(L.cl, f, b, H.stream);
    ck(cudaStreamSynchronize(H.stream), "rhs");
  });
}

int gcmg_rhs_dirichlet(gcmg_handle* h, int kind, int n, const double* params, double* b) {
  return guarded([&] {
    if (!h || !params) throw Error(GCMG_ERR_ARG, "bad arguments");
    std::vector<double> v;
    if (kind == GCMG_FUNC_GAUSSIAN) {
      if (n != 1 || !(params[0] > 0.0) || !std::isfinite(params[0])) throw Error(GCMG_ERR_ARG, "gaussian: n = 1, alpha > 0");
      v.assign(params, params + 4);
    } else if (kind == GCMG_FUNC_POLYNOMIAL) {
      if (n < 1 || n > 64) throw Error(GCMG_ERR_ARG, "polynomial: 1..64 terms");
      v.assign(params, params + 4 * n);
      for (int m = 0; m < n; ++m)
        for (int d = 1; d <= 3; ++d) {
          const double e = v[4 * m + d];
          if (!(e >= 0.0 && e <= 16.0 && e == std::floor(e))) throw Error(GCMG_ERR_ARG, "polynomial: exponents 0..16");
        }
    } else {
      throw Error(GCMG_ERR_ARG, "unknown function kind");
    }
    Handle& H = h->h;
    LevelDev& L = *H.lev.back();
    if (L.n() && !b) throw Error(GCMG_ERR_ARG, "bad vector");
    H.modes.upload(v, H.stream);
    RhsDesc u{kind, H.modes.as<double>(), n, 1.0};
    if (L.n()) {
      launch_rhs(L.cl, u, b, H.stream);       // C^T F, f = -Lap u
      launch_rhs_lift(L.cl, u, b, H.stream);  // - C^T A_all u_g
    }
    ck(cudaStreamSynchronize(H.stream), "rhs");
  });
}

int gcmg_get_lambda(const gcmg_handle* h, int level, double* lam) {
  return guarded([&] {
    if (!h || !lam) throw Error(GCMG_ERR_ARG, "null argument");
    check_level(h->h, level);
    *lam = h->h.lev[level]->lam;
  });
}

int gcmg_set_lambda(gcmg_handle* h, int level, double lam) {
  return guarded([&] {
    if (!h || !(lam > 0)) throw Error(GCMG_ERR_ARG, "bad lambda");
    check_level(h->h, level);
    h->h.lev[level]->lam = lam;
    h->h.g_core.reset();
  });
}

int gcmg_smooth(gcmg_handle* h, int level, int fp64, void* x, const void* b, int zero_init) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    LevelDev& L = *h->h.lev[level];
    if (L.n() == 0) return;
    if (!x || !b) throw Error(GCMG_ERR_ARG, "bad vectors");
    if (fp64)
      smooth(h->h, level, true, x, b, L.w64a.p, L.w64b.p, L.dinv64.p, zero_init != 0);
    else
      smooth(h->h, level, false, x, b, L.w32a.p, L.w32b.p, L.dinv32.p, zero_init != 0);
    ck_launches("smooth");
  });
}

int gcmg_prolongate_add(gcmg_handle* h, int fine_level, int fp64, const void* coarse, void* fine) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    if (fine_level < 1) throw Error(GCMG_ERR_ARG, "fine_level must be >= 1");
    check_level(h->h, fine_level);
    if (!h->h.tr[fine_level]) throw Error(GCMG_ERR_ARG, "no transfer into this level (the active mesh of local smoothing)");
    if (h->h.lev[fine_level - 1]->n() == 0 || h->h.lev[fine_level]->n() == 0) return;
    if (!coarse || !fine) throw Error(GCMG_ERR_ARG, "bad vectors");
    if (h->h.lev[fine_level - 1]->n())
      launch_prolongate_add(h->h.tr[fine_level]->tl, fp64 != 0, coarse, fine, h->h.stream);
    ck_launches("prolongate");
  });
}

int gcmg_restrict_add(gcmg_handle* h, int fine_level, int fp64, const void* fine, void* coarse) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    if (fine_level < 1) throw Error(GCMG_ERR_ARG, "fine_level must be >= 1");
    check_level(h->h, fine_level);
    if (!h->h.tr[fine_level]) throw Error(GCMG_ERR_ARG, "no transfer into this level (the active mesh of local smoothing)");
    if (h->h.lev[fine_level - 1]->n() == 0 || h->h.lev[fine_level]->n() == 0) return;
    if (!coarse || !fine) throw Error(GCMG_ERR_ARG, "bad vectors");
    if (h->h.lev[fine_level - 1]->n())
      launch_restrict_add(h->h.tr[fine_level]->tl, fp64 != 0, fine, coarse, h->h.stream);
    ck_launches("restrict");
  });
}

int gcmg_coarse_solve(gcmg_handle* h, int fp64, const void* b, void* x) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    if (h->h.n0 && (!b || !x)) throw Error(GCMG_ERR_ARG, "bad vectors");
    if (h->h.n0) launch_coarse_solve(fp64 != 0, h->h.Ainv.as<double>(), h->h.n0, b, x, h->h.stream);
    ck_launches("coarse solve");
  });
}

int gcmg_vcycle(gcmg_handle* h, const double* b, double* x) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    if (h->h.lev.back()->n() == 0) return;
    if (!b || !x) throw Error(GCMG_ERR_ARG, "bad vectors");
    vcycle(h->h, b, x);
    ck_launches("vcycle");
  });
}

int gcmg_cg_solve(gcmg_handle* h, const double* b, double* x, double rtol, int maxit, gcmg_solve_stats* stats) {
  int status = GCMG_OK;
  int rc = guarded([&] {
    if (!h || !(rtol > 0) || maxit < 0) throw Error(GCMG_ERR_ARG, "bad arguments");
    Handle& H = h->h;
    const int top = (int)H.lev.size() - 1;
    const int64_t n = H.lev[top]->n();
    if (n == 0) {
      if (stats) *stats = gcmg_solve_stats{0, 0.0, 0.0, GCMG_OK};
      return;
    }
    if (!b || !x) throw Error(GCMG_ERR_ARG, "bad vectors");
    double* xi = H.cg_x.as<double>();
    double* r = H.cg_r.as<double>();
    double* p = H.cg_p.as<double>();
    double* q = H.cg_q.as<double>();
    double* z = H.cg_z.as<double>();
    double* S = H.scal.as<double>();
    cudaStream_t s = H.stream;
    gcmg_solve_stats st{0, 0.0, 0.0, GCMG_OK};
    launch_zero(true, xi, n, s);
    ck(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    const double nb = std::sqrt(dot_host(H, r, r, n));
    st.r0 = nb;
    if (nb == 0.0) {
      launch_zero(true, x, n, s);
      ck(cudaStreamSynchronize(s), "cg");
      if (stats) *stats = st;
      return;
    }
    // with an fp32 V-cycle (global coarsening) the update of r also writes r in
    // fp32 into the finest level's right-hand side, and the V-cycle's fp32
    // output z feeds r.z and p = z + beta p directly: the two casts of the
    // V-cycle's entry and exit drop out, bit for bit the same values
    LevelDev& F = *H.lev[top];
    float* r32 = (F.fp32 && !H.ls) ? F.b.as<float>() : nullptr;
    // operator half of an iteration: q = A p, alpha, x += alpha p, r -= alpha q, r.r
    auto op_half = [&] {
      vmult(H, top, true, p, q, GCMG_STAGE_CG_VMULT);
      const int pr = prof_begin(H, top, GCMG_STAGE_CG_VECTOR);
      launch_dot(p, q, n, H.scratch.as<double>(), S, 0, DOT_ALPHA, H.stream);
      launch_cg_update_xr(xi, r, p, q, S, n, H.scratch.as<double>(), S, H.stream, r32);
      prof_end(H, pr);
    };
    const bool flexible = any_learned(H);
    const bool fused = r32 && !flexible;
    vcycle(H, r, z);
    launch_dot(r, z, n, H.scratch.as<double>(), S, 0, DOT_STORE, s);  // rz
    ck(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    if (H.use_graphs && !H.g_a.exec) capture(H, H.g_a, op_half);
    double rr = nb * nb;
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
      if (H.use_graphs) {
        ck(cudaGraphLaunch(H.g_a.exec, s), "graph launch");
        note_launches((int)H.g_a.kernels);
      } else {
        op_half();
      }
      double hs[6];
      ck(cudaMemcpyAsync(hs, S, sizeof(hs), cudaMemcpyDeviceToHost, s), "scalars");
      ck(cudaStreamSynchronize(s), "cg");
      if (H.use_graphs) {  // one replay of each graph completed since the last read
        prof_graph(H, H.g_a);
        prof_graph(H, H.g_core);
      }
      if (!(hs[1] > 0.0) || std::isnan(hs[2])) {
        status = GCMG_ERR_BREAKDOWN;
        break;
      }
      rr = hs[2];
      if (std::sqrt(rr) <= rtol * nb) break;
      if (flexible) {  // r_{k+1} . z_k before z is overwritten
        const int pc = prof_begin(H, top, GCMG_STAGE_CG_VECTOR);
        launch_dot(r, z, n, H.scratch.as<double>(), S, 6, DOT_STORE, s);
        prof_end(H, pc);
      }
      if (fused) {  // F.b holds r in fp32 (written by the update of r)
        vcycle_core(H);
        const float* z32 = F.x.as<float>();
        const int pz = prof_begin(H, top, GCMG_STAGE_CG_VECTOR);
        launch_dot(r, z32, n, H.scratch.as<double>(), S, 0, DOT_BETA, s);
        launch_cg_update_p(p, z32, S, n, s);
        prof_end(H, pz);
        continue;
      }
      vcycle(H, r, z);
      const int pz = prof_begin(H, top, GCMG_STAGE_CG_VECTOR);
      launch_dot(r, z, n, H.scratch.as<double>(), S, 0, flexible ? DOT_BETA_FLEX : DOT_BETA, s);
      launch_cg_update_p(p, z, S, n, s);
      prof_end(H, pz);
    }
    if (it > maxit) {
      it = maxit;
      status = GCMG_ERR_NOT_CONVERGED;
    }
    ck(cudaMemcpyAsync(x, xi, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    st.iterations = it;
    st.rel_residual = std::sqrt(rr) / nb;
    st.status = status;
    ck(cudaStreamSynchronize(s), "cg");
    ck_launches("cg");
    if (stats) *stats = st;
  });
  if (rc != GCMG_OK) return rc;
  if (status != GCMG_OK) g_err = status == GCMG_ERR_BREAKDOWN ? "CG breakdown" : "CG did not converge";
  return status;
}

int gcmg_level_cells(const gcmg_handle* h, int level, int32_t* lijk) {
  return guarded([&] {
    if (!h || !lijk) throw Error(GCMG_ERR_ARG, "null argument");
    check_level(h->h, level);
    const auto& cells = h->h.lev[level]->host.cells;
    for (size_t c = 0; c < cells.size(); ++c) {
      lijk[4 * c] = cells[c].l;
      lijk[4 * c + 1] = cells[c].i;
      lijk[4 * c + 2] = cells[c].j;
      lijk[4 * c + 3] = cells[c].k;
    }
  });
}

int gcmg_cell_gather(gcmg_handle* h, int level, const double* x, int64_t n_cells, const int32_t* cells,
                     double* out) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    LevelDev& L = *h->h.lev[level];
    if (n_cells < 0 || (!cells && n_cells > (int64_t)L.host.cells.size())) throw Error(GCMG_ERR_ARG, "bad cell count");
    if (n_cells == 0) return;
    if (!x || !out) throw Error(GCMG_ERR_ARG, "bad vectors");
    launch_cell_gather(L.host.k, x, cells, n_cells, L.gstart.as<int32_t>(), L.meta.as<CellMeta>(), out,
                       h->h.stream);
    ck_launches("cell gather");
  });
}

int gcmg_mlp_samples(gcmg_handle* h, int level, const double* b, const double* x, const double* xstar,
                     int64_t n_cells, const int32_t* cells, float* X, float* T, float* W) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    Handle& H = h->h;
    LevelDev& L = *H.lev[level];
    if (n_cells < 0 || (!cells && n_cells > (int64_t)L.host.cells.size())) throw Error(GCMG_ERR_ARG, "bad cell count");
    if (n_cells == 0 || L.n() == 0) return;
    if (!b || !x || !X || (T && !xstar)) throw Error(GCMG_ERR_ARG, "bad vectors");
    const int k = L.host.k, n3 = (k + 1) * (k + 1) * (k + 1);
    const int64_t n = L.n();
    double* r = L.w64a.as<double>();
    double* e = L.w64b.as<double>();
    vmult(H, level, true, x, r);  // r = b - A x
    launch_residual(true, r, b, r, n, H.stream);
    if (T) {  // e = xstar - x
      ck(cudaMemcpyAsync(e, xstar, n * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
      launch_axpy(true, e, x, -1.0, n, H.stream);
    }
    DevBuf R, E, D;
    R.alloc((size_t)n_cells * n3 * sizeof(double));
    D.alloc((size_t)n_cells * n3 * sizeof(double));
    if (T) E.alloc((size_t)n_cells * n3 * sizeof(double));
    const int32_t* gs = L.gstart.as<int32_t>();
    const CellMeta* meta = L.meta.as<CellMeta>();
    launch_cell_gather(k, r, cells, n_cells, gs, meta, R.as<double>(), H.stream);
    launch_cell_gather(k, L.diag64.as<double>(), cells, n_cells, gs, meta, D.as<double>(), H.stream);
    if (T) launch_cell_gather(k, e, cells, n_cells, gs, meta, E.as<double>(), H.stream);
    launch_mlp_samples(R.as<double>(), T ? E.as<double>() : nullptr, D.as<double>(), cells, n_cells, n3, meta,
                       L.cl.dom, mean_ref_diag(k), X, T, W, H.stream);
    ck(cudaStreamSynchronize(H.stream), "samples");  // the temporaries are freed on return
  });
}

static void check_q4_net(const LevelDev& L, const gcmg_mlp* net) {
  if (!net) throw Error(GCMG_ERR_ARG, "null network");
  if (L.host.k != 4) throw Error(GCMG_ERR_ARG, "the learned smoother runs on Q4 levels only");
  const MlpNet& N = net->net;
  if (N.n_in != 250 || N.n_h != 128 || N.n_out != 125)
    throw Error(GCMG_ERR_ARG, "the Q4 learned smoother needs a 250-128-128-125 network");
}

int gcmg_mlp_correct(gcmg_handle* h, int level, const gcmg_mlp* net, int fp64, const void* r, void* x) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    LevelDev& L = *h->h.lev[level];
    check_q4_net(L, net);
    if (L.n() == 0) return;
    if (!r || !x) throw Error(GCMG_ERR_ARG, "bad vectors");
    Handle& H = h->h;
    if (L.mlp_call_version != net->net.version) {
      mlp_prepare(H, level, net, L.mlp_image_call, L.mlp_dproj_call);
      L.mlp_call_version = net->net.version;
    }
    mlp_correct(H, level, L.mlp_image_call.p, L.mlp_dproj_call.as<float>(), fp64 != 0, r, x);
  });
}

int gcmg_wait_timeouts(unsigned int* count, int reset) {
  return guarded([&] {
    if (!count) throw Error(GCMG_ERR_ARG, "null count");
    const unsigned int n = wait_timeouts(reset != 0);
    if (n == ~0u) throw Error(GCMG_ERR_CUDA, "reading the wait counter");
    *count = n;
  });
}

int gcmg_set_smoother(gcmg_handle* h, int level, int kind, const gcmg_mlp* net) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    if (level < 1) throw Error(GCMG_ERR_ARG, "level 0 is solved exactly");
    if (kind < GCMG_SMOOTHER_CHEBYSHEV || kind > GCMG_SMOOTHER_MLP_REPLACE) throw Error(GCMG_ERR_ARG, "unknown smoother");
    if (h->h.ls) throw Error(GCMG_ERR_ARG, "the learned smoother is not available with local smoothing");
    Handle& H = h->h;
    LevelDev& L = *H.lev[level];
    if (kind != GCMG_SMOOTHER_CHEBYSHEV) {
      if (L.cl.coef) throw Error(GCMG_ERR_ARG, "the learned smoother assumes a unit coefficient");
      if (L.cl.geom) throw Error(GCMG_ERR_ARG, "the learned smoother assumes Cartesian cells");
      check_q4_net(L, net);
      mlp_prepare(H, level, net, L.mlp_image, L.mlp_dproj);
      if (!H.lscratch.p) H.lscratch.alloc((2 * DOT_BLOCKS + 2) * sizeof(double));
    }
    L.smoother = kind;
    H.g_core.reset();
  });
}

int gcmg_set_coefficient(gcmg_handle* h, int values_per_cell, const double* nu) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    Handle& H = h->h;
    LevelDev& F = *H.lev.back();
    const int k = F.cl.k;
    const int n3 = (k + 1) * (k + 1) * (k + 1);
    const int64_t ncf = (int64_t)F.host.cells.size();
    if (values_per_cell != 1 && values_per_cell != n3) throw Error(GCMG_ERR_ARG, "values_per_cell must be 1 or (k+1)^3");
    if (ncf > 0 && !nu) throw Error(GCMG_ERR_ARG, "null coefficient");
    if (any_learned(H)) throw Error(GCMG_ERR_ARG, "the learned smoother assumes a unit coefficient");
    if (H.ls) throw Error(GCMG_ERR_ARG, "a coefficient is not available with local smoothing");
    if (H.in_batch) throw Error(GCMG_ERR_ARG, "the problems of a batch keep their set-up");
    // validate the input before touching the level data
    {
      const int64_t n = ncf * values_per_cell;
      int* bad = H.scratch.as<int>();
      ck(cudaMemsetAsync(bad, 0, sizeof(int), H.stream), "memset");
      launch_check_positive(nu, n, bad, H.stream);
      int hb = 0;
      ck(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, H.stream), "copy");
      ck(cudaStreamSynchronize(H.stream), "sync");
      if (hb) throw Error(GCMG_ERR_ARG, "coefficient values must be positive and finite");
    }
    const int nl = (int)H.lev.size();
    for (int l = 0; l < nl; ++l) {
      LevelDev& L = *H.lev[l];
      if (!L.coef.p) L.coef.alloc(std::max<size_t>(1, L.host.cells.size()) * sizeof(double));
      L.cl.coef = L.coef.as<double>();
    }
    for (int l = 1; l < nl; ++l)
      if (H.tr[l]) H.tr[l]->tl.coarse = H.lev[l - 1]->cl;
    if (values_per_cell == 1)
      ck(cudaMemcpyAsync(F.coef.p, nu, ncf * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
    else
      launch_coef_harmonic(k, ncf, nu, F.coef.as<double>(), H.stream);
    for (int l = nl - 2; l >= 0; --l) {
      const TransferDev& T = *H.tr[l + 1];
      launch_coef_coarsen((int)H.lev[l]->host.cells.size(), T.fine_of.as<int32_t>(), T.refined.as<uint8_t>(),
                          H.lev[l + 1]->coef.as<double>(), H.lev[l]->coef.as<double>(), H.stream);
    }
    ck_launches("coefficient");
    setup_numerics(H);
    ck(cudaStreamSynchronize(H.stream), "coefficient");
  });
}

int gcmg_set_geometry(gcmg_handle* h, int kind, double eps) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    Handle& H = h->h;
    if (kind != 0 && kind != GCMG_GEOM_WARP) throw Error(GCMG_ERR_ARG, "unknown geometry");
    if (!std::isfinite(eps)) throw Error(GCMG_ERR_ARG, "eps must be finite");
    if (any_learned(H)) throw Error(GCMG_ERR_ARG, "the learned smoother assumes Cartesian cells");
    if (H.in_batch) throw Error(GCMG_ERR_ARG, "the problems of a batch keep their set-up");
    if (kind == GCMG_GEOM_WARP) {
      // the map must be invertible on the domain: det J_Phi > 0 on a 33^3 lattice
      const double lo = H.lev.back()->host.lo, hi = H.lev.back()->host.hi;
      double dmin = 1e300;
      for (int a = 0; a <= 32; ++a)
        for (int b = 0; b <= 32; ++b)
          for (int c = 0; c <= 32; ++c) {
            const double x = lo + (hi - lo) * a / 32, y = lo + (hi - lo) * b / 32, z = lo + (hi - lo) * c / 32;
            const double det = 1.0 - eps * eps * (x * x + 0.5 * y * y + 2.0 * z * z) + 2.0 * eps * eps * eps * x * y * z;
            dmin = std::min(dmin, det);
          }
      if (!(dmin > 0.05)) throw Error(GCMG_ERR_ARG, "the warp folds the domain (det J <= 0.05): reduce eps");
    }
    const int nl = (int)H.lev.size();
    if (kind)
      for (int l = 0; l < nl; ++l) {
        const CellLaunch& c = H.lev[l]->cl;
        if (cell_smem_bytes(c.k, true, c.tc, c.max_local, true) > 227 * 1024)
          throw Error(GCMG_ERR_ARG, "tiles too large for the mapped operator's shared memory (use tile_cells <= 32)");
      }
    for (int l = 0; l < nl; ++l) {
      H.lev[l]->cl.geom = kind;
      H.lev[l]->cl.geps = kind ? eps : 0.0;
    }
    for (int l = 1; l < nl; ++l)
      if (H.tr[l]) H.tr[l]->tl.coarse = H.lev[l - 1]->cl;
    setup_numerics(H);
    ck(cudaStreamSynchronize(H.stream), "geometry");
  });
}

int gcmg_get_coefficient(gcmg_handle* h, int level, double* nu) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    check_level(h->h, level);
    Handle& H = h->h;
    LevelDev& L = *H.lev[level];
    const size_t nc = L.host.cells.size();
    if (nc && !nu) throw Error(GCMG_ERR_ARG, "bad vector");
    if (L.cl.coef) {
      ck(cudaMemcpyAsync(nu, L.coef.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "copy");
    } else {
      std::vector<double> one(nc, 1.0);
      ck(cudaMemcpyAsync(nu, one.data(), nc * sizeof(double), cudaMemcpyHostToDevice, H.stream), "copy");
    }
    ck(cudaStreamSynchronize(H.stream), "copy");
  });
}

int gcmg_quadrature_points(gcmg_handle* h, double* xyz) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    Handle& H = h->h;
    LevelDev& F = *H.lev.back();
    const int64_t nc = (int64_t)F.host.cells.size();
    if (nc && !xyz) throw Error(GCMG_ERR_ARG, "bad vector");
    launch_quadrature_points(F.cl, nc, xyz, H.stream);
    ck(cudaStreamSynchronize(H.stream), "quadrature points");
  });
}

int gcmg_point_values(const double* xyz, int64_t n, uint64_t seed, double* out) {
  return guarded([&] {
    if (n < 0 || (n && (!xyz || !out))) throw Error(GCMG_ERR_ARG, "bad arguments");
    for (int64_t i = 0; i < n; ++i) out[i] = point_value(xyz + 3 * i, seed);
  });
}

int gcmg_set_graphs(gcmg_handle* h, int on) {
  return guarded([&] {
    if (!h) throw Error(GCMG_ERR_ARG, "null handle");
    h->h.use_graphs = on != 0;
    h->h.g_core.reset();
    h->h.g_a.reset();
  });
}

}  // extern "C"
