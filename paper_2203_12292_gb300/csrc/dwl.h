// Device work list: the launches of a solve recorded as operations that one
// persistent kernel executes (kernels_dwl.cu), instead of being launched.
//
// While a recorder is installed on the calling host thread, launch_pdl does
// not launch: it appends {operation, virtual grid, block, shared memory,
// packed arguments} to the recorder.  The operation is looked up by the
// kernel's address in a registry that each kernel translation unit fills for
// the kernels the persistent kernel can run; the persistent kernel runs the
// same kernel body, compiled as a device function, once per virtual block
// ("item") with blockIdx/gridDim replaced by the item and the item count.
//
// Arguments are packed like the members of a C struct of the kernel's
// parameter types in order (each at the next offset aligned for its type);
// host and device compute the offsets with the same constexpr function.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

namespace gcmg {

constexpr int DWL_ARG_BYTES = 256;  // largest packed argument list
constexpr int DWL_OP_CHECK = 100000;  // the CG loop test (recorded from cg_check_kernel)

template <typename... Ts>
__host__ __device__ constexpr size_t dwl_offset(size_t i) {
  constexpr size_t n = sizeof...(Ts);
  constexpr size_t sz[n + 1] = {sizeof(Ts)..., 0};
  constexpr size_t al[n + 1] = {alignof(Ts)..., 1};
  size_t o = 0;
  for (size_t j = 0; j < i; ++j) o = (o + al[j] - 1) / al[j] * al[j] + sz[j];
  return (o + al[i] - 1) / al[i] * al[i];
}
template <typename... Ts>
__host__ __device__ constexpr size_t dwl_size() {
  return dwl_offset<Ts...>(sizeof...(Ts));
}
template <typename... Ts>
constexpr size_t dwl_args_size(void (*)(Ts...)) {
  return dwl_size<Ts...>();
}

struct DwlOp {
  int32_t type;   // registry id (or DWL_OP_CHECK)
  int32_t items;  // virtual blocks
  int32_t block;  // threads of the recorded launch (<= BLOCK)
  int32_t smem;   // dynamic shared memory of the recorded launch
  int32_t prob;   // problem of a DWL_OP_CHECK
  int32_t pad[3];
  alignas(16) unsigned char args[DWL_ARG_BYTES];
};

constexpr int DWL_MAX_PROBS = 1024;  // problems of one persistent launch

// operations [pro, body) are the CG prologue, [body, epi) one CG iteration,
// [epi, end) the epilogue; a DWL_OP_CHECK ends the prologue and the body
struct DwlProb {
  int32_t pro, body, epi, end;
};

struct DwlParams {
  const DwlOp* ops;
  const DwlProb* probs;
  int np;
  int* go;              // per problem: the last loop test passed
  unsigned* bar;        // grid barrier: arrivals, generation (zero at launch)
  int* status;          // [0]: 0, 1 barrier wait gave up, 2 step bound reached; [1]: steps taken
  long long max_steps;  // bound on the schedule's length
  unsigned spin_limit;  // polls of a grid-barrier wait before it gives up
  int absent_cta;       // test of the bounded waits: this CTA leaves before the first barrier (-1: none)
};

// CTAs of the persistent kernel with `smem` bytes of dynamic shared memory
// (all resident at once), -1 if it cannot run
int dwl_grid(size_t smem, int n_sm);
cudaError_t launch_dwl(const DwlParams& P, int grid, size_t smem, cudaStream_t s);
void upload_tables_dwl();
void dwl_register_cell();
void dwl_register_transfer();
void dwl_register_vec();

struct DwlRecorder {
  std::vector<DwlOp> ops;
};

// the recorder of the calling host thread (null: launches run)
DwlRecorder*& dwl_recorder();
inline bool dwl_recording() { return dwl_recorder() != nullptr; }

// registry of the kernels the persistent kernel runs: id and packed size
void dwl_register(const void* kernel, int id, size_t arg_bytes);
// a registered grid-stride kernel runs with `factor` times fewer virtual
// blocks (its results do not depend on the grid)
void dwl_set_coarsen(const void* kernel, int factor);
// a registered kernel without block barriers, which may be recorded with
// fewer than 256 threads (the others must be launched with exactly 256)
void dwl_set_serial(const void* kernel);
// id of a registered kernel, -1 when absent; *bytes its packed size, *coarsen
// its factor, *serial whether it may run on fewer threads
int dwl_lookup(const void* kernel, size_t* bytes, int* coarsen, bool* serial);
// fills the registry (once per process)
void dwl_register_all();

template <typename... KArgs, size_t... I>
void dwl_pack(unsigned char* buf, std::index_sequence<I...>, const KArgs&... a) {
  (std::memcpy(buf + dwl_offset<KArgs...>(I), &a, sizeof(KArgs)), ...);
}

// the recording half of launch_pdl; false when the kernel cannot be recorded
template <typename... KArgs>
bool dwl_record(const void* kernel, unsigned grid, unsigned block, size_t smem, const KArgs&... a) {
  size_t bytes = 0;
  int coarsen = 1;
  bool serial = false;
  const int id = dwl_lookup(kernel, &bytes, &coarsen, &serial);
  if (id < 0 || bytes != dwl_size<KArgs...>() || bytes > (size_t)DWL_ARG_BYTES) return false;
  if (serial ? (block > 256u) : (block != 256u)) return false;
  DwlOp op{};
  op.type = id;
  op.items = (int32_t)((grid + coarsen - 1) / coarsen);
  op.block = (int32_t)block;
  op.smem = (int32_t)smem;
  op.prob = -1;
  dwl_pack<KArgs...>(op.args, std::index_sequence_for<KArgs...>{}, a...);
  dwl_recorder()->ops.push_back(op);
  return true;
}

// Kernels the persistent kernel runs, per translation unit, in id order: the
// fp32 V-cycle (line-parallel operators, halo passes, transfers, Chebyshev,
// residual, coarse solve) and the fp64 CG around it.  Each entry is a
// parenthesised kernel.  Kernels with block < 256 run on that many threads
// and must not synchronise the block (only the SERIAL list).
#define GCMG_DWL_CELL(X)                                                                            \
  X((vmult_lines<1, float, 1>)) X((vmult_lines<2, float, 1>)) X((vmult_lines<2, float, 2>))         \
  X((vmult_lines<3, float, 1>)) X((vmult_lines<3, float, 2>)) X((vmult_lines<4, float, 1>))         \
  X((vmult_lines<4, float, 2>)) X((vmult_lines<4, float, 4>)) X((vmult_lines_df<1>))                \
  X((vmult_lines_df<2>)) X((vmult_lines_df<3>)) X((vmult_lines_df<4>))                              \
  X((cell_kernel<1, float, MODE_VMULT, BLOCK>)) X((cell_kernel<2, float, MODE_VMULT, BLOCK>))       \
  X((cell_kernel<3, float, MODE_VMULT, BLOCK>)) X((cell_kernel<4, float, MODE_VMULT, BLOCK>))       \
  X((cell_kernel<1, double, MODE_VMULT, BLOCK>)) X((cell_kernel<2, double, MODE_VMULT, BLOCK>))     \
  X((cell_kernel<3, double, MODE_VMULT, BLOCK>)) X((cell_kernel<4, double, MODE_VMULT, BLOCK>))     \
  X((halo_add_kernel<float>)) X((halo_add_kernel<double>))
#define GCMG_DWL_TRANSFER(X)                                                                        \
  X((prolong_h<1, float>)) X((prolong_h<2, float>)) X((prolong_h<3, float>)) X((prolong_h<4, float>)) \
  X((restrict_h<1, float, 4>)) X((restrict_h<2, float, 4>)) X((restrict_h<3, float, 4>))            \
  X((restrict_h<4, float, 4>)) X((restrict_h<1, float, 8>)) X((restrict_h<2, float, 8>))            \
  X((restrict_h<3, float, 8>)) X((restrict_h<4, float, 8>)) X((prolong_p<2, float>))                \
  X((prolong_p<3, float>)) X((prolong_p<4, float>)) X((restrict_p<2, float>)) X((restrict_p<3, float>)) \
  X((restrict_p<4, float>))
#define GCMG_DWL_VEC(X)                                                                             \
  X((cast_kernel<float, double>)) X((cast_kernel<double, float>)) X((copy_kernel))                  \
  X((zero_kernel<float>)) X((zero_kernel<double>)) X((cheb_init_kernel<float>))                     \
  X((cheb_step_kernel<float, true>)) X((cheb_step_kernel<float, false>)) X((residual_kernel<float>)) \
  X((coarse_kernel<float>)) X((dot_partial_b<double>)) X((dot_partial_b<float>)) X((dot_final))     \
  X((cg_xr_b<false>)) X((cg_xr_b<true>)) X((cg_p_kernel<double>)) X((cg_p_kernel<float>))
#define GCMG_DWL_VEC_SERIAL(X) X((scalar_set_kernel)) X((cg_stats_kernel))

#define GCMG_DWL_COUNT(fn) +1
constexpr int DWL_BASE_CELL = 0;
constexpr int DWL_BASE_TRANSFER = DWL_BASE_CELL GCMG_DWL_CELL(GCMG_DWL_COUNT);
constexpr int DWL_BASE_VEC = DWL_BASE_TRANSFER GCMG_DWL_TRANSFER(GCMG_DWL_COUNT);
constexpr int DWL_BASE_SERIAL = DWL_BASE_VEC GCMG_DWL_VEC(GCMG_DWL_COUNT);
constexpr int DWL_N_OPS = DWL_BASE_SERIAL GCMG_DWL_VEC_SERIAL(GCMG_DWL_COUNT);

}  // namespace gcmg
