// Measured arithmetic peak of the CUDA cores (not of the tensor cores): the
// denominator of the ALU fractions the benchmark reports beside the HBM
// fractions.  Every thread runs NCH independent chains of fused multiply-adds
// x <- x a + b; the grid fills every SM with 2048 threads, so the FMA pipes,
// not the chains' latency, bound the rate.  FLOP/s counts a multiply-add as
// two operations.
#include <cuda_runtime.h>

#include "host.h"
#include "kernels.h"

namespace gcmg {
namespace {

constexpr int NCH = 8;    // independent chains per thread
constexpr int PT = 256;   // threads per block

template <typename T>
__global__ void __launch_bounds__(PT) fma_chains(T* out, int iters, T a, T b) {
  T x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c];
  if (s == (T)-1) out[blockIdx.x] = s;  // never true: keeps the chains alive
}

template <typename T>
double run(int n_sm, int iters, cudaStream_t s, T* out) {
  const int blocks = n_sm * (2048 / PT);
  cudaEvent_t e0, e1;
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  fma_chains<T><<<blocks, PT, 0, s>>>(out, iters / 16, (T)0.999999, (T)1e-7);  // warm-up
  ck(cudaEventRecord(e0, s), "event");
  fma_chains<T><<<blocks, PT, 0, s>>>(out, iters, (T)0.999999, (T)1e-7);
  ck(cudaEventRecord(e1, s), "event");
  ck(cudaEventSynchronize(e1), "event");
  float ms = 0.f;
  ck(cudaEventElapsedTime(&ms, e0, e1), "event");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ck_launches("fma peak");
  return 2.0 * NCH * (double)iters * blocks * PT / (ms * 1e-3) / 1e12;
}

}  // namespace
}  // namespace gcmg

using namespace gcmg;

extern "C" int gcmg_fma_peak(int fp64, int iters, void* stream, double* tflops) {
  return guarded([&] {
    if (!tflops || iters < 16) throw Error(GCMG_ERR_ARG, "bad arguments");
    int dev = 0, n_sm = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    ck(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf out;
    out.alloc((size_t)n_sm * (2048 / PT) * sizeof(double));
    *tflops = fp64 ? run<double>(n_sm, iters, s, out.as<double>()) : run<float>(n_sm, iters, s, out.as<float>());
  });
}
