// Training and inference sequences of the learned smoother's network
// (forward pass, backward pass by the chain rule, Adam) and its C ABI.
// The network and the update rule are an extension outside the paper: the
// paper smooths with Chebyshev around point Jacobi (Sec. 3.3).
#include <atomic>
#include <algorithm>
#include <cmath>
#include <memory>

#include "gcmg.h"
#include "kernels.h"
#include "mlp_net.h"

namespace gcmg {

void MlpNet::reserve(int64_t rows) {
  if (rows <= cap) return;
  const int64_t w = std::max(n_h, std::max(n_in, n_out));
  Xb.alloc(rows * n_in * sizeof(float));
  Tb.alloc(rows * n_out * sizeof(float));
  Wb.alloc(rows * sizeof(float));
  Z1.alloc(rows * n_h * sizeof(float));
  H1.alloc(rows * n_h * sizeof(float));
  Z2.alloc(rows * n_h * sizeof(float));
  H2.alloc(rows * n_h * sizeof(float));
  Y.alloc(rows * n_out * sizeof(float));
  dY.alloc(rows * n_out * sizeof(float));
  dA.alloc(rows * w * sizeof(float));
  dB.alloc(rows * w * sizeof(float));
  if (!loss.p) loss.alloc(sizeof(float));
  cap = rows;
}

// C = A W^T + b for row-major A (rows x k) and W (n x k)
static void linear(const float* A, int64_t rows, int k, const float* W, const float* b, int n, float* C,
                   cudaStream_t s) {
  GemmArgs g{A, k, 1, W, 1, k, C, n, b, (int)rows, n, k};
  launch_gemm_bf16(g, s);
}

void MlpNet::forward(const float* X, int64_t rows, float* Yout, cudaStream_t s) {
  const float* P = params.as<float>();
  linear(X, rows, n_in, P + oW1(), P + ob1(), n_h, Z1.as<float>(), s);
  launch_gelu(Z1.as<float>(), H1.as<float>(), rows * n_h, s);
  linear(H1.as<float>(), rows, n_h, P + oW2(), P + ob2(), n_h, Z2.as<float>(), s);
  launch_gelu(Z2.as<float>(), H2.as<float>(), rows * n_h, s);
  linear(H2.as<float>(), rows, n_h, P + oW3(), P + ob3(), n_out, Yout, s);
}

void MlpNet::gradient(const float* X, const float* T, const float* W, int B, float* loss_out, cudaStream_t s) {
  const float* P = params.as<float>();
  float* G = grad.as<float>();
  forward(X, B, Y.as<float>(), s);
  launch_mse(Y.as<float>(), T, W, dY.as<float>(), B, n_out, loss_out, s);
  // layer 3: gW3 = dY^T H2, gb3 = sum dY, dH2 = dY W3
  launch_gemm_bf16(GemmArgs{dY.as<float>(), 1, n_out, H2.as<float>(), n_h, 1, G + oW3(), n_h, nullptr, n_out, n_h, B}, s);
  launch_colsum(dY.as<float>(), B, n_out, G + ob3(), s);
  launch_gemm_bf16(GemmArgs{dY.as<float>(), n_out, 1, P + oW3(), n_h, 1, dA.as<float>(), n_h, nullptr, B, n_h, n_out}, s);
  launch_gelu_bwd(dA.as<float>(), Z2.as<float>(), dB.as<float>(), (int64_t)B * n_h, s);  // dZ2
  // layer 2: gW2 = dZ2^T H1, gb2 = sum dZ2, dH1 = dZ2 W2
  launch_gemm_bf16(GemmArgs{dB.as<float>(), 1, n_h, H1.as<float>(), n_h, 1, G + oW2(), n_h, nullptr, n_h, n_h, B}, s);
  launch_colsum(dB.as<float>(), B, n_h, G + ob2(), s);
  launch_gemm_bf16(GemmArgs{dB.as<float>(), n_h, 1, P + oW2(), n_h, 1, dA.as<float>(), n_h, nullptr, B, n_h, n_h}, s);
  launch_gelu_bwd(dA.as<float>(), Z1.as<float>(), dB.as<float>(), (int64_t)B * n_h, s);  // dZ1
  // layer 1: gW1 = dZ1^T X, gb1 = sum dZ1
  launch_gemm_bf16(GemmArgs{dB.as<float>(), 1, n_h, X, n_in, 1, G + oW1(), n_in, nullptr, n_h, n_in, B}, s);
  launch_colsum(dB.as<float>(), B, n_h, G + ob1(), s);
}

void MlpNet::touch() {
  static std::atomic<uint64_t> counter{0};
  version = ++counter;
}

void MlpNet::adam(float lr, cudaStream_t s) {
  touch();
  ++steps;
  const float bc1 = (float)(1.0 - std::pow((double)MLP_BETA1, (double)steps));
  const float bc2 = (float)(1.0 - std::pow((double)MLP_BETA2, (double)steps));
  launch_adam(params.as<float>(), grad.as<float>(), m.as<float>(), v.as<float>(), n_params, lr, bc1, bc2, s);
}

}  // namespace gcmg

using namespace gcmg;

static cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

extern "C" {

int gcmg_mlp_create(int n_in, int n_hidden, int n_out, gcmg_mlp** out) {
  return guarded([&] {
    if (!out || n_in <= 0 || n_hidden <= 0 || n_out <= 0 || n_in > 4096 || n_hidden > 4096 || n_out > 4096)
      throw Error(GCMG_ERR_ARG, "bad network size");
    auto net = std::make_unique<gcmg_mlp>();
    MlpNet& N = net->net;
    N.n_in = n_in;
    N.n_h = n_hidden;
    N.n_out = n_out;
    N.n_params = N.ob3() + n_out;
    const size_t b = N.n_params * sizeof(float);
    N.params.alloc(b);
    N.grad.alloc(b);
    N.m.alloc(b);
    N.v.alloc(b);
    ck(cudaMemset(N.params.p, 0, b), "memset");
    ck(cudaMemset(N.grad.p, 0, b), "memset");
    ck(cudaMemset(N.m.p, 0, b), "memset");
    ck(cudaMemset(N.v.p, 0, b), "memset");
    N.touch();
    *out = net.release();
  });
}

void gcmg_mlp_destroy(gcmg_mlp* net) { delete net; }

int gcmg_mlp_num_params(const gcmg_mlp* net, int64_t* n) {
  return guarded([&] {
    if (!net || !n) throw Error(GCMG_ERR_ARG, "null argument");
    *n = net->net.n_params;
  });
}

int gcmg_mlp_set_params(gcmg_mlp* net, const float* params, void* stream) {
  return guarded([&] {
    if (!net || !params) throw Error(GCMG_ERR_ARG, "null argument");
    MlpNet& N = net->net;
    const size_t b = N.n_params * sizeof(float);
    cudaStream_t s = as_stream(stream);
    ck(cudaMemcpyAsync(N.params.p, params, b, cudaMemcpyDeviceToDevice, s), "copy");
    ck(cudaMemsetAsync(N.m.p, 0, b, s), "memset");
    ck(cudaMemsetAsync(N.v.p, 0, b, s), "memset");
    N.steps = 0;
    N.touch();
  });
}

int gcmg_mlp_get_params(const gcmg_mlp* net, float* params, void* stream) {
  return guarded([&] {
    if (!net || !params) throw Error(GCMG_ERR_ARG, "null argument");
    ck(cudaMemcpyAsync(params, net->net.params.p, net->net.n_params * sizeof(float), cudaMemcpyDeviceToDevice,
                       as_stream(stream)),
       "copy");
  });
}

int gcmg_mlp_forward(gcmg_mlp* net, const float* X, int64_t n, float* Y, void* stream) {
  return guarded([&] {
    if (!net || n < 0 || (n && (!X || !Y))) throw Error(GCMG_ERR_ARG, "bad arguments");
    MlpNet& N = net->net;
    cudaStream_t s = as_stream(stream);
    const int64_t chunk = 65536;
    N.reserve(std::min(n, chunk));
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
      const int64_t rows = std::min(chunk, n - r0);
      N.forward(X + r0 * N.n_in, rows, Y + r0 * N.n_out, s);
    }
    ck_launches("mlp forward");
  });
}

int gcmg_mlp_gradient(gcmg_mlp* net, const float* X, const float* T, const float* W, int64_t n, float* grad,
                      float* loss, void* stream) {
  return guarded([&] {
    if (!net || !X || !T || !grad || n <= 0 || n > (1 << 20)) throw Error(GCMG_ERR_ARG, "bad arguments");
    MlpNet& N = net->net;
    cudaStream_t s = as_stream(stream);
    N.reserve(n);
    N.gradient(X, T, W, (int)n, loss ? loss : N.loss.as<float>(), s);
    ck(cudaMemcpyAsync(grad, N.grad.p, N.n_params * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy");
    ck_launches("mlp gradient");
  });
}

int gcmg_mlp_train(gcmg_mlp* net, const float* X, const float* T, const float* W, int64_t n_samples,
                   const int32_t* order, int64_t n_order, int batch, float lr, float* losses, void* stream) {
  return guarded([&] {
    if (!net || !X || !T || !order || n_samples <= 0 || batch <= 0 || batch > 65536 || n_order < batch ||
        !(lr > 0.0f))
      throw Error(GCMG_ERR_ARG, "bad arguments");
    MlpNet& N = net->net;
    cudaStream_t s = as_stream(stream);
    N.reserve(batch);
    const int64_t steps = n_order / batch;
    for (int64_t st = 0; st < steps; ++st) {
      const int32_t* idx = order + st * batch;
      launch_gather_rows(X, N.n_in, idx, batch, N.Xb.as<float>(), s);
      launch_gather_rows(T, N.n_out, idx, batch, N.Tb.as<float>(), s);
      if (W) launch_gather_rows(W, 1, idx, batch, N.Wb.as<float>(), s);
      N.gradient(N.Xb.as<float>(), N.Tb.as<float>(), W ? N.Wb.as<float>() : nullptr, batch,
                 losses ? losses + st : N.loss.as<float>(), s);
      N.adam(lr, s);
    }
    ck_launches("mlp train");
  });
}

}  // extern "C"
