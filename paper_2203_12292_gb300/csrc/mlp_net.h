// The per-cell network of the learned smoother (host object): fp32 master
// parameters and Adam moments on the device, batch work buffers, and the
// forward / backward / training sequences of kernels_mlp.cu launches.
#pragma once

#include <cstdint>

#include "host.h"

namespace gcmg {

struct MlpNet {
  int n_in = 0, n_h = 0, n_out = 0;
  int64_t n_params = 0;
  DevBuf params, grad, m, v;
  int64_t steps = 0;  // Adam steps taken since the parameters were set
  // process-wide unique tag of the current parameter values (new on creation,
  // gcmg_mlp_set_params and every Adam step), so that derived data (the
  // inference weight image) is rebuilt only when the parameters changed
  uint64_t version = 0;
  void touch();
  // work buffers for `cap` rows
  int64_t cap = 0;
  DevBuf Xb, Tb, Wb, Z1, H1, Z2, H2, Y, dY, dA, dB, loss;

  // offsets of W1, b1, W2, b2, W3, b3 in the packed parameter vector
  int64_t oW1() const { return 0; }
  int64_t ob1() const { return (int64_t)n_h * n_in; }
  int64_t oW2() const { return ob1() + n_h; }
  int64_t ob2() const { return oW2() + (int64_t)n_h * n_h; }
  int64_t oW3() const { return ob2() + n_h; }
  int64_t ob3() const { return oW3() + (int64_t)n_out * n_h; }

  void reserve(int64_t rows);
  // Y = network(X) for `rows` rows (rows <= cap); keeps Z1, H1, Z2, H2
  void forward(const float* X, int64_t rows, float* Y, cudaStream_t s);
  // loss and gradient (into `grad`) of sum w |Y - T|^2 / (2 sum w) over B
  // rows (W null: all weights 1)
  void gradient(const float* X, const float* T, const float* W, int B, float* loss, cudaStream_t s);
  void adam(float lr, cudaStream_t s);
};

}  // namespace gcmg

struct gcmg_mlp {
  gcmg::MlpNet net;
};
