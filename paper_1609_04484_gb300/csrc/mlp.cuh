// The learned coarse correction's network (bfloat16 tensor-core GEMMs with
// float accumulation, float master parameters, Adam): see mlp.cu.
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace stokes {
namespace mlp {

// Flat parameter layout W1 [n_in x hidden], b1, W2 [hidden x hidden], b2,
// W3 [hidden x n_out], b3 (row-major); in_p / out_p: n_in / n_out padded to
// multiples of 16 for the GEMMs.
struct Layout {
  int n_in, hidden, n_out, in_p, out_p;
  int64_t oW1, ob1, oW2, ob2, oW3, ob3, total;
};

struct Net {
  Layout L{};
  DevBuf<float> p, m, v, grad;           // master parameters, Adam moments, gradient (flat)
  DevBuf<__nv_bfloat16> w1, w2, w3;      // padded bf16 weights
  DevBuf<float> b1, b2, b3;              // padded float biases
  DevBuf<__nv_bfloat16> xb, h1, h2, dy, dh1, dh2;
  DevBuf<float> y;                       // output [rows_p][out_p]
  DevBuf<double> part, loss;
  int64_t rows_p = 0;
  int step = 0;

  Net(int n_in, int hidden, int n_out);
  int64_t n_params() const;
  void init(const float* host_params, cudaStream_t s);       // zero Adam moments, step 0
  void set_params(const float* params, bool device, cudaStream_t s);
  void pack(cudaStream_t s);                                   // bf16 / padded copies of p
  void reserve(int64_t rows);
  // y = net(standardise(x)); x [rows][n_in] float (device); mean/stdv may be null
  void forward(const float* x, int64_t rows, const float* mean, const float* stdv, cudaStream_t s);
  // loss (device scalar) and grad for targets t and mask [rows][n_out]
  void loss_and_grad(const float* x, const float* t, const float* mask, int64_t rows, double count,
                     const float* mean, const float* stdv, cudaStream_t s);
  // one Adam step with gradient g (device; null: the stored grad)
  void adam(const float* g, double lr, cudaStream_t s);
};

}  // namespace mlp
}  // namespace stokes
