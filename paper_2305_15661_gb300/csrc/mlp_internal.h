// The warm-start network's state, shared by the FP32 kernels (mlp.cu) and the
// tensor-core BF16 forward pass (mlp_tc.cu). Internal to the library.
#pragma once
#include <cuda_runtime.h>

#include <vector>

struct ift_mlp {
  int n_in = 0, width = 0, depth = 0, n_out = 0;
  cudaStream_t stream = nullptr;
  std::vector<int> lin, lout;      // per layer
  std::vector<size_t> woff, boff;  // parameter offsets
  size_t np = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  int cap = 0;                     // batch capacity of the work buffers
  std::vector<float*> A, Z, dA;    // per layer: input activations, pre-activations, gradients
  float *T = nullptr, *Y = nullptr, *dY = nullptr;
  double* loss_parts = nullptr;
  int* idx = nullptr;
  long adam_t = 0;
  std::vector<double> xm, xs, tm, ts;  // normalisation of inputs and targets (identity until trained)
  // buffers of the tensor-core BF16 forward pass (ift_mlp_predict_bf16), grown on demand
  float *tc_x = nullptr, *tc_y = nullptr;
  int* tc_status = nullptr;
  long long tc_cap = 0;
  unsigned char* tc_wpk = nullptr;  // BF16 operand images of the weights of layers 1..
  size_t tc_wpk_bytes = 0;
  int layers() const { return (int)lin.size(); }
};
