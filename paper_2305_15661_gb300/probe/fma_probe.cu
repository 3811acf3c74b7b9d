// FMA throughput probe used by the benchmark to measure the FP64 and FP32
// ALU peaks of the GPU it runs on (the roofline denominators of the element
// kernels). Each thread runs 8 independent FMA chains; the only memory access
// is one store per thread at the end.
#include <cuda_runtime.h>

namespace {

template <class T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <class T>
int run(int blocks, int threads, int iters, double* flops_per_s) {
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<blocks, threads>>>(out, iters / 10, (T)0.999, (T)0.001);  // warm-up
  cudaEventRecord(e0);
  fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return 2;
  *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return 0;
}

}  // namespace

extern "C" int fma_probe(int precision, int blocks, int threads, int iters, double* flops_per_s) {
  return precision == 0 ? run<double>(blocks, threads, iters, flops_per_s)
                        : run<float>(blocks, threads, iters, flops_per_s);
}
