// Throughput probes used by the benchmark to measure the FP64 and FP32 ALU
// peaks of the GPU it runs on (the roofline denominators of the element
// kernels), and the FP64 tensor-core rate (mma.sync m8n8k4 with FP64 operands
// and accumulators) to compare with the FP64 FMA pipe. Each thread runs 8
// independent FMA chains, or each warp 4 independent MMA accumulator chains; the
// only memory access is one store per thread at the end.
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

__global__ void dmma_chains(double* out, int iters) {
  const double a = 1.0 + 1e-3 * (threadIdx.x & 31), b = 1e-3;
  double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0, c4 = 0.0, c5 = 0.0, c6 = 0.0, c7 = 0.0;
  for (int i = 0; i < iters; ++i) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(c2), "+d"(c3) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(c4), "+d"(c5) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(c6), "+d"(c7) : "d"(a), "d"(b));
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
}

// FP64 MMA rate: 4 chains per warp, 2 * 8 * 8 * 4 FLOPs per instruction.
int run_dmma(int blocks, int threads, int iters, double* flops_per_s) {
  double* out = nullptr;
  if (threads % 32 != 0) return 3;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dmma_chains<<<blocks, threads>>>(out, iters / 10);  // warm-up
  cudaEventRecord(e0);
  dmma_chains<<<blocks, threads>>>(out, iters);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return 2;
  *flops_per_s = 2.0 * 8 * 8 * 4 * 4.0 * (double)iters * blocks * (threads / 32) / (ms * 1e-3);
  return 0;
}

// Do the FP64 FMA pipe and the FP64 MMA path share hardware? Even warps run FMA
// chains (iters_f), odd warps MMA chains (iters_m); mode 1 keeps only the FMA
// warps working, mode 2 only the MMA warps, mode 0 both. If the two paths are
// separate, the mode-0 time is near the larger of the other two; if they share
// one unit, near their sum.
__global__ void fp64_mixed_chains(double* out, int iters_f, int iters_m, int mode) {
  const bool mma_warp = (threadIdx.x >> 5) & 1;
  double r = 0.0;
  if (!mma_warp && mode != 2) {
    const double a = 0.999, b = 0.001;
    double x0 = (double)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
           x7 = x0 + 7;
    for (int i = 0; i < iters_f; ++i) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    r = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  } else if (mma_warp && mode != 1) {
    const double a = 1.0 + 1e-3 * (threadIdx.x & 31), b = 1e-3;
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0, c4 = 0.0, c5 = 0.0, c6 = 0.0, c7 = 0.0;
    for (int i = 0; i < iters_m; ++i) {
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c2), "+d"(c3) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c4), "+d"(c5) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c6), "+d"(c7) : "d"(a), "d"(b));
    }
    r = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

int run_mixed(int mode, int blocks, int threads, int iters_f, int iters_m, double* ms_out) {
  double* out = nullptr;
  if (threads % 64 != 0) return 3;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fp64_mixed_chains<<<blocks, threads>>>(out, iters_f / 10, iters_m / 10, mode);  // warm-up
  cudaEventRecord(e0);
  fp64_mixed_chains<<<blocks, threads>>>(out, iters_f, iters_m, mode);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return 2;
  *ms_out = ms;
  return 0;
}

// Float-float arithmetic (a value as an unevaluated sum hi + lo of two floats, about
// 48 significant bits): the multiply-add by Dekker's product error through fmaf and
// Knuth's error-free sum, on the FP32 pipe. 8 independent chains per thread.
struct ff_t {
  float hi, lo;
};
__device__ __forceinline__ ff_t ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff_t ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff_t ff_fma(ff_t a, ff_t b, ff_t c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const ff_t s = ff_two_sum(p, c.hi);
  return ff_fast_two_sum(s.hi, s.lo + e + c.lo);
}
__global__ void ff_chains(float* out, int iters) {
  ff_t x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = {1.0f + 1e-3f * threadIdx.x + j, 1e-9f};
  const ff_t a = {0.999f, 1e-9f}, b = {0.001f, 1e-11f};
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = ff_fma(x[j], a, b);
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j].hi + x[j].lo;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int run_ff(int blocks, int threads, int iters, double* fma_per_s) {
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ff_chains<<<blocks, threads>>>(out, iters / 10);  // warm-up
  cudaEventRecord(e0);
  ff_chains<<<blocks, threads>>>(out, iters);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return 2;
  *fma_per_s = 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return 0;
}

// FP64 FMA chains run by only the first `active` lanes of every warp (the others
// wait at the branch): does the FP64 unit charge a warp instruction by its active
// lanes or as a whole?
__global__ void fp64_lanes_chains(double* out, int iters, int active) {
  double x0 = (double)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  if ((int)(threadIdx.x & 31) < active) {
    const double a = 0.999, b = 0.001;
    for (int i = 0; i < iters; ++i) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

int run_lanes(int active, int blocks, int threads, int iters, double* ms_out) {
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fp64_lanes_chains<<<blocks, threads>>>(out, iters / 10, active);  // warm-up
  cudaEventRecord(e0);
  fp64_lanes_chains<<<blocks, threads>>>(out, iters, active);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return 2;
  *ms_out = ms;
  return 0;
}

}  // namespace

// Time (ms) of FP64 FMA chains on `active` lanes of every warp (1..32).
extern "C" int fp64_lanes_probe(int active, int blocks, int threads, int iters, double* ms) {
  return run_lanes(active, blocks, threads, iters, ms);
}

// Time (ms) of the FP64 FMA / MMA sharing test above (mode 0 both, 1 FMA warps only,
// 2 MMA warps only).
extern "C" int fp64_pipe_probe(int mode, int blocks, int threads, int iters_f, int iters_m, double* ms) {
  return run_mixed(mode, blocks, threads, iters_f, iters_m, ms);
}

// precision: 0 FP64 FMA, 1 FP32 FMA, 2 FP64 MMA (m8n8k4), 3 float-float multiply-adds
// (reported as 2 FLOPs each, like an FMA).
extern "C" int fma_probe(int precision, int blocks, int threads, int iters, double* flops_per_s) {
  if (precision == 2) return run_dmma(blocks, threads, iters, flops_per_s);
  if (precision == 3) {
    const int rc = run_ff(blocks, threads, iters, flops_per_s);
    *flops_per_s *= 2.0;
    return rc;
  }
  return precision == 0 ? run<double>(blocks, threads, iters, flops_per_s)
                        : run<float>(blocks, threads, iters, flops_per_s);
}
