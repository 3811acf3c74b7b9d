// Learned warm start of the LM solve: a fully connected network mu -> (w, tau)
// (GELU hidden layers, linear output, mean-squared-error training with Adam),
// trained and evaluated by the kernels below; and the nearest-training-point
// start it is compared with. The paper itself starts from the projected guess
// (Remark rem:solver); this network only supplies a better starting point for
// the same LM iteration.
//
// Layout: parameters flattened layer by layer as W_l (in x out, row-major), b_l.
// All arithmetic FP32 with FP32 accumulation; every output element of every
// product is summed by one thread in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ift.h"
#include "mlp_internal.h"

namespace {

constexpr int kTile = 16;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * __expf(-0.5f * z * z);
}

// C (M x N) = op(A) (M x K) * op(B) (K x N) [+ bias] ; optional GELU with the
// pre-activation stored in Z. op(A)(m, k) = transA ? A[k*lda + m] : A[m*lda + k].
__global__ void gemm_kernel(const float* A, int lda, int transA, const float* B, int ldb, int transB, float* C,
                            int M, int N, int K, const float* bias, int act, float* Z) {
  __shared__ float As[kTile][kTile + 1], Bs[kTile][kTile + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * kTile + ty, col = blockIdx.x * kTile + tx;
  float acc = 0.0f;
  for (int k0 = 0; k0 < K; k0 += kTile) {
    const int ka = k0 + tx, kb = k0 + ty;
    As[ty][tx] = (row < M && ka < K) ? (transA ? A[(size_t)ka * lda + row] : A[(size_t)row * lda + ka]) : 0.0f;
    Bs[ty][tx] = (kb < K && col < N) ? (transB ? B[(size_t)col * ldb + kb] : B[(size_t)kb * ldb + col]) : 0.0f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTile; ++kk) acc += As[ty][kk] * Bs[kk][tx];
    __syncthreads();
  }
  if (row < M && col < N) {
    float z = acc + (bias ? bias[col] : 0.0f);
    const size_t o = (size_t)row * N + col;
    if (Z) Z[o] = z;
    const float v = act ? gelu_f(z) : z;
    C[o] = v;
  }
}

// dZ = dA * gelu'(Z) (elementwise)
__global__ void gelu_back_kernel(const float* dA, const float* Z, float* dZ, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dZ[i] = dA[i] * gelu_grad_f(Z[i]);
}

// db[o] = sum_b dZ[b][o]
__global__ void colsum_kernel(const float* dZ, int Bn, int out, float* db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= out) return;
  float s = 0.0f;
  for (int b = 0; b < Bn; ++b) s += dZ[(size_t)b * out + o];
  db[o] = s;
}

// dY = 2 (Y - T) / (n d); loss partial sums per block (FP64) -> loss_parts
__global__ void mse_kernel(const float* Y, const float* T, size_t n, double scale, float* dY, double* loss_parts) {
  __shared__ double red[256];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    if (dY) dY[i] = (float)(2.0 * scale) * d;
    s += (double)d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_parts[blockIdx.x] = red[0] * scale;
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// rows[i] = src[idx[i]] for a batch of sample indices
__global__ void gather_rows_kernel(const float* src, int width, const int* idx, int n, float* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * width; i += gridDim.x * blockDim.x) {
    const int r = i / width, c = i - r * width;
    dst[i] = src[(size_t)idx[r] * width + c];
  }
}

// Nearest training point (Euclidean distance of scaled inputs; the lowest index wins ties).
__global__ void nearest_kernel(const double* xt, int64_t nt, int nin, const double* scale, const double* xq,
                               int64_t nq, int64_t* best) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double bd = INFINITY;
  int64_t bi = 0;
  for (int64_t t = 0; t < nt; ++t) {
    double d = 0.0;
    for (int j = 0; j < nin; ++j) {
      const double s = scale ? scale[j] : 1.0;
      const double u = (xq[q * nin + j] - xt[t * nin + j]) * s;
      d += u * u;
    }
    if (d < bd) {
      bd = d;
      bi = t;
    }
  }
  best[q] = bi;
}

inline unsigned grid_for(size_t n, int block) { return (unsigned)std::min<size_t>((n + block - 1) / block, 4096); }

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace


namespace {

template <class P>
void mfree(P*& x) {
  if (x) cudaFree((void*)x);
  x = nullptr;
}

cudaError_t ensure_capacity(ift_mlp* n, int b) {
  if (b <= n->cap) return cudaSuccess;
  for (auto& a : n->A) mfree(a);
  for (auto& z : n->Z) mfree(z);
  for (auto& d : n->dA) mfree(d);
  mfree(n->T);
  mfree(n->Y);
  mfree(n->dY);
  mfree(n->idx);
  const int L = n->layers();
  n->A.assign(L, nullptr);
  n->Z.assign(L, nullptr);
  n->dA.assign(L, nullptr);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    if ((e = cudaMalloc(&n->A[l], sizeof(float) * b * n->lin[l])) != cudaSuccess) break;
    if ((e = cudaMalloc(&n->Z[l], sizeof(float) * b * n->lout[l])) != cudaSuccess) break;
    e = cudaMalloc(&n->dA[l], sizeof(float) * b * std::max(n->lin[l], n->lout[l]));
  }
  if (e == cudaSuccess) e = cudaMalloc(&n->T, sizeof(float) * b * n->n_out);
  if (e == cudaSuccess) e = cudaMalloc(&n->Y, sizeof(float) * b * n->n_out);
  if (e == cudaSuccess) e = cudaMalloc(&n->dY, sizeof(float) * b * n->n_out);
  if (e == cudaSuccess) e = cudaMalloc(&n->idx, sizeof(int) * b);
  if (e == cudaSuccess) n->cap = b;
  return e;
}

void gemm(cudaStream_t s, const float* A, int lda, int tA, const float* B, int ldb, int tB, float* C, int M, int N,
          int K, const float* bias, int act, float* Z) {
  dim3 blk(kTile, kTile), grd((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  gemm_kernel<<<grd, blk, 0, s>>>(A, lda, tA, B, ldb, tB, C, M, N, K, bias, act, Z);
}

// Forward pass of the b rows in A[0] (normalised inputs); output in n->Y. Each
// hidden layer writes its GELU output straight into the next layer's input.
void forward(ift_mlp* n, int b) {
  const int L = n->layers();
  for (int l = 0; l < L; ++l) {
    float* out = (l == L - 1) ? n->Y : n->A[l + 1];
    gemm(n->stream, n->A[l], n->lin[l], 0, n->p + n->woff[l], n->lout[l], 0, out, b, n->lout[l], n->lin[l],
         n->p + n->boff[l], l < L - 1 ? 1 : 0, n->Z[l]);
  }
}

// Backward pass from dY (device) for b rows: parameter gradients into n->g.
void backward(ift_mlp* n, int b) {
  const int L = n->layers();
  float* dcur = n->dY;  // gradient with respect to the layer output (post-activation)
  for (int l = L - 1; l >= 0; --l) {
    const int in = n->lin[l], out = n->lout[l];
    float* dZ = dcur;
    if (l < L - 1) {  // through the GELU, in place
      gelu_back_kernel<<<grid_for((size_t)b * out, 256), 256, 0, n->stream>>>(dcur, n->Z[l], dcur, (size_t)b * out);
    }
    gemm(n->stream, n->A[l], in, 1, dZ, out, 0, n->g + n->woff[l], in, out, b, nullptr, 0, nullptr);  // A^T dZ
    colsum_kernel<<<(out + 127) / 128, 128, 0, n->stream>>>(dZ, b, out, n->g + n->boff[l]);
    if (l > 0) {  // dA_{l-1} = dZ W_l^T
      gemm(n->stream, dZ, out, 0, n->p + n->woff[l], out, 1, n->dA[l - 1], b, in, out, nullptr, 0, nullptr);
      dcur = n->dA[l - 1];
    }
  }
}

// Loss (and gradient) of the b rows already in A[0] against targets T (device).
double loss_and_grad_device(ift_mlp* n, const float* T, int b, bool grad) {
  forward(n, b);
  const size_t cnt = (size_t)b * n->n_out;
  const int blocks = 32;
  mse_kernel<<<blocks, 256, 0, n->stream>>>(n->Y, T, cnt, 1.0 / (double)cnt, grad ? n->dY : nullptr, n->loss_parts);
  if (grad) backward(n, b);
  double parts[32];
  cudaMemcpyAsync(parts, n->loss_parts, sizeof(parts), cudaMemcpyDeviceToHost, n->stream);
  cudaStreamSynchronize(n->stream);
  double s = 0.0;
  for (int i = 0; i < blocks; ++i) s += parts[i];
  return s;
}

}  // namespace

extern "C" {

ift_status ift_mlp_create(int n_in, int width, int depth, int n_out, uint64_t seed, void* stream, ift_mlp** out) {
  if (!out || n_in < 1 || n_out < 1 || depth < 0 || (depth > 0 && width < 1) || depth > 16) return IFT_ERR_ARG;
  ift_mlp* n = new ift_mlp();
  n->n_in = n_in;
  n->width = width;
  n->depth = depth;
  n->n_out = n_out;
  n->stream = (cudaStream_t)stream;
  std::vector<int> dims;
  dims.push_back(n_in);
  for (int i = 0; i < depth; ++i) dims.push_back(width);
  dims.push_back(n_out);
  for (size_t l = 0; l + 1 < dims.size(); ++l) {
    n->lin.push_back(dims[l]);
    n->lout.push_back(dims[l + 1]);
    n->woff.push_back(n->np);
    n->np += (size_t)dims[l] * dims[l + 1];
    n->boff.push_back(n->np);
    n->np += dims[l + 1];
  }
  // seeded initialisation: W ~ N(0, 1/in) by Box-Muller on splitmix64 draws, b = 0
  std::vector<float> h(n->np, 0.0f);
  uint64_t ctr = 0;
  auto unif = [&]() { return ((mix64(seed * 0x9E3779B97F4A7C15ull + (++ctr)) >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
  for (int l = 0; l < n->layers(); ++l) {
    const double sd = 1.0 / std::sqrt((double)n->lin[l]);
    for (size_t i = 0; i < (size_t)n->lin[l] * n->lout[l]; ++i) {
      const double u1 = unif(), u2 = unif();
      h[n->woff[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  bool ok = cudaMalloc(&n->p, sizeof(float) * n->np) == cudaSuccess &&
            cudaMalloc(&n->g, sizeof(float) * n->np) == cudaSuccess &&
            cudaMalloc(&n->m, sizeof(float) * n->np) == cudaSuccess &&
            cudaMalloc(&n->v, sizeof(float) * n->np) == cudaSuccess &&
            cudaMalloc(&n->loss_parts, sizeof(double) * 32) == cudaSuccess &&
            cudaMemcpy(n->p, h.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(n->m, 0, sizeof(float) * n->np) == cudaSuccess &&
            cudaMemset(n->v, 0, sizeof(float) * n->np) == cudaSuccess;
  n->xm.assign(n_in, 0.0);
  n->xs.assign(n_in, 1.0);
  n->tm.assign(n_out, 0.0);
  n->ts.assign(n_out, 1.0);
  if (!ok) {
    ift_mlp_destroy(n);
    return IFT_ERR_OOM;
  }
  *out = n;
  return IFT_OK;
}

ift_status ift_mlp_destroy(ift_mlp* n) {
  if (!n) return IFT_ERR_ARG;
  if (n->stream) cudaStreamSynchronize(n->stream);
  mfree(n->p);
  mfree(n->g);
  mfree(n->m);
  mfree(n->v);
  mfree(n->loss_parts);
  for (auto& a : n->A) mfree(a);
  for (auto& z : n->Z) mfree(z);
  for (auto& d : n->dA) mfree(d);
  mfree(n->T);
  mfree(n->Y);
  mfree(n->dY);
  mfree(n->idx);
  mfree(n->tc_x);
  mfree(n->tc_y);
  mfree(n->tc_status);
  mfree(n->tc_wpk);
  delete n;
  return IFT_OK;
}

ift_status ift_mlp_num_params(const ift_mlp* n, int64_t* count) {
  if (!n || !count) return IFT_ERR_ARG;
  *count = (int64_t)n->np;
  return IFT_OK;
}

ift_status ift_mlp_get_params(const ift_mlp* n, double* params) {
  if (!n || !params) return IFT_ERR_ARG;
  std::vector<float> h(n->np);
  if (cudaMemcpy(h.data(), n->p, sizeof(float) * n->np, cudaMemcpyDeviceToHost) != cudaSuccess) return IFT_ERR_CUDA;
  for (size_t i = 0; i < n->np; ++i) params[i] = h[i];
  return IFT_OK;
}

ift_status ift_mlp_set_params(ift_mlp* n, const double* params) {
  if (!n || !params) return IFT_ERR_ARG;
  std::vector<float> h(n->np);
  for (size_t i = 0; i < n->np; ++i) h[i] = (float)params[i];
  if (cudaMemcpy(n->p, h.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice) != cudaSuccess) return IFT_ERR_CUDA;
  return IFT_OK;
}

ift_status ift_mlp_get_scaling(const ift_mlp* n, double* x_mean, double* x_std, double* t_mean, double* t_std) {
  if (!n || !x_mean || !x_std || !t_mean || !t_std) return IFT_ERR_ARG;
  for (int j = 0; j < n->n_in; ++j) {
    x_mean[j] = n->xm[j];
    x_std[j] = n->xs[j];
  }
  for (int j = 0; j < n->n_out; ++j) {
    t_mean[j] = n->tm[j];
    t_std[j] = n->ts[j];
  }
  return IFT_OK;
}

ift_status ift_mlp_set_scaling(ift_mlp* n, const double* x_mean, const double* x_std, const double* t_mean,
                               const double* t_std) {
  if (!n || !x_mean || !x_std || !t_mean || !t_std) return IFT_ERR_ARG;
  for (int j = 0; j < n->n_in; ++j)
    if (!(x_std[j] > 0.0) || !std::isfinite(x_mean[j])) return IFT_ERR_ARG;
  for (int j = 0; j < n->n_out; ++j)
    if (!(t_std[j] > 0.0) || !std::isfinite(t_mean[j])) return IFT_ERR_ARG;
  for (int j = 0; j < n->n_in; ++j) {
    n->xm[j] = x_mean[j];
    n->xs[j] = x_std[j];
  }
  for (int j = 0; j < n->n_out; ++j) {
    n->tm[j] = t_mean[j];
    n->ts[j] = t_std[j];
  }
  return IFT_OK;
}

ift_status ift_mlp_loss_grad(ift_mlp* n, int64_t count, const double* x, const double* t, double* loss, double* grad) {
  if (!n || count < 1 || count > (1 << 20) || !x || !t) return IFT_ERR_ARG;
  const int b = (int)count;
  if (ensure_capacity(n, b) != cudaSuccess) return IFT_ERR_OOM;
  std::vector<float> hx((size_t)b * n->n_in), ht((size_t)b * n->n_out);
  for (size_t i = 0; i < hx.size(); ++i) hx[i] = (float)x[i];
  for (size_t i = 0; i < ht.size(); ++i) ht[i] = (float)t[i];
  cudaMemcpyAsync(n->A[0], hx.data(), hx.size() * 4, cudaMemcpyHostToDevice, n->stream);
  cudaMemcpyAsync(n->T, ht.data(), ht.size() * 4, cudaMemcpyHostToDevice, n->stream);
  const double L = loss_and_grad_device(n, n->T, b, grad != nullptr);
  if (loss) *loss = L;
  if (grad) {
    std::vector<float> hg(n->np);
    if (cudaMemcpy(hg.data(), n->g, sizeof(float) * n->np, cudaMemcpyDeviceToHost) != cudaSuccess) return IFT_ERR_CUDA;
    for (size_t i = 0; i < n->np; ++i) grad[i] = hg[i];
  }
  return cudaGetLastError() == cudaSuccess ? IFT_OK : IFT_ERR_CUDA;
}

ift_status ift_mlp_train(ift_mlp* n, int64_t count, const double* x, const double* t, int epochs, int batch, double lr,
                         uint64_t seed, double* final_loss) {
  if (!n || count < 2 || !x || !t || epochs < 0 || batch < 1 || !(lr > 0.0)) return IFT_ERR_ARG;
  const int ni = n->n_in, no = n->n_out;
  // normalisation from the training data (mean and standard deviation per column)
  for (int j = 0; j < ni; ++j) {
    double s = 0, s2 = 0;
    for (int64_t i = 0; i < count; ++i) s += x[i * ni + j];
    const double mu = s / count;
    for (int64_t i = 0; i < count; ++i) s2 += (x[i * ni + j] - mu) * (x[i * ni + j] - mu);
    n->xm[j] = mu;
    n->xs[j] = std::sqrt(s2 / count) > 0 ? std::sqrt(s2 / count) : 1.0;
  }
  for (int j = 0; j < no; ++j) {
    double s = 0, s2 = 0;
    for (int64_t i = 0; i < count; ++i) s += t[i * no + j];
    const double mu = s / count;
    for (int64_t i = 0; i < count; ++i) s2 += (t[i * no + j] - mu) * (t[i * no + j] - mu);
    n->tm[j] = mu;
    n->ts[j] = std::sqrt(s2 / count) > 0 ? std::sqrt(s2 / count) : 1.0;
  }
  std::vector<float> hx((size_t)count * ni), ht((size_t)count * no);
  for (int64_t i = 0; i < count; ++i) {
    for (int j = 0; j < ni; ++j) hx[i * ni + j] = (float)((x[i * ni + j] - n->xm[j]) / n->xs[j]);
    for (int j = 0; j < no; ++j) ht[i * no + j] = (float)((t[i * no + j] - n->tm[j]) / n->ts[j]);
  }
  float *dX = nullptr, *dT = nullptr;
  int* dperm = nullptr;
  if (cudaMalloc(&dX, hx.size() * 4) != cudaSuccess || cudaMalloc(&dT, ht.size() * 4) != cudaSuccess ||
      cudaMalloc(&dperm, sizeof(int) * count) != cudaSuccess) {
    mfree(dX);
    mfree(dT);
    mfree(dperm);
    return IFT_ERR_OOM;
  }
  cudaMemcpyAsync(dX, hx.data(), hx.size() * 4, cudaMemcpyHostToDevice, n->stream);
  cudaMemcpyAsync(dT, ht.data(), ht.size() * 4, cudaMemcpyHostToDevice, n->stream);
  const int b = (int)std::min<int64_t>(batch, count);
  if (ensure_capacity(n, std::max(b, (int)std::min<int64_t>(count, 4096))) != cudaSuccess) {
    mfree(dX);
    mfree(dT);
    mfree(dperm);
    return IFT_ERR_OOM;
  }
  std::vector<int> perm(count);
  uint64_t ctr = 0;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  // the step decays from lr to lr / 100 along a half cosine over the run's steps:
  // with a constant step the final weights are one point of Adam's noise band, and
  // a change in the last bits of the targets picks another one
  const double steps_total = (double)epochs * (double)(count / b);
  double step_no = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t i = 0; i < count; ++i) perm[i] = (int)i;
    for (int64_t i = count - 1; i > 0; --i) {  // Fisher-Yates with splitmix64 draws
      const int64_t j = (int64_t)(mix64(seed * 0xD1B54A32D192ED03ull + (++ctr)) % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * count, cudaMemcpyHostToDevice, n->stream);
    for (int64_t s0 = 0; s0 + b <= count; s0 += b) {
      gather_rows_kernel<<<grid_for((size_t)b * ni, 256), 256, 0, n->stream>>>(dX, ni, dperm + s0, b, n->A[0]);
      gather_rows_kernel<<<grid_for((size_t)b * no, 256), 256, 0, n->stream>>>(dT, no, dperm + s0, b, n->T);
      forward(n, b);
      const size_t cnt = (size_t)b * no;
      mse_kernel<<<32, 256, 0, n->stream>>>(n->Y, n->T, cnt, 1.0 / (double)cnt, n->dY, n->loss_parts);
      backward(n, b);
      ++n->adam_t;
      const float c1 = 1.0f / (1.0f - std::pow(b1, (float)n->adam_t));
      const float c2 = 1.0f / (1.0f - std::pow(b2, (float)n->adam_t));
      const double lr_t =
          lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(3.141592653589793 * step_no / std::max(steps_total, 1.0))));
      step_no += 1.0;
      adam_kernel<<<grid_for(n->np, 256), 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, n->np, (float)lr_t, b1, b2,
                                                               eps, c1, c2);
    }
  }
  double total = 0.0;
  int64_t done = 0;
  while (done < count) {
    const int bb = (int)std::min<int64_t>(count - done, n->cap);
    cudaMemcpyAsync(n->A[0], dX + done * ni, sizeof(float) * bb * ni, cudaMemcpyDeviceToDevice, n->stream);
    total += loss_and_grad_device(n, dT + done * no, bb, false) * bb;
    done += bb;
  }
  if (final_loss) *final_loss = total / (double)count;
  mfree(dX);
  mfree(dT);
  mfree(dperm);
  return cudaGetLastError() == cudaSuccess ? IFT_OK : IFT_ERR_CUDA;
}

ift_status ift_mlp_predict(ift_mlp* n, int64_t count, const double* x, double* out) {
  if (!n || count < 1 || !x || !out) return IFT_ERR_ARG;
  const int ni = n->n_in, no = n->n_out;
  const int b = (int)std::min<int64_t>(count, 4096);
  if (ensure_capacity(n, b) != cudaSuccess) return IFT_ERR_OOM;
  std::vector<float> hx((size_t)b * ni), hy((size_t)b * no);
  for (int64_t s0 = 0; s0 < count; s0 += b) {
    const int bb = (int)std::min<int64_t>(b, count - s0);
    for (int i = 0; i < bb; ++i)
      for (int j = 0; j < ni; ++j) hx[(size_t)i * ni + j] = (float)((x[(s0 + i) * ni + j] - n->xm[j]) / n->xs[j]);
    cudaMemcpyAsync(n->A[0], hx.data(), (size_t)bb * ni * 4, cudaMemcpyHostToDevice, n->stream);
    forward(n, bb);
    cudaMemcpyAsync(hy.data(), n->Y, (size_t)bb * no * 4, cudaMemcpyDeviceToHost, n->stream);
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) return IFT_ERR_CUDA;
    for (int i = 0; i < bb; ++i)
      for (int j = 0; j < no; ++j) out[(s0 + i) * no + j] = hy[(size_t)i * no + j] * n->ts[j] + n->tm[j];
  }
  return IFT_OK;
}

ift_status ift_nearest_start(int64_t n_train, int n_in, const double* x_train, int n_out, const double* y_train,
                             int64_t n_query, const double* x_query, const double* scale, double* y_out) {
  if (n_train < 1 || n_in < 1 || n_out < 1 || n_query < 1 || !x_train || !y_train || !x_query || !y_out)
    return IFT_ERR_ARG;
  double *dxt = nullptr, *dxq = nullptr, *dsc = nullptr;
  int64_t* dbest = nullptr;
  auto cleanup = [&]() {
    mfree(dxt);
    mfree(dxq);
    mfree(dsc);
    mfree(dbest);
  };
  if (cudaMalloc(&dxt, sizeof(double) * n_train * n_in) != cudaSuccess ||
      cudaMalloc(&dxq, sizeof(double) * n_query * n_in) != cudaSuccess ||
      cudaMalloc(&dsc, sizeof(double) * n_in) != cudaSuccess ||
      cudaMalloc(&dbest, sizeof(int64_t) * n_query) != cudaSuccess) {
    cleanup();
    return IFT_ERR_OOM;
  }
  std::vector<double> sc(n_in, 1.0);
  if (scale) std::memcpy(sc.data(), scale, sizeof(double) * n_in);
  cudaMemcpy(dxt, x_train, sizeof(double) * n_train * n_in, cudaMemcpyHostToDevice);
  cudaMemcpy(dxq, x_query, sizeof(double) * n_query * n_in, cudaMemcpyHostToDevice);
  cudaMemcpy(dsc, sc.data(), sizeof(double) * n_in, cudaMemcpyHostToDevice);
  nearest_kernel<<<(unsigned)((n_query + 127) / 128), 128>>>(dxt, n_train, n_in, dsc, dxq, n_query, dbest);
  std::vector<int64_t> best(n_query);
  const cudaError_t e = cudaMemcpy(best.data(), dbest, sizeof(int64_t) * n_query, cudaMemcpyDeviceToHost);
  cleanup();
  if (e != cudaSuccess) return IFT_ERR_CUDA;
  for (int64_t q = 0; q < n_query; ++q)
    std::memcpy(y_out + q * n_out, y_train + best[q] * n_out, sizeof(double) * n_out);
  return IFT_OK;
}

}  // extern "C"
