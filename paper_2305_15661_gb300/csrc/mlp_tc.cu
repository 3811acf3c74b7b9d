// The warm-start network's forward pass on the fifth-generation tensor cores, in
// BF16 with FP32 accumulation (ift_mlp_predict_bf16).
//
// One CTA of 128 threads evaluates 128 queries through the whole network:
// - the first layer (n_in inputs, too few for a tensor-core K step) in FP32 by
//   one thread per query;
// - every width x width hidden layer and the output layer as one 128 x N x K
//   product D = A W issued by one thread as tcgen05.mma (kind::f16, BF16
//   operands, FP32 accumulator in tensor memory), K in steps of 16;
// - the epilogue (bias, GELU, rounding to BF16 for the next layer's operand) by
//   the four warps, each reading its 32 accumulator rows with tcgen05.ld.
// Operands live in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, consecutive along K 128 bytes apart,
// consecutive 8-row groups SBO = (K / 8) * 128 bytes apart. A (activations) is
// 128 rows x K, B (weights, one row per output) N rows x K. A small kernel first
// writes each layer's weights in BF16 in exactly that image to global memory;
// each CTA brings them in with one bulk copy per layer (cp.async.bulk completing
// on an mbarrier), the next layer's copy running under the current epilogue.
//
// Waits: on the mbarrier of the weight copies and on the one tcgen05.commit
// arrives on when a layer's products are done; each is bounded (kSpinLimit polls),
// after which the CTA records a timeout in the status word, waits once more
// (bounded) for its products and copies in flight, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/ift.h"
#include "mlp_internal.h"

namespace {

constexpr int kRows = 128;       // queries per CTA = accumulator rows = TMEM lanes
constexpr int kMaxWidth = 256;   // widest layer the kernel takes (N and K)
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between core matrices along K), stride-dimension byte offset
// (between 8-row groups), all in 16-byte units; bits 46-48 = 0b001; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor for kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Makes this thread's generic-proxy shared-memory stores visible to the tensor cores.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Polls the mbarrier for the completion of phase `parity`, at most `limit` times.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Arms the mbarrier for `bytes` of asynchronous copies (one arrival) and starts a
// bulk copy of `bytes` from global memory into shared memory that completes on it.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// 32 lanes x 16 columns of FP32 from tensor memory: thread t of the warp gets
// columns [col, col + 16) of lane (lane base + t).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// Byte offset of element (row, k) in a K-major, no-swizzle operand of K columns.
__host__ __device__ constexpr uint32_t kmajor_offset(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

}  // namespace

namespace {

constexpr int kMaxLayers = 17;
constexpr int kMaxIn = 32;

struct NetArgs {
  const float* x;  // count x n_in, standardised inputs
  float* y;        // count x n_out, standardised outputs
  const float* p;  // FP32 parameters, W_l (in x out, row-major) then b_l per layer
  long long woff[kMaxLayers], boff[kMaxLayers];
  // layers 1.. in BF16, each already in its shared-memory operand image (N rows x K,
  // K-major, no swizzle), at byte offset wpk_off[l] of wpk
  const unsigned char* wpk;
  long long wpk_off[kMaxLayers];
  int count, n_in, width, n_out, layers;
  int n_out_pad;   // n_out rounded up to 16 (the last product's N)
  int tmem_cols;   // tensor-memory columns allocated per CTA (power of two >= 32, >= every N)
  int* status;     // set to 1 if a bounded wait ran out
};

__device__ __forceinline__ void put_bf16(__nv_bfloat16* base, int row, int k, int K, float v) {
  base[kmajor_offset(row, k, K) >> 1] = __float2bfloat16_rn(v);
}

// The operand image of W_l (in = K rows of the parameter matrix, out = Nreal columns):
// row n of the image is output n, K-major; rows Nreal..N-1 are zero.
__global__ void pack_weights_kernel(const float* Wl, int K, int N, int Nreal, __nv_bfloat16* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * K; i += gridDim.x * blockDim.x) {
    const int k = i / N, n = i - k * N;
    put_bf16(out, n, k, K, n < Nreal ? Wl[(size_t)k * Nreal + n] : 0.0f);
  }
}

__global__ void __launch_bounds__(kRows, 1) mlp_bf16_kernel(NetArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int W = a.width;
  const size_t act_bytes = (size_t)kRows * W * 2;
  const int nmax = W > a.n_out_pad ? W : a.n_out_pad;
  __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(sm);
  __nv_bfloat16* wt = reinterpret_cast<__nv_bfloat16*>(sm + act_bytes);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + act_bytes + (size_t)nmax * W * 2);  // products done
  uint64_t* tbar = mbar + 1;                                                               // weights arrived
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long row0 = (long long)blockIdx.x * kRows;
  auto layer_bytes = [&](int l) { return (uint32_t)((l == a.layers - 1 ? a.n_out_pad : W) * W * 2); };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_u32(mbar));
    mbar_init(smem_u32(tbar));
    // the first product's weights, while layer 0 runs on the FMA pipe
    bulk_copy_g2s(smem_u32(wt), a.wpk + a.wpk_off[1], layer_bytes(1), smem_u32(tbar));
  }

  // layer 0 (n_in -> W, GELU) in FP32, one thread per query
  {
    const long long r = row0 + tid;
    float xin[kMaxIn];
    for (int j = 0; j < a.n_in; ++j) xin[j] = r < a.count ? a.x[r * a.n_in + j] : 0.0f;
    const float* W0 = a.p + a.woff[0];
    const float* b0 = a.p + a.boff[0];
    for (int o = 0; o < W; ++o) {
      float z = b0[o];
      for (int j = 0; j < a.n_in; ++j) z += xin[j] * W0[j * W + o];
      put_bf16(act, tid, o, W, gelu(z));
    }
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t sbo = (uint32_t)(W / 8) * 128;
  uint32_t mparity = 0, tparity = 0;
  bool timed_out = false, copy_pending = true;
  for (int l = 1; l < a.layers; ++l) {
    const bool last = l == a.layers - 1;
    const int N = last ? a.n_out_pad : W, Nreal = last ? a.n_out : W;
    // this layer's weights (bulk copy started one layer earlier)
    const bool wok = mbar_wait(smem_u32(tbar), tparity, kSpinLimit);
    if (__syncthreads_or(!wok)) {
      timed_out = true;
      break;
    }
    copy_pending = false;
    tparity ^= 1u;
    if (tid == 0) {
      fence_after_sync();
      const uint32_t ia = smem_u32(act), ib = smem_u32(wt), id = idesc_bf16(kRows, N);
      for (int kk = 0; kk < W / 16; ++kk)
        mma_bf16(tbase, smem_desc(ia + kk * 256, 128, sbo), smem_desc(ib + kk * 256, 128, sbo), id, kk > 0);
      mma_commit(smem_u32(mbar));
    }
    const bool ok = mbar_wait(smem_u32(mbar), mparity, kSpinLimit);
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    mparity ^= 1u;
    fence_after_sync();
    // the products have read this layer's weights and activations: start the next
    // layer's weights now, under the epilogue
    if (!last && tid == 0) bulk_copy_g2s(smem_u32(wt), a.wpk + a.wpk_off[l + 1], layer_bytes(l + 1), smem_u32(tbar));
    copy_pending = !last;
    // epilogue: this warp's 32 accumulator rows, 16 columns at a time
    const int r = warp * 32 + lane;
    const long long grow = row0 + r;
    const float* bl = a.p + a.boff[l];
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (!last) {
#pragma unroll
        for (int i = 0; i < 16; ++i) put_bf16(act, r, c0 + i, W, gelu(v[i] + bl[c0 + i]));
      } else if (grow < a.count) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (c0 + i < Nreal) a.y[grow * Nreal + c0 + i] = v[i] + bl[c0 + i];
      }
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  if (timed_out) {
    if (tid == 0) atomicExch(a.status, 1);
    // products and a weight copy that may still be in flight, each wait bounded
    mbar_wait(smem_u32(mbar), mparity, kSpinLimit);
    if (copy_pending) mbar_wait(smem_u32(tbar), tparity, kSpinLimit);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(a.tmem_cols)
                 : "memory");
}

}  // namespace

extern "C" ift_status ift_mlp_predict_bf16(ift_mlp* n, int64_t count, const double* x, double* out) {
  if (!n || count < 1 || count > ((int64_t)1 << 26) || !x || !out) return IFT_ERR_ARG;
  const int L = n->layers();
  const int W = n->width, ni = n->n_in, no = n->n_out;
  if (n->depth < 1 || L > kMaxLayers || ni > kMaxIn || W < 16 || W % 16 != 0 || W > kMaxWidth || no > kMaxWidth)
    return IFT_ERR_NOTIMPL;
  const int npad = (no + 15) / 16 * 16, nmax = std::max(W, npad);
  int cols = 32;
  while (cols < nmax) cols <<= 1;
  const size_t smem = (size_t)kRows * W * 2 + (size_t)nmax * W * 2 + 32;  // + two mbarriers, TMEM slot
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return IFT_ERR_CUDA;
  if (smem > (size_t)optin) return IFT_ERR_NOTIMPL;
  if (count > n->tc_cap) {
    if (n->tc_x) cudaFree(n->tc_x);
    if (n->tc_y) cudaFree(n->tc_y);
    n->tc_x = n->tc_y = nullptr;
    n->tc_cap = 0;
    if (cudaMalloc(&n->tc_x, sizeof(float) * count * ni) != cudaSuccess ||
        cudaMalloc(&n->tc_y, sizeof(float) * count * no) != cudaSuccess)
      return IFT_ERR_OOM;
    n->tc_cap = count;
  }
  if (!n->tc_status && cudaMalloc(&n->tc_status, sizeof(int)) != cudaSuccess) return IFT_ERR_OOM;
  // the BF16 operand images of layers 1.., rebuilt on every call (training may
  // have changed the parameters)
  long long wpk_off[kMaxLayers] = {0};
  size_t wpk_bytes = 0;
  for (int l = 1; l < L; ++l) {
    wpk_off[l] = (long long)wpk_bytes;
    wpk_bytes += (size_t)(l == L - 1 ? npad : W) * W * 2;
  }
  if (wpk_bytes > n->tc_wpk_bytes) {
    if (n->tc_wpk) cudaFree(n->tc_wpk);
    n->tc_wpk = nullptr;
    n->tc_wpk_bytes = 0;
    if (cudaMalloc(&n->tc_wpk, wpk_bytes) != cudaSuccess) return IFT_ERR_OOM;
    n->tc_wpk_bytes = wpk_bytes;
  }
  std::vector<float> hx((size_t)count * ni), hy((size_t)count * no);
  for (int64_t i = 0; i < count; ++i)
    for (int j = 0; j < ni; ++j) hx[(size_t)i * ni + j] = (float)((x[i * ni + j] - n->xm[j]) / n->xs[j]);
  NetArgs a;
  a.x = n->tc_x;
  a.y = n->tc_y;
  a.p = n->p;
  for (int l = 0; l < kMaxLayers; ++l) {
    a.woff[l] = l < L ? (long long)n->woff[l] : 0;
    a.boff[l] = l < L ? (long long)n->boff[l] : 0;
    a.wpk_off[l] = wpk_off[l];
  }
  a.wpk = n->tc_wpk;
  a.count = (int)count;
  a.n_in = ni;
  a.width = W;
  a.n_out = no;
  a.layers = L;
  a.n_out_pad = npad;
  a.tmem_cols = cols;
  a.status = n->tc_status;
  cudaStream_t s = n->stream;
  if (cudaFuncSetAttribute(mlp_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return IFT_ERR_CUDA;
  if (cudaMemcpyAsync(n->tc_x, hx.data(), hx.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(n->tc_status, 0, sizeof(int), s) != cudaSuccess)
    return IFT_ERR_CUDA;
  for (int l = 1; l < L; ++l) {
    const int N = l == L - 1 ? npad : W, Nreal = l == L - 1 ? no : W;
    pack_weights_kernel<<<(N * W + 255) / 256, 256, 0, s>>>(n->p + n->woff[l], W, N, Nreal,
                                                           reinterpret_cast<__nv_bfloat16*>(n->tc_wpk + wpk_off[l]));
  }
  const unsigned grid = (unsigned)((count + kRows - 1) / kRows);
  mlp_bf16_kernel<<<grid, kRows, smem, s>>>(a);
  int st = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(hy.data(), n->tc_y, hy.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&st, n->tc_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return IFT_ERR_CUDA;
  if (st != 0) return IFT_ERR_TIMEOUT;
  for (int64_t i = 0; i < count; ++i)
    for (int j = 0; j < no; ++j) out[i * no + j] = hy[(size_t)i * no + j] * n->ts[j] + n->tm[j];
  return IFT_OK;
}
