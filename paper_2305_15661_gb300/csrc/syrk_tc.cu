// H = sum_r a_r^T a_r over the stacked rows a_r (1 x k) of sqrt(rho_e) A_e (Eq.
// levmarq-elem's rho-weighted Gauss-Newton matrix), on the fifth-generation tensor
// cores: BF16 operands, FP32 accumulation in tensor memory.
//
// The element kernel writes the rows transposed, At[m][r] (k rows of ldr BF16
// values, r = item * n_u + i), so that one 64-row slice of the stack is, for every
// m, 128 contiguous bytes. Each CTA takes a contiguous range of 64-row tiles and
// accumulates D = T T^T with T the 128 x 64 tile image (rows m < k from At, rows
// k..127 zero): one tcgen05.mma.cta_group::1.kind::f16 with M = 128, N = k rounded
// up to 16, K = 16 per quarter tile, A and B the same shared-memory image. Tiles
// come in by 16-byte cp.async copies into the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices, 128 bytes apart along K, 8-row groups
// 1,024 bytes apart) through a ring of kStages buffers; a stage is refilled after
// the tcgen05.commit of the products that read it has arrived on its mbarrier.
// At the end warps 0 and 1 read the k x k accumulator from tensor memory
// (tcgen05.ld) and write it as one partial row [H | 0 ... 0] in FP64.
//
// Every mbarrier wait is bounded (kSpinLimit polls); a CTA that runs out records
// it in the status word, waits once more (bounded) for its products, frees its
// tensor memory and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "syrk_tc.h"

namespace {

constexpr int kThreads = 128;
constexpr int kTileRows = 64;                 // rows of the stack (the K extent) per tile
constexpr int kStageBytes = 128 * kTileRows * 2;  // 128 x 64 BF16 image: 16 KB
constexpr int kStages = 6;
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading-dimension byte offset (core
// matrices along K), stride-dimension byte offset (8-row groups), 16-byte units;
// bit 46 set; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
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
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

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

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// 32 lanes x 16 columns of FP32 from tensor memory.
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

// The tile of stack rows [row0, row0 + 64) into stage image `stage`: for m < k the
// 128 bytes At[m][row0 .. row0 + 63] as eight 16-byte chunks; chunk c of row m goes to
// (m / 8) * 1024 + c * 128 + (m % 8) * 16.
__device__ __forceinline__ void load_tile(uint32_t stage, const uint16_t* At, long ldr, long row0, int k, int tid) {
  for (int idx = tid; idx < k * 8; idx += kThreads) {
    const int m = idx >> 3, c = idx & 7;
    cp_async16(stage + (uint32_t)((m >> 3) * 1024 + c * 128 + (m & 7) * 16), At + (size_t)m * ldr + row0 + c * 8);
  }
}

// Two CTAs per SM (2 x 98 KB of shared memory): the stack is read once, and the
// copies in flight across both CTAs' rings set the bandwidth.
__global__ void __launch_bounds__(kThreads, 2)
    syrk_tc_kernel(const uint16_t* At, long ldr, int k, long tiles, long tiles_per_cta, double* partial, int nacc,
                   const int* skip, int* status) {
  if (skip != nullptr && *(volatile const int*)skip) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + (size_t)kStages * kStageBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long t0 = (long)blockIdx.x * tiles_per_cta;
  const long t1 = t0 + tiles_per_cta < tiles ? t0 + tiles_per_cta : tiles;
  const int nt = t1 > t0 ? (int)(t1 - t0) : 0;
  const int kn = (k + 15) / 16 * 16;  // N of the products
  constexpr int kCols = 64;           // tensor-memory columns (>= kn, k <= 64)

  // rows k..127 of every stage stay zero: clear all stages once
  for (int i = tid; i < kStages * kStageBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0)
    for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(mbar + s));
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t sm0 = smem_u32(sm);
  auto stage_addr = [&](int s) { return sm0 + (uint32_t)s * kStageBytes; };

  // prologue: tiles 0 .. kStages - 2
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nt) load_tile(stage_addr(s), At, ldr, (t0 + s) * kTileRows, k, tid);
    cp_async_commit();
  }
  bool timed_out = false;
  int issued = 0;  // tiles whose products were issued
  for (int t = 0; t < nt; ++t) {
    const int u = t + kStages - 1;  // the tile to prefetch, into the stage tile u - kStages used
    if (u < nt && u >= kStages) {
      const bool ok = mbar_wait(smem_u32(mbar + u % kStages), (uint32_t)(((u - kStages) / kStages) & 1), kSpinLimit);
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
    }
    if (u < nt) load_tile(stage_addr(u % kStages), At, ldr, (t0 + u) * kTileRows, k, tid);
    cp_async_commit();
    cp_async_wait<kStages - 1>();  // tile t has landed (this thread's copies)
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid == 0) {
      const uint32_t a = stage_addr(t % kStages), id = idesc_bf16(128, kn);
#pragma unroll
      for (int q = 0; q < kTileRows / 16; ++q) {
        const uint64_t d = smem_desc(a + q * 256, 128, 1024);
        mma_bf16(tbase, d, d, id, (t > 0 || q > 0) ? 1 : 0);
      }
      mma_commit(smem_u32(mbar + t % kStages));
    }
    issued = t + 1;
  }
  // the last products (each commit covers every product issued before it)
  bool done_ok = true;
  if (issued > 0) {
    const int last = issued - 1;
    done_ok = mbar_wait(smem_u32(mbar + last % kStages), (uint32_t)((last / kStages) & 1), kSpinLimit);
  }
  cp_async_wait<0>();
  if (__syncthreads_or(!done_ok)) timed_out = true;
  fence_after_sync();
  // partial row: H (k x k, from accumulator rows m < k), then zeros for g, J, count
  double* row = partial + (size_t)blockIdx.x * nacc;
  if (!timed_out && nt > 0) {
    if (warp < 2) {
      const int m = warp * 32 + lane;
      for (int c0 = 0; c0 < kn; c0 += 16) {
        float v[16];
        tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (m < k) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c0 + i < k) row[(size_t)m * k + c0 + i] = (double)v[i];
        }
      }
    }
  } else {
    for (int i = tid; i < k * k; i += kThreads) row[i] = 0.0;
  }
  for (int i = k * k + tid; i < nacc; i += kThreads) row[i] = 0.0;
  if (timed_out && tid == 0) atomicExch(status, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(kCols) : "memory");
}

}  // namespace

namespace ift {

size_t syrk_tc_smem() { return (size_t)kStages * kStageBytes + kStages * 8 + 16; }

cudaError_t syrk_tc_prepare() {
  return cudaFuncSetAttribute(syrk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)syrk_tc_smem());
}

long syrk_tc_rows(long n_stack) { return (n_stack + kTileRows - 1) / kTileRows * kTileRows; }

cudaError_t syrk_tc_launch(const uint16_t* At, long ldr, long n_stack, int k, int max_ctas, double* partial,
                           int nacc, const int* skip, int* status, int* ctas, cudaStream_t s) {
  *ctas = 0;
  if (k < 1 || k > 64 || ldr % kTileRows != 0 || n_stack > ldr || max_ctas < 1) return cudaErrorInvalidValue;
  const long tiles = (n_stack + kTileRows - 1) / kTileRows;
  if (tiles == 0) return cudaSuccess;
  long grid = tiles < max_ctas ? tiles : max_ctas;
  const long per = (tiles + grid - 1) / grid;
  grid = (tiles + per - 1) / per;
  syrk_tc_kernel<<<(int)grid, kThreads, syrk_tc_smem(), s>>>(At, ldr, k, tiles, per, partial, nacc, skip, status);
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) *ctas = (int)grid;
  return e;
}

}  // namespace ift
