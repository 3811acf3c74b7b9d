// Builds a KernelSet for one (problem, degree, precision) instantiation.
#pragma once
#include <mutex>
#include <type_traits>

#include "elem.cuh"
#include "kernels.h"

namespace ift {

// Raises a kernel's dynamic shared-memory limit to at least smem bytes on the
// current device and never lowers it: several callers (contexts planned for
// different basis sizes, the allocation-free entry point) share one kernel
// instantiation, and a launch planned by one of them must stay valid after
// another has prepared the kernel for a smaller size.
inline std::mutex& smem_attr_mutex() {
  static std::mutex m;
  return m;
}
template <class F>
inline cudaError_t raise_smem(F* f, size_t smem) {
  std::lock_guard<std::mutex> lock(smem_attr_mutex());
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, (const void*)f);
  if (e != cudaSuccess) return e;
  if ((size_t)at.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  return cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class T, int PROB, int P>
struct KernelSetImpl {
  // FP32 sets also hold the tensor-core contraction variants of the fused kernels
  static constexpr bool kTC = std::is_same<T, float>::value;

  static cudaError_t assemble(const void* args, bool jac, int grid, int block, size_t smem, cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    if (jac) {
      if constexpr (kTC) {
        if (a.contraction != 0) {
          assemble_kernel<T, PROB, P, true, true><<<grid, block, smem, s>>>(a);
          return cudaGetLastError();
        }
      }
      assemble_kernel<T, PROB, P, true><<<grid, block, smem, s>>>(a);
    } else {
      assemble_kernel<T, PROB, P, false><<<grid, block, smem, s>>>(a);
    }
    return cudaGetLastError();
  }
  static size_t smem_bytes(bool jac, int ku, int kx, int warps) {
    return jac ? assemble_smem_bytes<T, PROB, P, true>(ku, kx, warps)
               : assemble_smem_bytes<T, PROB, P, false>(ku, kx, warps);
  }
  static size_t smem_bytes_fused(bool jac, int ku, int kx, int warps) {
    return jac ? assemble_smem_bytes<T, PROB, P, true, false, true>(ku, kx, warps)
               : assemble_smem_bytes<T, PROB, P, false, false, true>(ku, kx, warps);
  }
  static cudaError_t prepare(bool jac, size_t smem) {
    if (jac) {
      cudaError_t e = raise_smem(assemble_kernel<T, PROB, P, true>, smem);
      if (e != cudaSuccess) return e;
      if constexpr (kTC) {
        e = raise_smem(assemble_kernel<T, PROB, P, true, true>, smem);
        if (e != cudaSuccess) return e;
      }
      return raise_smem(inspect_kernel<T, PROB, P>, smem);
    }
    return raise_smem(assemble_kernel<T, PROB, P, false>, smem);
  }
  static int blocks_per_sm(bool jac, int block, size_t smem) {
    int n = 0;
    cudaError_t e = jac ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, assemble_kernel<T, PROB, P, true>, block,
                                                                        smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, assemble_kernel<T, PROB, P, false>,
                                                                        block, smem);
    return e == cudaSuccess ? n : 0;
  }
  static cudaError_t inspect(const void* args, const double* U, const double* x, double* R, double* J, double* N,
                             double* dN, int grid, int block, size_t smem, cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    inspect_kernel<T, PROB, P><<<grid, block, smem, s>>>(a, U, x, R, J, N, dN);
    return cudaGetLastError();
  }
  static cudaError_t assemble_batched(const void* args, const void* bargs, bool jac, int grid, int block,
                                      size_t smem, cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    const BatchArgs& b = *(const BatchArgs*)bargs;
    if (jac) {
      if constexpr (kTC) {
        if (a.contraction != 0) {
          assemble_batched_kernel<T, PROB, P, true, true><<<grid, block, smem, s>>>(a, b);
          return cudaGetLastError();
        }
      }
      assemble_batched_kernel<T, PROB, P, true><<<grid, block, smem, s>>>(a, b);
    } else {
      assemble_batched_kernel<T, PROB, P, false><<<grid, block, smem, s>>>(a, b);
    }
    return cudaGetLastError();
  }
  static cudaError_t prepare_batched(bool jac, size_t smem) {
    if (!jac)
      return raise_smem(assemble_batched_kernel<T, PROB, P, false>, smem);
    cudaError_t e = raise_smem(assemble_batched_kernel<T, PROB, P, true>, smem);
    if constexpr (kTC) {
      if (e == cudaSuccess)
        e = raise_smem(assemble_batched_kernel<T, PROB, P, true, true>, smem);
    }
    return e;
  }
  static int blocks_per_sm_batched(bool jac, int block, size_t smem) {
    int n = 0;
    cudaError_t e = jac ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                              &n, assemble_batched_kernel<T, PROB, P, true>, block, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                              &n, assemble_batched_kernel<T, PROB, P, false>, block, smem);
    return e == cudaSuccess ? n : 0;
  }
  static cudaError_t residual_norms(const void* args, const double* wpts, long wstride, const double* mu,
                                    int mustride, int B, int nchunk, int chunk, double* out, int grid, int block,
                                    size_t smem, cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    residual_norms_kernel<T, PROB, P><<<grid, block, smem, s>>>(a, wpts, wstride, mu, mustride, B, nchunk, chunk,
                                                                 out);
    return cudaGetLastError();
  }
  static cudaError_t element_gradients(const void* args, double* out, int grid, int block, size_t smem,
                                       cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    cudaError_t e = raise_smem(element_gradients_kernel<T, PROB, P>, smem);
    if (e != cudaSuccess) return e;
    element_gradients_kernel<T, PROB, P><<<grid, block, smem, s>>>(a, out);
    return cudaGetLastError();
  }
  static cudaError_t prepare_norms(size_t smem) {
    return raise_smem(residual_norms_kernel<T, PROB, P>, smem);
  }
  static int blocks_per_sm_norms(int block, size_t smem) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, residual_norms_kernel<T, PROB, P>, block, smem);
    return e == cudaSuccess ? n : 0;
  }
  // the gradient pass (FP64 sets): its own, smaller shared-memory layout
  static size_t smem_bytes_grad(int ku, int kx, int warps) {
    return assemble_smem_bytes<T, PROB, P, true, true>(ku, kx, warps);
  }
  static int blocks_per_sm_grad(bool batched, int block, size_t smem) {
    int n = 0;
    cudaError_t e = batched ? raise_smem(assemble_batched_kernel<T, PROB, P, true, false, true>, smem)
                            : raise_smem(assemble_kernel<T, PROB, P, true, false, true>, smem);
    if (e != cudaSuccess) return 0;
    e = batched ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, assemble_batched_kernel<T, PROB, P, true, false, true>, block, smem)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, assemble_kernel<T, PROB, P, true, false, true>,
                                                                block, smem);
    return e == cudaSuccess ? n : 0;
  }
  template <int MODE>
  static cudaError_t align_mode(const AsmArgs<T>& a, const double* Xref, const double* vU, const double* vx,
                                const double* vN, double* outU, double* outX, int grid, int block, size_t smem,
                                cudaStream_t s) {
    cudaError_t e = raise_smem(align_kernel<T, PROB, P, MODE>, smem);
    if (e != cudaSuccess) return e;
    align_kernel<T, PROB, P, MODE><<<grid, block, smem, s>>>(a, Xref, vU, vx, vN, outU, outX);
    return cudaGetLastError();
  }
  static cudaError_t align(int mode, const void* args, const double* Xref, const double* vU, const double* vx,
                           const double* vN, double* outU, double* outX, int grid, int block, size_t smem,
                           cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    if (mode == 0) return align_mode<0>(a, Xref, vU, vx, vN, outU, outX, grid, block, smem, s);
    if (mode == 1) return align_mode<1>(a, Xref, vU, vx, vN, outU, outX, grid, block, smem, s);
    return align_mode<2>(a, Xref, vU, vx, vN, outU, outX, grid, block, smem, s);
  }
  // snapshot alignment with stored element systems (FP64 sets)
  static size_t align_jac_smem(int ku, int warps) {
    return cta_bytes<T, PROB, P>(ku, 0) + (size_t)warps * WarpLayout<T, PROB, P, true>(ku, Disc<PROB, P>::NXE).bytes;
  }
  // warps per CTA (1, 2 or 4: the most warps resident on an SM, shared memory being
  // handed out CTA by CTA) and the grid (resident CTAs on sm_count SMs, at most one
  // warp per element)
  static cudaError_t align_jac_plan(int ku, long n, int sm_count, int* warps, int* grid) {
    int best_w = 0, best_occ = 0;
    for (int w : {4, 2, 1}) {
      const size_t smem = align_jac_smem(ku, w);
      if (raise_smem(align_jac_kernel<T, PROB, P>, smem) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, align_jac_kernel<T, PROB, P>, 32 * w, smem) !=
          cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (occ * w > best_occ * best_w) {
        best_w = w;
        best_occ = occ;
      }
    }
    if (best_occ < 1) return cudaErrorInvalidConfiguration;
    cudaError_t e = raise_smem(align_jac_kernel<T, PROB, P>, align_jac_smem(ku, best_w));
    if (e != cudaSuccess) return e;
    long g = (n + best_w - 1) / best_w;
    if (g > (long)sm_count * best_occ) g = (long)sm_count * best_occ;
    *warps = best_w;
    *grid = (int)(g < 1 ? 1 : g);
    return cudaSuccess;
  }
  static cudaError_t align_jac(const void* args, const double* Xref, double* M, double* g, double* F, double* nbad,
                               double* hpart, int warps, int grid, cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    align_jac_kernel<T, PROB, P><<<grid, 32 * warps, align_jac_smem(a.ku, warps), s>>>(a, Xref, M, g, F, nbad,
                                                                                       hpart);
    return cudaGetLastError();
  }
  static size_t align_apply_smem(int ku, int warps) {
    using Dd = Disc<PROB, P>;
    return (size_t)warps * align_apply_warp_doubles(Dd::NXE, ku) * sizeof(double);
  }
  // warps per CTA (as many as fit 96 KB of staging, so that two CTAs share an SM; at
  // most 8) and the grid (resident CTAs of the product kernel on sm_count SMs, at
  // most one warp per element group)
  static cudaError_t align_apply_plan(int ku, long n, int sm_count, int* warps, int* grid) {
    const size_t per = align_apply_smem(ku, 1);
    int w = (int)((96u * 1024u) / (per > 0 ? per : 1));
    w = w < 1 ? 1 : (w > 8 ? 8 : w);
    const size_t smem = align_apply_smem(ku, w);
    using Dd = Disc<PROB, P>;
    auto kern = align_apply_kernel<Dd::NXE, 0>;
    // the shared-memory limit, set here (before any graph capture)
    cudaError_t e = raise_smem(kern, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * w, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const long groups = (n + align_group(Dd::NXE) - 1) / align_group(Dd::NXE);
    long g = (groups + w - 1) / w;
    if (g > (long)sm_count * occ) g = (long)sm_count * occ;
    *warps = w;
    *grid = (int)(g < 1 ? 1 : g);
    return cudaSuccess;
  }
  static cudaError_t align_apply(int mode, const double* M, const double* g, const int* efree, const double* xdir,
                                 long n, int ku, const double* dw, double* part, double* yslot, int grid,
                                 int warps, cudaStream_t s) {
    using Dd = Disc<PROB, P>;
    if (ku > 96 || warps < 1 || warps > 8) return cudaErrorInvalidValue;
    const int block = 32 * warps;
    if (mode == 0)
      align_apply_kernel<Dd::NXE, 0><<<grid, block, align_apply_smem(ku, warps), s>>>(M, g, efree, xdir, n, ku, dw,
                                                                                        part, yslot);
    else if (mode == 1)
      align_apply_kernel<Dd::NXE, 1><<<grid, block, 0, s>>>(M, g, efree, xdir, n, ku, dw, part, yslot);
    else
      align_apply_kernel<Dd::NXE, 2><<<grid, block, 0, s>>>(M, g, efree, xdir, n, ku, dw, part, yslot);
    return cudaGetLastError();
  }
  static cudaError_t assemble_grad(const void* args, int grid, int block, size_t smem, cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    cudaError_t e = raise_smem(assemble_kernel<T, PROB, P, true, false, true>, smem);
    if (e != cudaSuccess) return e;
    assemble_kernel<T, PROB, P, true, false, true><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t assemble_batched_grad(const void* args, const void* bargs, int grid, int block, size_t smem,
                                           cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    const BatchArgs& b = *(const BatchArgs*)bargs;
    cudaError_t e = raise_smem(assemble_batched_kernel<T, PROB, P, true, false, true>, smem);
    if (e != cudaSuccess) return e;
    assemble_batched_kernel<T, PROB, P, true, false, true><<<grid, block, smem, s>>>(a, b);
    return cudaGetLastError();
  }
  static KernelSet make() {
    KernelSet k;
    k.valid = true;
    k.assemble = &assemble;
    k.smem_bytes = &smem_bytes;
    k.smem_bytes_fused = &smem_bytes_fused;
    k.prepare = &prepare;
    k.blocks_per_sm = &blocks_per_sm;
    k.inspect = &inspect;
    k.assemble_batched = &assemble_batched;
    k.prepare_batched = &prepare_batched;
    k.blocks_per_sm_batched = &blocks_per_sm_batched;
    k.residual_norms = &residual_norms;
    k.prepare_norms = &prepare_norms;
    k.element_gradients = &element_gradients;
    if constexpr (!kTC) {
      k.assemble_grad = &assemble_grad;
      k.assemble_batched_grad = &assemble_batched_grad;
      k.smem_bytes_grad = &smem_bytes_grad;
      k.align = &align;
      k.align_jac = &align_jac;
      k.align_jac_smem = &align_jac_smem;
      k.align_apply = &align_apply;
      k.align_apply_plan = &align_apply_plan;
      k.align_jac_plan = &align_jac_plan;
      k.blocks_per_sm_grad = &blocks_per_sm_grad;
    }
    k.blocks_per_sm_norms = &blocks_per_sm_norms;
    return k;
  }
};

}  // namespace ift
