// Builds a KernelSet for one (problem, degree, precision) instantiation.
#pragma once
#include "elem.cuh"
#include "kernels.h"

namespace ift {

template <class T, int PROB, int P>
struct KernelSetImpl {
  static cudaError_t assemble(const void* args, bool jac, int grid, int block, size_t smem, cudaStream_t s) {
    const AsmArgs<T>& a = *(const AsmArgs<T>*)args;
    if (jac)
      assemble_kernel<T, PROB, P, true><<<grid, block, smem, s>>>(a);
    else
      assemble_kernel<T, PROB, P, false><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
  }
  static size_t smem_bytes(bool jac, int ku, int kx, int warps) {
    return jac ? assemble_smem_bytes<T, PROB, P, true>(ku, kx, warps)
               : assemble_smem_bytes<T, PROB, P, false>(ku, kx, warps);
  }
  static cudaError_t prepare(bool jac, size_t smem) {
    if (jac) {
      cudaError_t e = cudaFuncSetAttribute(assemble_kernel<T, PROB, P, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(inspect_kernel<T, PROB, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem);
    }
    return cudaFuncSetAttribute(assemble_kernel<T, PROB, P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
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
  static KernelSet make() {
    KernelSet k;
    k.valid = true;
    k.assemble = &assemble;
    k.smem_bytes = &smem_bytes;
    k.prepare = &prepare;
    k.blocks_per_sm = &blocks_per_sm;
    k.inspect = &inspect;
    return k;
  }
};

}  // namespace ift
