// Host-side table of the element kernels instantiated for each
// (problem, degree, precision), so the C-ABI code can dispatch at run time.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace ift {

struct KernelSet {
  bool valid = false;
  // launch the fused assembly (jac = true) or the objective-only pass (jac = false);
  // args points to an AsmArgs<T> of the set's precision
  cudaError_t (*assemble)(const void* args, bool jac, int grid, int block, size_t smem, cudaStream_t s) = nullptr;
  // dynamic shared memory: smem_bytes for the kernels that share the element layout
  // (inspection, per-element gradients, norms, alignment), smem_bytes_fused for the
  // fused assembly kernels (assemble and assemble_batched), whose FP32 layout is smaller
  size_t (*smem_bytes)(bool jac, int ku, int kx, int warps) = nullptr;
  size_t (*smem_bytes_fused)(bool jac, int ku, int kx, int warps) = nullptr;
  cudaError_t (*prepare)(bool jac, size_t smem) = nullptr;
  int (*blocks_per_sm)(bool jac, int block, size_t smem) = nullptr;
  cudaError_t (*inspect)(const void* args, const double* U, const double* x, double* R, double* J, double* N,
                         double* dN, int grid, int block, size_t smem, cudaStream_t s) = nullptr;
  // batched fused assembly over query chunks; bargs points to a BatchArgs
  cudaError_t (*assemble_batched)(const void* args, const void* bargs, bool jac, int grid, int block, size_t smem,
                                  cudaStream_t s) = nullptr;
  cudaError_t (*prepare_batched)(bool jac, size_t smem) = nullptr;
  int (*blocks_per_sm_batched)(bool jac, int block, size_t smem) = nullptr;
  // HDM residual norms of many points (rho = 1, no Jacobians); args as for assemble
  cudaError_t (*residual_norms)(const void* args, const double* wpts, long wstride, const double* mu, int mustride,
                                int B, int nchunk, int chunk, double* out, int grid, int block, size_t smem,
                                cudaStream_t s) = nullptr;
  cudaError_t (*prepare_norms)(size_t smem) = nullptr;
  // FP64 sets: the gradient pass (rows of [g | J | count] per CTA or per chunk)
  cudaError_t (*assemble_grad)(const void* args, int grid, int block, size_t smem, cudaStream_t s) = nullptr;
  cudaError_t (*assemble_batched_grad)(const void* args, const void* bargs, int grid, int block, size_t smem,
                                       cudaStream_t s) = nullptr;
  size_t (*smem_bytes_grad)(int ku, int kx, int warps) = nullptr;
  // FP64 sets: the snapshot-alignment element pass (mode 0 residual, 1 J v, 2 J^T v;
  // see align_kernel), shared memory as the fused kernel's with kx = 0
  cudaError_t (*align)(int mode, const void* args, const double* Xref, const double* vU, const double* vx,
                       const double* vN, double* outU, double* outX, int grid, int block, size_t smem,
                       cudaStream_t s) = nullptr;
  // FP64 sets: snapshot alignment with stored element systems. align_jac writes per
  // element (M_e)_wx and (M_e)_xx (k_u n_xe + n_xe^2 doubles), g_e (k = k_u + n_xe)
  // and F, and per CTA its part of H_ww (packed, hpart: grid x k_u (k_u + 1) / 2), at
  // the state of args, in the launch shape of align_jac_plan; align_apply forms the
  // non-H_ww parts of mode 0 J^T J v, 1 J^T F, 2 diag(J^T J) (see align_apply_kernel;
  // efree: the free index of each element coordinate, -1 fixed; xdir: the mesh
  // direction per element for mode 0; part: grid x k_u; yslot: the mesh rows per
  // element coordinate), in the launch shape of align_apply_plan
  cudaError_t (*align_jac_plan)(int ku, long n, int sm_count, int* warps, int* grid) = nullptr;
  cudaError_t (*align_jac)(const void* args, const double* Xref, double* M, double* g, double* F, double* nbad,
                           double* hpart, int warps, int grid, cudaStream_t s) = nullptr;
  size_t (*align_jac_smem)(int ku, int warps) = nullptr;
  cudaError_t (*align_apply)(int mode, const double* M, const double* g, const int* efree, const double* xdir,
                             long n, int ku, const double* dw, double* part, double* yslot, int grid, int warps,
                             cudaStream_t s) = nullptr;
  cudaError_t (*align_apply_plan)(int ku, long n, int sm_count, int* warps, int* grid) = nullptr;
  int (*blocks_per_sm_grad)(bool batched, int block, size_t smem) = nullptr;
  // per-element [S^(e); T^(e); J^(e)] rows; args as for assemble
  cudaError_t (*element_gradients)(const void* args, double* out, int grid, int block, size_t smem,
                                   cudaStream_t s) = nullptr;
  int (*blocks_per_sm_norms)(int block, size_t smem) = nullptr;
};

// precision: 0 = FP64, 1 = FP32
KernelSet euler_kernels(int p, int precision);
// Euler on curved (q = 2) six-node triangles
KernelSet euler_curved_kernels(int p, int precision);
KernelSet burgers_kernels(int p, int precision);

}  // namespace ift
