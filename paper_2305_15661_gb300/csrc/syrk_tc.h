// The rho-weighted Gauss-Newton matrix from the element kernel's transposed BF16
// rows of sqrt(rho_e) A_e, on the tcgen05 tensor cores (syrk_tc.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace ift {

// Rows of the transposed stack a buffer must hold for n_stack stacked rows (a
// multiple of the kernel's 64-row tile; the rows past n_stack must be zero).
long syrk_tc_rows(long n_stack);
// Dynamic shared memory of the kernel; syrk_tc_prepare raises the kernel's limit to
// it (call before any stream capture).
size_t syrk_tc_smem();
cudaError_t syrk_tc_prepare();
// Writes one FP64 partial row [H (k x k) | zeros] of nacc entries per CTA at partial,
// at most max_ctas CTAs; *ctas receives the count. At: k rows of ldr BF16 values (ldr
// a multiple of 64, rows n_stack..ldr-1 zero), 1 <= k <= 64. skip: as for the element
// kernels. status: set to 1 if a bounded wait ran out.
cudaError_t syrk_tc_launch(const uint16_t* At, long ldr, long n_stack, int k, int max_ctas, double* partial,
                           int nacc, const int* skip, int* status, int* ctas, cudaStream_t s);

}  // namespace ift
