// ift_reduced_residual_jacobian_static: the fused FP64 assembly for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the reduced
// system: code running while a stream is being captured into a CUDA graph (an
// allocation there breaks the capture), code that owns all device memory through
// its own pool or arena and forbids other allocators, and hosts where an
// allocation would synchronise the device in a latency-critical loop. The
// context-based calls allocate their scratch (per-CTA partial sums) in
// ift_set_bases; this entry point instead takes every input and output as a
// caller-owned device pointer and keeps its scratch in the file-scope array
// below, so it calls no cudaMalloc, cudaFree or allocating library routine.
//
// Scratch: g_static_scratch, 2 MiB of doubles, allocated by the CUDA module
// when the library is loaded and held by every GPU that loads the library until
// the process exits. It holds the reference-element tables, the per-CTA partial
// sums and the reduced result of the current call. Every call shares it and it
// keeps the last call's contents; each call overwrites what it reads, so nothing
// needs clearing, but calls whose GPU work overlaps (different streams, or
// different host threads, on the same device) race on it and must be serialised
// by the caller.
//
// Set-up: the first call on each device looks up the device address of the array
// with cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture on the device.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "../../include/ift.h"
#include "elem.cuh"
#include "kernels.h"
#include "refelem.h"

namespace ift {
__global__ void reduce_partials_kernel(const double* partial, int nparts, int nacc, double* out, const int* skip);
}  // namespace ift

using namespace ift;

namespace {

constexpr size_t kStaticScratchDoubles = 262144;  // 2 MiB
constexpr int kStaticMaxDevices = 64;
constexpr int kStaticWarps = 2;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

std::mutex g_static_mu;
double* g_static_ptr[kStaticMaxDevices] = {nullptr};

__global__ void static_unpack_kernel(const double* res, int ku, int kx, double* S, double* T, double* H,
                                     double* J) {
  const int k = ku + kx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k * k + k + 1; i += gridDim.x * blockDim.x) {
    if (i < k * k) {
      if (H) H[i] = res[i];
    } else if (i < k * k + ku) {
      if (S) S[i - k * k] = res[i];
    } else if (i < k * k + k) {
      if (T) T[i - k * k - ku] = res[i];
    } else if (J) {
      J[0] = res[k * k + k + 1] > 0.0 ? INFINITY : res[k * k + k];
    }
  }
}

// Device address of the static scratch on the current device (looked up once).
cudaError_t static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_ptr[dev] == nullptr) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

// Reference tables packed as the element kernels read them (D | B | Lt | fw | qw | qxi),
// built once per (problem, degree) in host memory that lives until exit.
const std::vector<double>* packed_tables(int problem, int p) {
  static std::vector<double> cache[3][4];
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  std::vector<double>& t = cache[problem][p];
  if (t.empty()) {
    RefTables R;
    if (!build_tables(problem == IFT_BURGERS1D ? 1 : 2, p, R)) return nullptr;
    t.insert(t.end(), R.D.begin(), R.D.end());
    t.insert(t.end(), R.B.begin(), R.B.end());
    t.insert(t.end(), R.Lt.begin(), R.Lt.end());
    t.insert(t.end(), R.fw.begin(), R.fw.end());
    t.insert(t.end(), R.qw.begin(), R.qw.end());
    if (problem == IFT_BURGERS1D) {
      t.insert(t.end(), R.qxi.begin(), R.qxi.end());
    } else {
      t.insert(t.end(), (size_t)R.nq, 0.0);
    }
  }
  return &t;
}

}  // namespace

extern "C" ift_status ift_reduced_residual_jacobian_static(
    int problem, int p, int64_t n_verts, const double* X, int64_t n_elems, const int32_t* elem_verts,
    const int32_t* nbr, const int32_t* nbr_face, const int8_t* bc, const double* Phi, int k_u, const double* Psi,
    int k_x, int64_t nnz, const int32_t* elems, const double* rho, const double* mu, const double* y,
    const double* z, double gamma, double kappa, double eps_g, double* S, double* T, double* H, double* J,
    void* stream) {
  if (problem != IFT_BURGERS1D && problem != IFT_EULER2D) return IFT_ERR_ARG;
  if (p < 1 || p > 3) return IFT_ERR_ARG;
  if (n_verts < 1 || n_elems < 1 || n_elems > ((int64_t)1 << 30)) return IFT_ERR_ARG;
  if (k_u < 1 || k_x < 0 || k_u + k_x > 64) return IFT_ERR_ARG;
  if (!X || !elem_verts || !nbr || !nbr_face || !bc || !Phi || (k_x > 0 && (!Psi || !z)) || !mu || !y)
    return IFT_ERR_ARG;
  if (nnz == 0 || (nnz > 0 && (!elems || !rho))) return IFT_ERR_ARG;
  const KernelSet ks = (problem == IFT_BURGERS1D) ? burgers_kernels(p, 0) : euler_kernels(p, 0);
  if (!ks.valid) return IFT_ERR_NOTIMPL;
  const std::vector<double>* tab = packed_tables(problem, p);
  if (!tab) return IFT_ERR_ARG;
  const int k = k_u + k_x;
  const int nacc = k * k + k + 2;
  // scratch layout: [tables | result (nacc) | partials (grid x nacc)], each 32-double aligned
  auto up32 = [](size_t n) { return (n + 31) & ~size_t(31); };
  const size_t o_res = up32(tab->size());
  const size_t o_part = o_res + up32(nacc);
  if (o_part + (size_t)nacc > kStaticScratchDoubles) return IFT_ERR_ARG;  // k too large for the scratch
  const size_t max_grid = (kStaticScratchDoubles - o_part) / nacc;

  double* scratch = nullptr;
  if (static_scratch(&scratch) != cudaSuccess) return IFT_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int block = 32 * kStaticWarps;
  const size_t smem = ks.smem_bytes(true, k_u, k_x, kStaticWarps);
  if (ks.prepare(true, smem) != cudaSuccess) return IFT_ERR_CUDA;
  const int bps = ks.blocks_per_sm(true, block, smem);
  int dev = 0, sms = 0;
  if (bps < 1 || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IFT_ERR_CUDA;
  const long items = nnz > 0 ? nnz : n_elems;
  long grid = (long)sms * bps;
  const long need = (items + kStaticWarps - 1) / kStaticWarps;
  if (grid > need) grid = need;
  if (grid > (long)max_grid) grid = (long)max_grid;
  if (grid < 1) grid = 1;

  if (cudaMemcpyAsync(scratch, tab->data(), tab->size() * sizeof(double), cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return IFT_ERR_CUDA;
  AsmArgs<double> a;
  a.X = X;
  a.ev = elem_verts;
  a.nbr = nbr;
  a.nbr_face = nbr_face;
  a.bc = (const signed char*)bc;
  a.Phi = Phi;
  a.Psi = Psi;
  a.ku = k_u;
  a.kx = k_x;
  a.elems = nnz > 0 ? elems : nullptr;
  a.rho = nnz > 0 ? rho : nullptr;
  a.n_items = items;
  a.w = y;
  a.tau = k_x > 0 ? z : y;  // not read when k_x = 0
  a.mu = mu;
  a.tables = scratch;
  a.gamma = gamma;
  a.kappa = kappa;
  a.eps = eps_g;
  a.partial = scratch + o_part;
  a.skip = nullptr;
  a.contraction = 0;
  a.need_hn = 0;
  if (ks.assemble(&a, true, (int)grid, block, smem, s) != cudaSuccess) return IFT_ERR_CUDA;
  reduce_partials_kernel<<<(nacc + 31) / 32, 256, 0, s>>>(scratch + o_part, (int)grid, nacc, scratch + o_res, nullptr);
  static_unpack_kernel<<<(nacc + 255) / 256, 256, 0, s>>>(scratch + o_res, k_u, k_x, S, T, H, J);
  if (cudaGetLastError() != cudaSuccess) return IFT_ERR_CUDA;
  return IFT_OK;
}
