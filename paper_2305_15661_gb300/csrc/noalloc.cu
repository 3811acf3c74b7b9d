// ift_reduced_residual_jacobian_static: the fused FP64 assembly for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the reduced
// system: code that owns all device memory through its own pool or arena and
// forbids other allocators, programs that reserve their whole memory budget at
// start-up, and hosts where an allocation would synchronise the device in a
// latency-critical loop. The context-based calls allocate their scratch (per-CTA
// partial sums) in ift_set_bases; this entry point instead takes every input and
// output as a caller-owned device pointer and keeps its scratch in the file-scope
// array below, so it calls no cudaMalloc, cudaFree or allocating library routine.
//
// Scratch: g_static_scratch, 8 MiB of doubles, allocated by the CUDA module when
// the library is loaded and held by every GPU that loads the library until the
// process exits. It holds the reference-element tables of every (problem, degree)
// (uploaded once per device), an error flag, the per-CTA partial sums and the
// reduced result of the current call. Every call shares it and it keeps the last
// call's contents; each call clears the flag and overwrites the rest before it
// reads it, but calls whose GPU work overlaps (different streams, or different
// host threads, on the same device) race on it and must be serialised by the
// caller.
//
// Set-up: the first call on each device looks up the device address of the array
// with cudaGetSymbolAddress (with that device current), caches it, and copies the
// reference tables into the array with a synchronous cudaMemcpy. Later calls
// launch kernels only.
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

constexpr size_t kStaticScratchDoubles = (size_t)1 << 20;  // 8 MiB
constexpr int kStaticMaxDevices = 64;
constexpr int kStaticWarps = 2;
constexpr int kStaticMaxK = 64;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

size_t up32(size_t n) { return (n + 31) & ~size_t(31); }

// Reference tables of every (problem, degree) packed as the element kernels read
// them (D | B | Lt | fw | qw | qxi), one 32-double-aligned region each, built once
// in host memory that lives until exit. off[problem][p] is the region's start.
struct StaticTables {
  bool ok = false;
  std::vector<double> data;
  size_t off[3][4] = {};
};

const StaticTables& static_tables() {
  static StaticTables st;
  static std::once_flag once;
  std::call_once(once, [] {
    for (int problem : {IFT_BURGERS1D, IFT_EULER2D})
      for (int p = 1; p <= 3; ++p) {
        RefTables R;
        if (!build_tables(problem == IFT_BURGERS1D ? 1 : 2, p, R)) return;
        std::vector<double>& t = st.data;
        st.off[problem][p] = t.size();
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
        t.resize(up32(t.size()), 0.0);
      }
    st.ok = true;
  });
  return st;
}

// Scratch layout (doubles): [tables | flag (32) | result (up32(nacc)) | partials (grid x nacc)].
size_t static_flag_offset() { return static_tables().data.size(); }

std::mutex g_static_mu;
double* g_static_ptr[kStaticMaxDevices] = {nullptr};

// Device address of the static scratch on the current device. The first call on a
// device looks it up and copies the reference tables into it (synchronously).
cudaError_t static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_ptr[dev] == nullptr) {
    const StaticTables& st = static_tables();
    if (!st.ok) return cudaErrorInvalidValue;
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(p, st.data.data(), st.data.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

// Checks what the element kernel will index with, for every listed element (all
// elements when elems is NULL): the element id, its vertex ids and its neighbour
// ids, and the weight (finite, >= 0). Sets *flag = 1 on the first violation; the
// assembly and the reduction then return at once and the outputs become NaN.
__global__ void static_check_kernel(long items, int64_t n_elems, int64_t n_verts, int nv, int nf,
                                    const int32_t* elems, const double* rho, const int32_t* ev, const int32_t* nbr,
                                    int* flag) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < items; i += (long)gridDim.x * blockDim.x) {
    bool bad = false;
    long e = i;
    if (elems) {
      e = elems[i];
      const double r = rho[i];
      bad = !(r >= 0.0 && r <= 1.79e308);
    }
    if (e < 0 || e >= n_elems) {
      bad = true;
    } else {
      for (int v = 0; v < nv; ++v) {
        const long iv = ev[e * nv + v];
        bad |= iv < 0 || iv >= n_verts;
      }
      for (int f = 0; f < nf; ++f) bad |= nbr[e * nf + f] >= n_elems;
    }
    if (bad) atomicOr(flag, 1);
  }
}

__global__ void static_unpack_kernel(const double* res, const int* flag, int ku, int kx, double* S, double* T,
                                     double* H, double* J) {
  const int k = ku + kx;
  const bool bad = *flag != 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k * k + k + 1; i += gridDim.x * blockDim.x) {
    const double v = bad ? NAN : res[i];
    if (i < k * k) {
      if (H) H[i] = v;
    } else if (i < k * k + ku) {
      if (S) S[i - k * k] = v;
    } else if (i < k * k + k) {
      if (T) T[i - k * k - ku] = v;
    } else if (J) {
      J[0] = bad ? NAN : (res[k * k + k + 1] > 0.0 ? INFINITY : res[k * k + k]);
    }
  }
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
  if (n_verts < 1 || n_elems < 1 || n_elems > ((int64_t)1 << 30) || n_verts > ((int64_t)1 << 30))
    return IFT_ERR_ARG;
  if (k_u < 1 || k_x < 0 || k_u + k_x > kStaticMaxK) return IFT_ERR_ARG;
  if (!X || !elem_verts || !nbr || !nbr_face || !bc || !Phi || (k_x > 0 && (!Psi || !z)) || !mu || !y)
    return IFT_ERR_ARG;
  if (nnz == 0 || nnz < -1 || nnz > ((int64_t)1 << 30) || (nnz > 0 && (!elems || !rho))) return IFT_ERR_ARG;
  const KernelSet ks = (problem == IFT_BURGERS1D) ? burgers_kernels(p, 0) : euler_kernels(p, 0);
  if (!ks.valid) return IFT_ERR_NOTIMPL;
  const StaticTables& st = static_tables();
  if (!st.ok) return IFT_ERR_ARG;
  const int k = k_u + k_x;
  const int nacc = k * k + k + 2;
  const size_t o_flag = static_flag_offset();
  const size_t o_res = o_flag + 32;
  const size_t o_part = o_res + up32(nacc);
  if (o_part + (size_t)nacc > kStaticScratchDoubles) return IFT_ERR_ARG;  // k too large for the scratch
  const size_t max_grid = (kStaticScratchDoubles - o_part) / nacc;

  double* scratch = nullptr;
  if (static_scratch(&scratch) != cudaSuccess) return IFT_ERR_CUDA;
  int* flag = (int*)(scratch + o_flag);
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

  const int nv = problem == IFT_BURGERS1D ? 2 : 3, nf = nv;
  if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) return IFT_ERR_CUDA;
  long cgrid = (items + 255) / 256;
  if (cgrid > (long)sms * 8) cgrid = (long)sms * 8;
  static_check_kernel<<<(int)cgrid, 256, 0, s>>>(items, n_elems, n_verts, nv, nf, nnz > 0 ? elems : nullptr,
                                                 nnz > 0 ? rho : nullptr, elem_verts, nbr, flag);
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
  a.tables = scratch + st.off[problem][p];
  a.gamma = gamma;
  a.kappa = kappa;
  a.eps = eps_g;
  a.partial = scratch + o_part;
  a.skip = flag;
  a.contraction = 0;
  a.need_hn = 0;
  if (ks.assemble(&a, true, (int)grid, block, smem, s) != cudaSuccess) return IFT_ERR_CUDA;
  reduce_partials_kernel<<<(nacc + 31) / 32, 256, 0, s>>>(scratch + o_part, (int)grid, nacc, scratch + o_res, flag);
  static_unpack_kernel<<<(nacc + 255) / 256, 256, 0, s>>>(scratch + o_res, flag, k_u, k_x, S, T, H, J);
  if (cudaGetLastError() != cudaSuccess) return IFT_ERR_CUDA;
  return IFT_OK;
}
