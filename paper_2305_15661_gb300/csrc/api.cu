// C ABI of the EQP-IFT GB300 library (declared in include/ift.h).
//
// The context owns every device buffer: mesh and connectivity, bases, weights,
// reference tables, per-CTA partial sums, the reduced result and the solver
// state. The solve is a CUDA graph whose while-loop body is
// [assemble at the trial point -> reduce the CTA partials -> LM step]; the LM
// step kernel sets the loop condition, so a whole solve is one graph launch.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "syrk_tc.h"
#include "../../include/ift.h"
#include "elem.cuh"
#include "kernels.h"
#include "lm.cuh"
#include "refelem.h"

namespace ift {
__global__ void lm_step_kernel(LMState* sp, const double* res, LMConsts c, unsigned long long cond_handle,
                               int use_cond);
__global__ void lm_init_kernel(LMState* sp, const double* w0, const double* tau0, int ku, int kx, int phase);
__global__ void reduce_partials_kernel(const double* partial, int nparts, int nacc, double* out, const int* skip);
__global__ void phit_u_partial_kernel(const double* Phi, long Nu, int ku, int m, int problem, double gamma,
                                      const double* mu, long chunk, double* part);
__global__ void sum_columns_kernel(const double* part, int nparts, int ku, double* w);
__global__ void lm_step_batched_kernel(LMState* states, const double* res, int nacc, LMConsts c);
__global__ void batch_condition_kernel(const LMState* states, int B, int* active, unsigned long long cond_handle,
                                       int use_cond);
__global__ void reduce_chunks_kernel(const double* partial, const int* qchunk, int nacc, const LMState* states,
                                     double* res, int skip_kept);
__global__ void lm_init_batched_kernel(LMState* states, int B, int ku, int kx, int m, int problem, double gamma,
                                       const double* mu, int mustride, const double* colsum, const double* y0,
                                       const double* z0, int phase);
__global__ void phi_colsum_kernel(const double* Phi, long Nu, int ku, int m, double* colsum);
__global__ void geo32_kernel(const double* X, const int* ev, const double* Psi, int kx, long n_elems, float4* out);
__global__ void lm_restart_kernel(LMState* states, int B, int ku, int kx);
__global__ void residual_norms_finish_kernel(const double* part, int B, int nchunk, double* norms);
__global__ void merge_grad_kernel(const double* g, int k, int nacc, double* res, const LMState* states);
__global__ void dot_partial_kernel(const double* a, const double* b, long n, double* part);
__global__ void axpy_kernel(long n, double alpha, const double* x, double* y);
__global__ void scatter_free_kernel(const int* idx, int nfree, const double* v, double* x);
__global__ void cg_start_kernel(long n, int ku, const double* g, const double* diag, const CGState* st, double* d,
                                double* r, double* z, double* p, double* part, const int* off, const int* slots,
                                double* xdir);
__global__ void cg_start_finish_kernel(const double* part, int nblk, CGState* st);
__global__ void cg_update_kernel(long n, int ku, const double* pap_part, int nblk, CGState* st, const double* p,
                                 const double* Ap, const double* diag, double* d, double* r, double* z,
                                 double* part);
__global__ void align_finish_kernel(const double* part, int nparts, int ku, const double* H, const double* p,
                                    int nfree, const double* yslot, const int* off, const int* slots,
                                    const CGState* st, double* Ap, double* dotpart);
__global__ void cg_beta_kernel(const double* part, int nblk, CGState* st, unsigned long long cond_handle,
                               int use_cond);
__global__ void cg_dir_kernel(long n, int ku, const CGState* st, const double* z, double* p, const int* off,
                              const int* slots, double* xdir);
__global__ void take_free_kernel(int nfree, const double* yslot, const int* off, const int* slots, double* out);
__global__ void align_wrows_kernel(const double* part, int nparts, int ku, const double* H, const double* dw,
                                   int mode, double* out);
}  // namespace ift

using namespace ift;

namespace {

// A named range for profilers (NVTX) around each public call that launches work.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace

namespace {

constexpr int kWarpsPerCta = 2;  // default warps per CTA of the element kernels
constexpr int kChunk = 8;        // default elements per chunk of the batched path
constexpr int kPhitBlocks = 256;
thread_local std::string g_create_error;

// Unpack [H | g | J | count] into separate outputs; J = +inf if any element was non-physical.
__global__ void unpack_kernel(const double* res, int ku, int kx, double* S, double* T, double* H, double* J) {
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

}  // namespace

struct ift_ctx {
  ift_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  RefTables T;
  int dim = 1, m = 1, nv = 2, nb = 0, nu = 0, nup = 0, nxe = 0, nface = 0, ntrace = 0, nq = 0, nfq = 0;
  KernelSet ks[2];  // element kernels: [0] FP64, [1] FP32 (FP32 and mixed contexts)
  int sm_count = 0;
  int smem_optin = 0;  // largest dynamic shared memory a CTA may opt into
  double* d_tables = nullptr;
  // mesh
  bool have_mesh = false;
  int64_t n_verts = 0, n_elems = 0;
  double* d_X = nullptr;
  int* d_ev = nullptr;
  int* d_nbr = nullptr;
  int* d_nbrf = nullptr;
  signed char* d_bc = nullptr;
  // bases
  bool have_bases = false;
  int ku = 0, kx = 0;
  double* d_Phi = nullptr;
  float* d_Phi32 = nullptr;
  float4* d_geo32 = nullptr;  // FP32 edge table of straight-sided triangles (FP32 contexts)
  // FP32 contexts with BF16 contraction: the transposed BF16 stack of sqrt(rho_e) A_e
  // rows (k rows of at_ld values) the tensor-core product reads, and its status word
  uint16_t* d_at = nullptr;
  long at_ld = 0, at_rows = 0;
  int* d_tc_status = nullptr;
  double* d_Psi = nullptr;
  // weights
  int64_t nnz = -1;
  int* d_elems = nullptr;
  double* d_rho = nullptr;
  // work buffers
  double* d_mu = nullptr;       // 4
  double* d_w = nullptr;        // LM_KMAX
  double* d_tau = nullptr;      // LM_KMAX
  double* d_res = nullptr;      // nacc
  double* d_partial = nullptr;  // max_parts * nacc
  int max_parts = 0;
  double* d_phit = nullptr;     // kPhitBlocks * LM_KMAX
  LMState* d_lm = nullptr;
  // launch plans of the element kernels, [working precision][0: objective only, 1: fused assembly]
  int plan_grid[2][2] = {{0, 0}, {0, 0}};
  size_t plan_smem[2][2] = {{0, 0}, {0, 0}};
  int plan_grid_grad = 0;    // the FP64 gradient pass (its own shared-memory layout)
  size_t plan_smem_grad = 0;
  int plan_epoch[2] = {-1, -1};
  // launch shapes (set by ift_autotune): warps per CTA of the single-query and the
  // batched element kernels, elements per chunk of the batched path
  int wpc[2] = {kWarpsPerCta, kWarpsPerCta}, bwpc[2] = {kWarpsPerCta, kWarpsPerCta}, chunk = kChunk;
  // batched queries (per-query weight sets split into chunks)
  std::vector<int64_t> h_offsets;  // host copy of the per-query offsets (to re-chunk)
  int B = 0;
  int n_chunks = 0;
  int* d_chunk_start = nullptr;
  int* d_chunk_query = nullptr;
  int* d_qchunk = nullptr;
  int* d_belems = nullptr;
  double* d_brho = nullptr;
  double* d_bmu = nullptr;
  double* d_bw = nullptr;
  double* d_bres = nullptr;
  double* d_bpartial = nullptr;
  LMState* d_blm = nullptr;
  int* d_active = nullptr;
  double* d_colsum = nullptr;
  // HDM residual norms (greedy-search indicator): points, parameters, chunk partials, norms
  double* d_rn_pts = nullptr;
  double* d_rn_mu = nullptr;
  double* d_rn_part = nullptr;
  double* d_rn_norms = nullptr;
  size_t rn_cap_B = 0, rn_cap_parts = 0;
  int bplan_grid[2][2] = {{0, 0}, {0, 0}};
  size_t bplan_smem[2][2] = {{0, 0}, {0, 0}};
  int bplan_grid_grad = 0;
  size_t bplan_smem_grad = 0;
  int bplan_epoch[2] = {-1, -1};
  cudaGraph_t bgraph[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t bgraph_exec[4] = {nullptr, nullptr, nullptr, nullptr};
  int bgraph_epoch[4] = {-1, -1, -1, -1};
  // FP64 gradient pass results: [g | J | count] for the single query (k + 2) and per query (B x (k + 2))
  double* d_gres = nullptr;
  double* d_bgres = nullptr;
  // solve graphs, per working precision
  // solve graphs per body kind: [0] FP64, [1] FP32, [2] FP32 Jacobians + FP64 gradient
  cudaGraph_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t graph_exec[4] = {nullptr, nullptr, nullptr, nullptr};
  int graph_epoch[4] = {-1, -1, -1, -1};
  int epoch = 0;
  bool graph_failed = false;

  ift_status fail(ift_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return st;
  }
  ift_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // the status is returned here; leave no error behind for the caller's next CUDA call
    return fail(e == cudaErrorMemoryAllocation ? IFT_ERR_OOM : IFT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  }
  int nacc() const { return (ku + kx) * (ku + kx) + ku + kx + 2; }
  // working precision of the evaluation calls: FP64 contexts 0, FP32 and mixed contexts 1
  int eval_wp() const { return cfg.precision == IFT_FP64 ? 0 : 1; }
  // body kind of an evaluation call: FP64, FP32, or FP32 Jacobians with the FP64 gradient
  int eval_slot() const { return cfg.precision == IFT_FP32_JACOBIAN ? 2 : eval_wp(); }
};

#define CK(call, what)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return c->cuda_fail(e_, what); \
  } while (0)

namespace {

template <class P>
void dfree(P*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

template <class P>
cudaError_t dalloc(P*& p, size_t n) {
  dfree(p);
  return cudaMalloc((void**)&p, n * sizeof(P));
}

void drop_graph(ift_ctx* c) {
  for (int wp = 0; wp < 4; ++wp) {
    if (c->graph_exec[wp]) cudaGraphExecDestroy(c->graph_exec[wp]);
    if (c->graph[wp]) cudaGraphDestroy(c->graph[wp]);
    c->graph_exec[wp] = nullptr;
    c->graph[wp] = nullptr;
    c->graph_epoch[wp] = -1;
  }
}

// Fill the kernel arguments for the configured precision (or FP64 if force64).
template <class TT>
AsmArgs<TT> make_args(ift_ctx* c, const TT* Phi, const double* w, const double* tau, const double* mu, bool dense,
                      const int* skip) {
  AsmArgs<TT> a;
  a.X = c->d_X;
  a.ev = c->d_ev;
  a.nbr = c->d_nbr;
  a.nbr_face = c->d_nbrf;
  a.bc = c->d_bc;
  a.Phi = Phi;
  a.Psi = c->d_Psi;
  a.ku = c->ku;
  a.kx = c->kx;
  if (dense || c->nnz < 0) {
    a.elems = nullptr;
    a.rho = nullptr;
    a.n_items = c->n_elems;
  } else {
    a.elems = c->d_elems;
    a.rho = c->d_rho;
    a.n_items = c->nnz;
  }
  a.w = w;
  a.tau = tau;
  a.mu = mu;
  a.tables = c->d_tables;
  a.gamma = c->cfg.gamma;
  a.kappa = c->cfg.kappa;
  a.eps = c->cfg.eps_g;
  a.partial = c->d_partial;
  a.skip = skip;
  a.contraction = c->cfg.contraction;
  a.need_hn = 0;
  a.geo32 = c->d_geo32;
  return a;
}

// Grid and shared memory of the element kernels for the current bases and
// weights: as many CTAs as fit on the GPU at once, but no more than the items
// need; the shape is fixed per configuration, so sums are reproducible.
// Dynamic shared memory of the fused element kernel of precision wp for w warps per CTA.
size_t shapes_smem(const ift_ctx* c, int wp, int w) {
  return c->ks[wp].valid ? c->ks[wp].smem_bytes_fused(true, c->ku, c->kx, w) : 0;
}

// Warps of the fused element kernel of precision wp resident per SM with w warps per CTA
// (0 if a CTA does not fit).
int resident_warps(ift_ctx* c, int wp, int w) {
  if (!c->ks[wp].valid) return 0;
  const size_t smem = shapes_smem(c, wp, w);
  if (smem > (size_t)c->smem_optin) return 0;
  if (c->ks[wp].prepare(true, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return w * c->ks[wp].blocks_per_sm(true, 32 * w, smem);
}

ift_status plan_launch(ift_ctx* c, int wp) {
  const KernelSet& ks = c->ks[wp];
  const int wpc = c->wpc[wp], block = 32 * wpc;
  const long items = (c->nnz < 0) ? c->n_elems : c->nnz;
  for (int j = 0; j < 2; ++j) {
    const bool jac = j == 1;
    const size_t smem = ks.smem_bytes_fused(jac, c->ku, c->kx, wpc);
    if (smem > (size_t)c->smem_optin)
      return c->fail(IFT_ERR_ARG, "%d warps per CTA need %zu bytes of shared memory (at most %d)", wpc, smem,
                     c->smem_optin);
    cudaError_t e = ks.prepare(jac, smem);
    if (e != cudaSuccess) return c->cuda_fail(e, "kernel attributes");
    const int bps = ks.blocks_per_sm(jac, block, smem);
    if (bps < 1) return c->fail(IFT_ERR_CUDA, "element kernel does not fit on an SM (%zu bytes shared)", smem);
    long grid = (long)c->sm_count * bps;
    const long need = (items + wpc - 1) / wpc;
    if (grid > need) grid = need;
    if (grid > c->max_parts) grid = c->max_parts;
    if (grid < 1) grid = 1;
    c->plan_grid[wp][j] = (int)grid;
    c->plan_smem[wp][j] = smem;
  }
  if (ks.smem_bytes_grad) {
    // the gradient pass: same warps per CTA, its own (smaller) layout and occupancy
    const size_t smem = ks.smem_bytes_grad(c->ku, c->kx, wpc);
    const int bps = smem <= (size_t)c->smem_optin ? ks.blocks_per_sm_grad(false, block, smem) : 0;
    if (bps < 1) return c->fail(IFT_ERR_CUDA, "gradient kernel does not fit on an SM (%zu bytes shared)", smem);
    long grid = (long)c->sm_count * bps;
    const long need = (items + wpc - 1) / wpc;
    if (grid > need) grid = need;
    if (grid > c->max_parts) grid = c->max_parts;
    if (grid < 1) grid = 1;
    c->plan_grid_grad = (int)grid;
    c->plan_smem_grad = smem;
  }
  // FP32 with BF16 contraction: the stack of the tensor-core product (zero past the
  // items' rows), sized for the current items; allocated here, before any capture
  const int kk = c->ku + c->kx;
  if (wp == 1 && c->cfg.contraction == IFT_CONTRACT_BF16 && c->nu % 2 == 0 && kk <= 64) {
    const long rows = (long)items * c->nu;
    const long ld = syrk_tc_rows(rows);
    if (!c->d_at || c->at_ld != ld) {
      CK(dalloc(c->d_at, (size_t)kk * ld), "alloc tensor-core stack");
      CK(cudaMemset(c->d_at, 0, (size_t)kk * ld * sizeof(uint16_t)), "clear tensor-core stack");
      c->at_ld = ld;
    }
    c->at_rows = rows;
    if (!c->d_tc_status) {
      CK(dalloc(c->d_tc_status, 1), "alloc status");
      CK(cudaMemset(c->d_tc_status, 0, sizeof(int)), "clear status");
    }
    CK(syrk_tc_prepare(), "tensor-core product attributes");
  } else {
    c->at_rows = 0;
  }
  // the inspection kernel shares the fused kernel's attribute; make sure it covers its layout
  const size_t ismem = ks.smem_bytes(true, 1, 0, wpc);
  if (ismem > c->plan_smem[wp][1]) {
    cudaError_t e = ks.prepare(true, ismem);
    if (e != cudaSuccess) return c->cuda_fail(e, "kernel attributes");
  }
  c->plan_epoch[wp] = c->epoch;
  return IFT_OK;
}

// Launch the element pass (jac: fused assembly, else objective only) in working
// precision wp and the partial reduction into out.
ift_status launch_assemble(ift_ctx* c, int wp, bool jac, const double* w, const double* tau, const double* mu,
                           double* out, const int* skip, cudaStream_t s) {
  if (c->plan_epoch[wp] != c->epoch) {
    ift_status st = plan_launch(c, wp);
    if (st != IFT_OK) return st;
  }
  const KernelSet& ks = c->ks[wp];
  const int block = 32 * c->wpc[wp];
  const int grid = c->plan_grid[wp][jac ? 1 : 0];
  const size_t smem = c->plan_smem[wp][jac ? 1 : 0];
  cudaError_t e;
  const bool tc_stack = wp == 1 && jac && c->at_rows > 0;
  if (wp == 1) {
    AsmArgs<float> a = make_args<float>(c, c->d_Phi32, w, tau, mu, false, skip);
    if (tc_stack) {
      a.at_out = reinterpret_cast<uint32_t*>(c->d_at);
      a.at_ld = c->at_ld;
    }
    e = ks.assemble(&a, jac, grid, block, smem, s);
  } else {
    AsmArgs<double> a = make_args<double>(c, c->d_Phi, w, tau, mu, false, skip);
    e = ks.assemble(&a, jac, grid, block, smem, s);
  }
  if (e != cudaSuccess) return c->cuda_fail(e, "element kernel launch");
  const int nacc = c->nacc();
  int nparts = grid;
  if (tc_stack) {
    // H from the stack on the tensor cores: its partial rows follow the element CTAs'
    int ctas = 0;
    e = syrk_tc_launch(c->d_at, c->at_ld, c->at_rows, c->ku + c->kx, std::min(2 * c->sm_count, c->max_parts - grid),
                       c->d_partial + (size_t)grid * nacc, nacc, skip, c->d_tc_status, &ctas, s);
    if (e != cudaSuccess) return c->cuda_fail(e, "tensor-core product launch");
    nparts += ctas;
  }
  reduce_partials_kernel<<<(nacc + 31) / 32, 1024, 0, s>>>(c->d_partial, nparts, nacc, out, skip);
  e = cudaGetLastError();
  if (e != cudaSuccess) return c->cuda_fail(e, "reduce launch");
  return IFT_OK;
}

// After a synchronised evaluation or solve: IFT_ERR_TIMEOUT (and the word cleared)
// if the tensor-core product recorded a bounded wait that ran out.
ift_status tc_status_check(ift_ctx* c) {
  if (!c->d_tc_status) return IFT_OK;
  int tcs = 0;
  CK(cudaMemcpy(&tcs, c->d_tc_status, sizeof(int), cudaMemcpyDeviceToHost), "status");
  if (tcs == 0) return IFT_OK;
  cudaMemset(c->d_tc_status, 0, sizeof(int));
  return c->fail(IFT_ERR_TIMEOUT, "the tensor-core product timed out waiting for its operands");
}

// The FP64 gradient pass at (w, tau): S~, T~, J~ and the non-physical count into
// the [g | J | count] part of out (the H part is left as it is). states (optional):
// the solve's LM state, whose flags say whether the FP32 pass ran in this body.
ift_status launch_grad(ift_ctx* c, const double* w, const double* tau, const double* mu, double* out,
                       const int* skip, cudaStream_t s, const LMState* states = nullptr) {
  if (c->plan_epoch[0] != c->epoch) {
    ift_status st = plan_launch(c, 0);
    if (st != IFT_OK) return st;
  }
  const KernelSet& ks = c->ks[0];
  const int k = c->ku + c->kx, grid = c->plan_grid_grad;
  AsmArgs<double> a = make_args<double>(c, c->d_Phi, w, tau, mu, false, skip);
  cudaError_t e = ks.assemble_grad(&a, grid, 32 * c->wpc[0], c->plan_smem_grad, s);
  if (e != cudaSuccess) return c->cuda_fail(e, "gradient pass launch");
  reduce_partials_kernel<<<(k + 2 + 31) / 32, 1024, 0, s>>>(c->d_partial, grid, k + 2, c->d_gres, skip);
  merge_grad_kernel<<<1, 64, 0, s>>>(c->d_gres, k, c->nacc(), out, states);
  e = cudaGetLastError();
  if (e != cudaSuccess) return c->cuda_fail(e, "gradient reduce launch");
  return IFT_OK;
}

// Evaluation for a loop body or an evaluation call: slot 0/1 the FP64 / FP32 fused
// assembly; slot 2 the FP32 fused assembly (H) followed by the FP64 gradient pass;
// slot 3 as slot 2, with the FP32 pass (and its reduction) skipped while the LM state
// keeps H (hskip: its flag; states: the LM state).
ift_status launch_eval(ift_ctx* c, int slot, const double* w, const double* tau, const double* mu, double* out,
                       const int* skip, cudaStream_t s, const int* hskip = nullptr,
                       const LMState* states = nullptr) {
  if (slot < 2) return launch_assemble(c, slot, true, w, tau, mu, out, skip, s);
  ift_status st = launch_assemble(c, 1, true, w, tau, mu, out, slot == 3 ? hskip : skip, s);
  if (st != IFT_OK) return st;
  return launch_grad(c, w, tau, mu, out, skip, s, slot == 3 ? states : nullptr);
}

ift_status check_ready(ift_ctx* c) {
  if (!c) return IFT_ERR_ARG;
  if (!c->have_mesh || !c->have_bases) return c->fail(IFT_ERR_STATE, "set_mesh and set_bases must come first");
  return IFT_OK;
}

}  // namespace

extern "C" {

void ift_config_default(ift_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->problem = IFT_EULER2D;
  cfg->q = 1;
  cfg->p = 2;
  cfg->precision = IFT_FP64;
  cfg->gamma = 1.4;
  cfg->kappa = 0.0;
  cfg->eps_g = 1e-8;
  cfg->tol = 1e-8;
  cfg->max_iters = 200;
  cfg->lm_init = IFT_INIT_PAPER;
  cfg->contraction = IFT_CONTRACT_FP;
  cfg->align_cg_tol = 1e-12;
}

const char* ift_create_error(void) { return g_create_error.c_str(); }

ift_status ift_create(const ift_config* cfg, void* stream, ift_ctx** out) {
  g_create_error.clear();
  if (!cfg || !out) {
    g_create_error = "null argument";
    return IFT_ERR_ARG;
  }
  *out = nullptr;
  if (cfg->problem != IFT_BURGERS1D && cfg->problem != IFT_EULER2D) {
    g_create_error = "unknown problem";
    return IFT_ERR_ARG;
  }
  if (cfg->p < 1 || cfg->p > 3) {
    g_create_error = "degree p must be 1, 2 or 3";
    return IFT_ERR_ARG;
  }
  if (cfg->q != 1 && !(cfg->q == 2 && cfg->problem == IFT_EULER2D)) {
    g_create_error = "geometry degree q must be 1, or 2 for IFT_EULER2D";
    return IFT_ERR_ARG;
  }
  if (cfg->precision != IFT_FP64 && cfg->precision != IFT_FP32 && cfg->precision != IFT_MIXED &&
      cfg->precision != IFT_FP32_JACOBIAN) {
    g_create_error = "precision must be IFT_FP64, IFT_FP32, IFT_MIXED or IFT_FP32_JACOBIAN";
    return IFT_ERR_ARG;
  }
  if (cfg->contraction != IFT_CONTRACT_FP && cfg->contraction != IFT_CONTRACT_TF32 &&
      cfg->contraction != IFT_CONTRACT_3XTF32 && cfg->contraction != IFT_CONTRACT_BF16) {
    g_create_error = "contraction must be IFT_CONTRACT_FP, _TF32, _3XTF32 or _BF16";
    return IFT_ERR_ARG;
  }
  if (!(cfg->align_cg_tol >= 0.0 && cfg->align_cg_tol < 1.0)) {
    g_create_error = "align_cg_tol must lie in [0, 1)";
    return IFT_ERR_ARG;
  }
  if (cfg->max_loop_bodies < 0) {
    g_create_error = "max_loop_bodies must be >= 0";
    return IFT_ERR_ARG;
  }
  if (cfg->contraction != IFT_CONTRACT_FP && cfg->precision == IFT_FP64) {
    g_create_error = "tensor-core contraction needs IFT_FP32 or IFT_MIXED";
    return IFT_ERR_ARG;
  }
  if (!(cfg->gamma > 1.0) || !(cfg->kappa >= 0.0) || !(cfg->eps_g > 0.0) || !(cfg->tol >= 0.0) ||
      cfg->max_iters < 0 || (cfg->lm_init != IFT_INIT_PAPER && cfg->lm_init != IFT_INIT_GIVEN)) {
    g_create_error = "bad configuration value";
    return IFT_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return IFT_ERR_CUDA;
  }
  ift_ctx* c = new ift_ctx();
  c->cfg = *cfg;
  const int dim = (cfg->problem == IFT_BURGERS1D) ? 1 : 2;
  if (!build_tables(dim, cfg->p, c->T)) {
    delete c;
    g_create_error = "reference element construction failed";
    return IFT_ERR_ARG;
  }
  c->dim = dim;
  c->m = (dim == 1) ? 1 : 4;
  c->nv = (cfg->q == 2) ? 6 : dim + 1;
  c->nb = c->T.nb;
  c->nu = c->nb * c->m;
  c->nface = c->T.nface;
  c->ntrace = c->T.ntrace;
  c->nup = c->nface * c->ntrace * c->m;
  c->nxe = c->nv * dim;
  c->nq = c->T.nq;
  c->nfq = c->T.nfq;
  auto kernels_for = [&](int prec) {
    if (dim == 1) return burgers_kernels(cfg->p, prec);
    return cfg->q == 2 ? euler_curved_kernels(cfg->p, prec) : euler_kernels(cfg->p, prec);
  };
  c->ks[0] = kernels_for(0);
  if (cfg->precision != IFT_FP64) c->ks[1] = kernels_for(1);
  if (!c->ks[0].valid || (cfg->precision != IFT_FP64 && !c->ks[1].valid)) {
    delete c;
    g_create_error = "kernels for this problem/degree/precision are not built";
    return IFT_ERR_NOTIMPL;
  }
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      g_create_error = std::string("stream: ") + cudaGetErrorString(e);
      return IFT_ERR_CUDA;
    }
    c->own_stream = true;
  }
  // reference tables, packed D | B | Lt | fw | qw | qxi (see elem.cuh Tabs)
  std::vector<double> tab;
  tab.insert(tab.end(), c->T.D.begin(), c->T.D.end());
  tab.insert(tab.end(), c->T.B.begin(), c->T.B.end());
  tab.insert(tab.end(), c->T.Lt.begin(), c->T.Lt.end());
  tab.insert(tab.end(), c->T.fw.begin(), c->T.fw.end());
  tab.insert(tab.end(), c->T.qw.begin(), c->T.qw.end());
  if (dim == 1) {
    tab.insert(tab.end(), c->T.qxi.begin(), c->T.qxi.end());
  } else {
    tab.insert(tab.end(), (size_t)c->nq, 0.0);  // 2-D kernels do not read the 1-D point table
  }
  if (cfg->q == 2) {  // curved: the geometry shape-function derivatives (see refelem.h)
    std::vector<double> gdv, gtf;
    build_curved_tables(c->T, gdv, gtf);
    tab.insert(tab.end(), gdv.begin(), gdv.end());
    tab.insert(tab.end(), gtf.begin(), gtf.end());
  }
  c->max_parts = c->sm_count * 32;
  bool ok = dalloc(c->d_tables, tab.size()) == cudaSuccess &&
            cudaMemcpy(c->d_tables, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            dalloc(c->d_mu, 4) == cudaSuccess && dalloc(c->d_w, LM_KMAX) == cudaSuccess &&
            dalloc(c->d_tau, LM_KMAX) == cudaSuccess && dalloc(c->d_phit, (size_t)kPhitBlocks * LM_KMAX) == cudaSuccess &&
            dalloc(c->d_lm, 1) == cudaSuccess;
  if (ok) {
    cudaMemset(c->d_w, 0, LM_KMAX * 8);
    cudaMemset(c->d_tau, 0, LM_KMAX * 8);
    cudaMemset(c->d_mu, 0, 4 * 8);
    cudaMemset(c->d_lm, 0, sizeof(LMState));
  }
  if (!ok) {
    g_create_error = "device allocation failed";
    ift_destroy(c);
    return IFT_ERR_OOM;
  }
  *out = c;
  return IFT_OK;
}

ift_status ift_destroy(ift_ctx* c) {
  if (!c) return IFT_ERR_ARG;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  dfree(c->d_tables);
  dfree(c->d_X);
  dfree(c->d_ev);
  dfree(c->d_nbr);
  dfree(c->d_nbrf);
  dfree(c->d_bc);
  dfree(c->d_Phi);
  dfree(c->d_Phi32);
  dfree(c->d_geo32);
  dfree(c->d_at);
  dfree(c->d_tc_status);
  dfree(c->d_Psi);
  dfree(c->d_elems);
  dfree(c->d_rho);
  dfree(c->d_mu);
  dfree(c->d_w);
  dfree(c->d_tau);
  dfree(c->d_res);
  dfree(c->d_partial);
  dfree(c->d_phit);
  dfree(c->d_lm);
  for (int wp = 0; wp < 4; ++wp) {
    if (c->bgraph_exec[wp]) cudaGraphExecDestroy(c->bgraph_exec[wp]);
    if (c->bgraph[wp]) cudaGraphDestroy(c->bgraph[wp]);
  }
  dfree(c->d_gres);
  dfree(c->d_bgres);
  dfree(c->d_chunk_start);
  dfree(c->d_chunk_query);
  dfree(c->d_qchunk);
  dfree(c->d_belems);
  dfree(c->d_brho);
  dfree(c->d_bmu);
  dfree(c->d_bw);
  dfree(c->d_bres);
  dfree(c->d_bpartial);
  dfree(c->d_blm);
  dfree(c->d_active);
  dfree(c->d_colsum);
  dfree(c->d_rn_pts);
  dfree(c->d_rn_mu);
  dfree(c->d_rn_part);
  dfree(c->d_rn_norms);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return IFT_OK;
}

const char* ift_last_error(const ift_ctx* c) { return c ? c->err.c_str() : "null context"; }

ift_status ift_sizes(const ift_ctx* c, int64_t* s) {
  if (!c || !s) return IFT_ERR_ARG;
  s[0] = c->nb;
  s[1] = c->nu;
  s[2] = c->nup;
  s[3] = c->nxe;
  s[4] = c->nface;
  s[5] = c->ntrace;
  s[6] = c->nq;
  s[7] = c->nfq;
  return IFT_OK;
}

ift_status ift_reference_nodes(const ift_ctx* c, double* nodes, int32_t* face_nodes) {
  if (!c) return IFT_ERR_ARG;
  if (nodes) std::memcpy(nodes, c->T.nodes.data(), c->T.nodes.size() * sizeof(double));
  if (face_nodes)
    for (size_t i = 0; i < c->T.face_nodes.size(); ++i) face_nodes[i] = c->T.face_nodes[i];
  return IFT_OK;
}

ift_status ift_set_mesh(ift_ctx* c, int64_t n_verts, const double* X, int64_t n_elems, const int32_t* ev) {
  if (!c) return IFT_ERR_ARG;
  if (n_verts < c->nv || n_elems < 1 || !X || !ev) return c->fail(IFT_ERR_ARG, "empty mesh or null pointer");
  if (n_elems > (int64_t)1 << 30 || n_verts > (int64_t)1 << 30) return c->fail(IFT_ERR_ARG, "mesh too large");
  const int dim = c->dim, nv = c->nv, nf = c->nface;
  for (int64_t i = 0; i < n_elems * nv; ++i)
    if (ev[i] < 0 || ev[i] >= n_verts) return c->fail(IFT_ERR_ARG, "vertex index out of range in element %lld",
                                                      (long long)(i / nv));
  for (int64_t e = 0; e < n_elems; ++e) {
    const int32_t* v = &ev[e * nv];
    double det;
    if (dim == 1) {
      det = X[v[1]] - X[v[0]];
    } else {
      det = (X[2 * v[1]] - X[2 * v[0]]) * (X[2 * v[2] + 1] - X[2 * v[0] + 1]) -
            (X[2 * v[2]] - X[2 * v[0]]) * (X[2 * v[1] + 1] - X[2 * v[0] + 1]);
    }
    if (!(det > 0.0)) return c->fail(IFT_ERR_ARG, "element %lld is inverted or degenerate", (long long)e);
  }
  // faces matched by their vertex set
  std::vector<int> nbr(n_elems * nf, -1), nbrf(n_elems * nf, -1);
  std::vector<signed char> bc(n_elems * nf, 0);
  std::unordered_map<uint64_t, int64_t> open_faces;
  open_faces.reserve((size_t)n_elems * nf);
  for (int64_t e = 0; e < n_elems; ++e)
    for (int k = 0; k < nf; ++k) {
      uint64_t key;
      if (dim == 1) {
        key = (uint64_t)(uint32_t)ev[e * 2 + k];
      } else {
        uint32_t a = (uint32_t)ev[e * nv + k], b = (uint32_t)ev[e * nv + (k + 1) % 3];
        key = ((uint64_t)(a < b ? a : b) << 32) | (uint64_t)(a < b ? b : a);
      }
      auto it = open_faces.find(key);
      if (it == open_faces.end()) {
        open_faces.emplace(key, e * nf + k);
      } else {
        const int64_t other = it->second;
        if (other < 0) return c->fail(IFT_ERR_ARG, "a face is shared by more than two elements");
        const int64_t e2 = other / nf;
        const int k2 = (int)(other % nf);
        if (dim == 1 && k2 == k) return c->fail(IFT_ERR_ARG, "1-D elements must run left to right");
        nbr[e * nf + k] = (int)e2;
        nbrf[e * nf + k] = k2;
        nbr[e2 * nf + k2] = (int)e;
        nbrf[e2 * nf + k2] = k;
        it->second = -1;
      }
    }
  for (int64_t i = 0; i < n_elems * nf; ++i)
    if (nbr[i] < 0) bc[i] = (dim == 1) ? ((i % nf == 0) ? 1 : 2) : 1;
  drop_graph(c);
  c->have_mesh = false;
  c->have_bases = false;
  c->nnz = -1;
  CK(dalloc(c->d_X, (size_t)n_verts * dim), "alloc X");
  CK(dalloc(c->d_ev, (size_t)n_elems * nv), "alloc elements");
  CK(dalloc(c->d_nbr, (size_t)n_elems * nf), "alloc neighbours");
  CK(dalloc(c->d_nbrf, (size_t)n_elems * nf), "alloc neighbours");
  CK(dalloc(c->d_bc, (size_t)n_elems * nf), "alloc boundary types");
  CK(cudaMemcpy(c->d_X, X, (size_t)n_verts * dim * 8, cudaMemcpyHostToDevice), "copy X");
  CK(cudaMemcpy(c->d_ev, ev, (size_t)n_elems * nv * 4, cudaMemcpyHostToDevice), "copy elements");
  CK(cudaMemcpy(c->d_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice), "copy neighbours");
  CK(cudaMemcpy(c->d_nbrf, nbrf.data(), nbrf.size() * 4, cudaMemcpyHostToDevice), "copy neighbours");
  CK(cudaMemcpy(c->d_bc, bc.data(), bc.size(), cudaMemcpyHostToDevice), "copy boundary types");
  c->n_verts = n_verts;
  c->n_elems = n_elems;
  c->have_mesh = true;
  c->epoch++;
  return IFT_OK;
}

ift_status ift_set_bases(ift_ctx* c, int64_t N_u, int k_u, const double* Phi, int64_t N_x, int k_x,
                         const double* Psi) {
  if (!c) return IFT_ERR_ARG;
  if (!c->have_mesh) return c->fail(IFT_ERR_STATE, "set_mesh must come first");
  if (N_u != c->n_elems * c->nu) return c->fail(IFT_ERR_ARG, "N_u must be n_elems * n_u = %lld",
                                                (long long)(c->n_elems * c->nu));
  if (N_x != c->n_verts * c->dim) return c->fail(IFT_ERR_ARG, "N_x must be n_verts * dim = %lld",
                                                 (long long)(c->n_verts * c->dim));
  if (k_u < 1 || k_x < 0 || k_u + k_x > LM_KMAX) return c->fail(IFT_ERR_ARG, "need k_u >= 1, k_x >= 0, k_u + k_x <= %d",
                                                              LM_KMAX);
  if (!Phi || (k_x > 0 && !Psi)) return c->fail(IFT_ERR_ARG, "null basis pointer");
  drop_graph(c);
  c->have_bases = false;
  CK(dalloc(c->d_Phi, (size_t)N_u * k_u), "alloc Phi");
  CK(cudaMemcpy(c->d_Phi, Phi, (size_t)N_u * k_u * 8, cudaMemcpyHostToDevice), "copy Phi");
  if (c->cfg.precision != IFT_FP64) {
    std::vector<float> p32((size_t)N_u * k_u);
    for (size_t i = 0; i < p32.size(); ++i) p32[i] = (float)Phi[i];
    CK(dalloc(c->d_Phi32, p32.size()), "alloc Phi (FP32)");
    CK(cudaMemcpy(c->d_Phi32, p32.data(), p32.size() * 4, cudaMemcpyHostToDevice), "copy Phi (FP32)");
  }
  CK(dalloc(c->d_Psi, (size_t)N_x * (k_x > 0 ? k_x : 1)), "alloc Psi");
  if (k_x > 0) CK(cudaMemcpy(c->d_Psi, Psi, (size_t)N_x * k_x * 8, cudaMemcpyHostToDevice), "copy Psi");
  dfree(c->d_geo32);
  if (c->cfg.precision != IFT_FP64 && c->dim == 2 && c->nv == 3) {
    // straight-sided triangles: the FP32 element pass takes its geometry from this table
    CK(dalloc(c->d_geo32, (size_t)c->n_elems * (1 + k_x)), "alloc edge table");
    const long g = std::min<long>((c->n_elems + 255) / 256, 4096);
    geo32_kernel<<<(int)(g > 0 ? g : 1), 256, 0, c->stream>>>(c->d_X, c->d_ev, c->d_Psi, k_x, c->n_elems,
                                                             c->d_geo32);
    CK(cudaGetLastError(), "edge table");
  }
  c->ku = k_u;
  c->kx = k_x;
  const int nacc = c->nacc();
  CK(dalloc(c->d_res, nacc), "alloc result");
  CK(dalloc(c->d_partial, (size_t)c->max_parts * nacc), "alloc partials");
  CK(dalloc(c->d_colsum, (size_t)4 * k_u), "alloc column sums");
  CK(dalloc(c->d_gres, (size_t)nacc), "alloc gradient result");
  phi_colsum_kernel<<<k_u, 256, 0, c->stream>>>(c->d_Phi, (long)N_u, k_u, c->m, c->d_colsum);
  CK(cudaGetLastError(), "column sums");
  CK(cudaStreamSynchronize(c->stream), "column sums");
  c->B = 0;  // batched weight sets are sized for the bases: set them again
  c->have_bases = true;
  // default launch shapes for these bases: the warps per CTA (at most the default)
  // that keep the most warps resident per SM; large k need fewer warps per CTA,
  // both to fit and because shared memory is handed out CTA by CTA
  for (int wp = 0; wp < 2; ++wp) {
    int best = 1, best_res = -1;
    for (int w = kWarpsPerCta; w >= 1; w /= 2) {
      const int res = resident_warps(c, wp, w);
      if (res > best_res) {
        best = w;
        best_res = res;
      }
    }
    c->wpc[wp] = c->bwpc[wp] = best;
  }
  c->epoch++;
  return IFT_OK;
}

ift_status ift_set_eq_weights(ift_ctx* c, int64_t nnz, const int32_t* elem, const double* rho) {
  if (!c) return IFT_ERR_ARG;
  if (!c->have_mesh) return c->fail(IFT_ERR_STATE, "set_mesh must come first");
  drop_graph(c);
  c->epoch++;
  if (nnz < 0) {
    c->nnz = -1;
    return IFT_OK;
  }
  if (nnz == 0) return c->fail(IFT_ERR_ARG, "an empty weight set has no objective");
  if (!elem || !rho) return c->fail(IFT_ERR_ARG, "null weight pointer");
  std::vector<char> seen(c->n_elems, 0);
  for (int64_t i = 0; i < nnz; ++i) {
    if (elem[i] < 0 || elem[i] >= c->n_elems) return c->fail(IFT_ERR_ARG, "weight element out of range");
    if (seen[elem[i]]) return c->fail(IFT_ERR_ARG, "element %d listed twice", elem[i]);
    seen[elem[i]] = 1;
    if (!(rho[i] > 0.0) || !std::isfinite(rho[i])) return c->fail(IFT_ERR_ARG, "weights must be positive and finite");
  }
  CK(dalloc(c->d_elems, (size_t)nnz), "alloc weights");
  CK(dalloc(c->d_rho, (size_t)nnz), "alloc weights");
  CK(cudaMemcpy(c->d_elems, elem, (size_t)nnz * 4, cudaMemcpyHostToDevice), "copy weights");
  CK(cudaMemcpy(c->d_rho, rho, (size_t)nnz * 8, cudaMemcpyHostToDevice), "copy weights");
  c->nnz = nnz;
  return IFT_OK;
}

ift_status ift_reduced_residual_jacobian_dev(ift_ctx* c, const double* mu, const double* y, const double* z,
                                             double* S, double* T, double* H, double* J, void* stream) {
  NvtxRange nvtx_range("ift_reduced_residual_jacobian_dev");
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (!mu || !y || (c->kx > 0 && !z)) return c->fail(IFT_ERR_ARG, "null input pointer");
  cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
  st = launch_eval(c, c->eval_slot(), y, c->kx > 0 ? z : c->d_tau, mu, c->d_res, nullptr, s);
  if (st != IFT_OK) return st;
  const int nacc = c->nacc();
  unpack_kernel<<<(nacc + 255) / 256, 256, 0, s>>>(c->d_res, c->ku, c->kx, S, T, H, J);
  CK(cudaGetLastError(), "unpack launch");
  return IFT_OK;
}

ift_status ift_reduced_residual_jacobian(ift_ctx* c, const double* mu, const double* y, const double* z, double* S,
                                         double* T, double* H, double* J) {
  NvtxRange nvtx_range("ift_reduced_residual_jacobian");
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (!mu || !y || (c->kx > 0 && !z)) return c->fail(IFT_ERR_ARG, "null input pointer");
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(c->d_mu, mu, (c->dim == 1 ? 1 : 2) * 8, cudaMemcpyHostToDevice, s), "copy mu");
  CK(cudaMemcpyAsync(c->d_w, y, c->ku * 8, cudaMemcpyHostToDevice, s), "copy y");
  if (c->kx > 0) CK(cudaMemcpyAsync(c->d_tau, z, c->kx * 8, cudaMemcpyHostToDevice, s), "copy z");
  st = launch_eval(c, c->eval_slot(), c->d_w, c->d_tau, c->d_mu, c->d_res, nullptr, s);
  if (st != IFT_OK) return st;
  const int nacc = c->nacc(), k = c->ku + c->kx;
  std::vector<double> res(nacc);
  CK(cudaMemcpyAsync(res.data(), c->d_res, nacc * 8, cudaMemcpyDeviceToHost, s), "copy result");
  CK(cudaStreamSynchronize(s), "assembly");
  st = tc_status_check(c);
  if (st != IFT_OK) return st;
  if (H) std::memcpy(H, res.data(), (size_t)k * k * 8);
  if (S) std::memcpy(S, res.data() + k * k, c->ku * 8);
  if (T && c->kx > 0) std::memcpy(T, res.data() + k * k + c->ku, c->kx * 8);
  const bool bad = res[k * k + k + 1] > 0.0;
  if (J) J[0] = bad ? INFINITY : res[k * k + k];
  if (bad) return c->fail(IFT_ERR_NONPHYSICAL, "%d elements are non-physical at this point", (int)res[k * k + k + 1]);
  return IFT_OK;
}

ift_status ift_element_eval(ift_ctx* c, const double* mu, const double* U, const double* x, int64_t n,
                            const int32_t* elems, double* R, double* JU, double* JUp, double* Jx, double* N,
                            double* dN) {
  NvtxRange nvtx_range("ift_element_eval");
  if (!c) return IFT_ERR_ARG;
  if (!c->have_mesh) return c->fail(IFT_ERR_STATE, "set_mesh must come first");
  if (!mu || !U || !x || !elems || n < 1) return c->fail(IFT_ERR_ARG, "bad inspection arguments");
  for (int64_t i = 0; i < n; ++i)
    if (elems[i] < 0 || elems[i] >= c->n_elems) return c->fail(IFT_ERR_ARG, "element out of range");
  const int nu = c->nu, nup = c->nup, nxe = c->nxe, nd = nu + nup + nxe;
  const size_t Nu = (size_t)c->n_elems * nu, Nx = (size_t)c->n_verts * c->dim;
  double *dU = nullptr, *dx = nullptr, *dR = nullptr, *dJ = nullptr, *dNn = nullptr, *ddN = nullptr;
  int* dl = nullptr;
  auto cleanup = [&]() {
    dfree(dU);
    dfree(dx);
    dfree(dR);
    dfree(dJ);
    dfree(dNn);
    dfree(ddN);
    dfree(dl);
  };
  cudaError_t e = cudaSuccess;
  if ((e = dalloc(dU, Nu)) != cudaSuccess || (e = dalloc(dx, Nx)) != cudaSuccess ||
      (e = dalloc(dR, (size_t)n * nu)) != cudaSuccess || (e = dalloc(dJ, (size_t)n * nu * nd)) != cudaSuccess ||
      (e = dalloc(dNn, (size_t)n)) != cudaSuccess || (e = dalloc(ddN, (size_t)n * nxe)) != cudaSuccess ||
      (e = dalloc(dl, (size_t)n)) != cudaSuccess) {
    cleanup();
    return c->cuda_fail(e, "inspection buffers");
  }
  cudaStream_t s = c->stream;
  cudaMemcpyAsync(dU, U, Nu * 8, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dx, x, Nx * 8, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dl, elems, (size_t)n * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(c->d_mu, mu, (c->dim == 1 ? 1 : 2) * 8, cudaMemcpyHostToDevice, s);
  const int wp = c->eval_wp();
  const KernelSet& ks = c->ks[wp];
  const int wpc = c->wpc[wp], block = 32 * wpc;
  const size_t smem = ks.smem_bytes(true, 1, 0, wpc);
  e = ks.prepare(true, c->have_bases && c->plan_smem[wp][1] > smem ? c->plan_smem[wp][1] : smem);
  if (e == cudaSuccess) {
    const int grid = (int)((n + wpc - 1) / wpc);
    if (wp == 1) {
      AsmArgs<float> a = make_args<float>(c, c->d_Phi32, c->d_w, c->d_tau, c->d_mu, true, nullptr);
      a.ku = 1;
      a.kx = 0;
      a.elems = dl;
      a.n_items = n;
      e = ks.inspect(&a, dU, dx, dR, dJ, dNn, ddN, grid, block, smem, s);
    } else {
      AsmArgs<double> a = make_args<double>(c, c->d_Phi, c->d_w, c->d_tau, c->d_mu, true, nullptr);
      a.ku = 1;
      a.kx = 0;
      a.elems = dl;
      a.n_items = n;
      e = ks.inspect(&a, dU, dx, dR, dJ, dNn, ddN, grid, block, smem, s);
    }
  }
  std::vector<double> hR((size_t)n * nu), hJ((size_t)n * nu * nd), hN(n), hdN((size_t)n * nxe);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hR.data(), dR, hR.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hJ.data(), dJ, hJ.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hN.data(), dNn, hN.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hdN.data(), ddN, hdN.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return c->cuda_fail(e, "element inspection");
  for (int64_t i = 0; i < n; ++i) {
    for (int r = 0; r < nu; ++r) {
      const double* row = &hJ[((size_t)i * nu + r) * nd];
      if (JU) std::memcpy(&JU[((size_t)i * nu + r) * nu], row, nu * 8);
      if (JUp) std::memcpy(&JUp[((size_t)i * nu + r) * nup], row + nu, nup * 8);
      if (Jx) std::memcpy(&Jx[((size_t)i * nu + r) * nxe], row + nu + nup, nxe * 8);
    }
  }
  if (R) std::memcpy(R, hR.data(), hR.size() * 8);
  if (N) std::memcpy(N, hN.data(), hN.size() * 8);
  if (dN) std::memcpy(dN, hdN.data(), hdN.size() * 8);
  return IFT_OK;
}

}  // extern "C"

namespace {

// Starting point of a solve: paper initialisation (w0 = Phi^T U_guess(mu), tau = 0,
// w-only phase first) or the caller's (y, z) (joint phase only).
ift_status solve_prologue(ift_ctx* c, const double* d_mu, const double* d_y0, const double* d_z0, cudaStream_t s) {
  const int ku = c->ku, kx = c->kx;
  if (c->cfg.lm_init == IFT_INIT_PAPER) {
    const long Nu = (long)c->n_elems * c->nu;
    const long chunk = (Nu + kPhitBlocks - 1) / kPhitBlocks;
    int block = 256;
    if (block < ku) block = ku;
    phit_u_partial_kernel<<<kPhitBlocks, block, block * sizeof(double), s>>>(
        c->d_Phi, Nu, ku, c->m, c->cfg.problem, c->cfg.gamma, d_mu, chunk, c->d_phit);
    sum_columns_kernel<<<1, 64, 0, s>>>(c->d_phit, kPhitBlocks, ku, c->d_w);
    CK(cudaMemsetAsync(c->d_tau, 0, LM_KMAX * 8, s), "zero tau");
    lm_init_kernel<<<1, 64, 0, s>>>(c->d_lm, c->d_w, c->d_tau, ku, kx, 0);
  } else {
    lm_init_kernel<<<1, 64, 0, s>>>(c->d_lm, d_y0, kx > 0 ? d_z0 : nullptr, ku, kx, 1);
  }
  CK(cudaGetLastError(), "solve prologue");
  return IFT_OK;
}

// Stage 1 of a mixed-precision solve: FP32 iterations until this relative optimality,
// or until FP32 rounding in J stalls the line search (the first trial step that
// needs a second halving ends the stage), then FP64 iterations finish from that
// point. Measured on GB300 against caps of 2, 4 and 8 halvings: 1 was fastest on
// every workload (256 config-3 queries 1,156 -> 1,403 solves/s, 4,096 warm-started
// queries 5,049 -> 5,344) with the same converged set.
constexpr double kMixedStage1Tol = 1e-6;
constexpr int kMaxHalvings = 30, kMixedStage1Halvings = 1;

LMConsts lm_consts(ift_ctx* c, double tol) {
  LMConsts k;
  k.keep_h = 0;
  k.tol = tol;
  k.max_iters = c->cfg.max_iters;
  k.ku = c->ku;
  k.kx = c->kx;
  k.body_limit = c->cfg.max_loop_bodies > 0 ? c->cfg.max_loop_bodies : (2 * c->cfg.max_iters + 4) * 34;
  k.max_halvings = kMaxHalvings;
  return k;
}

// Tolerance of the LM run in working precision wp: the final tolerance, except for
// the FP32 stage of a mixed-precision solve.
double stage_tol(ift_ctx* c, int wp) {
  return (c->cfg.precision == IFT_MIXED && wp == 1) ? std::max(c->cfg.tol, kMixedStage1Tol) : c->cfg.tol;
}

LMConsts stage_consts(ift_ctx* c, int wp) {
  LMConsts k = lm_consts(c, stage_tol(c, wp));
  if (c->cfg.precision == IFT_MIXED && wp == 1) k.max_halvings = kMixedStage1Halvings;
  return k;
}

// LM constants of a loop body in evaluation slot 0..3 (slots 2 and 3 run the LM with
// the FP64 constants; slot 3 keeps H after full steps).
LMConsts slot_consts(ift_ctx* c, int slot) {
  LMConsts k = stage_consts(c, slot >= 2 ? 0 : slot);
  k.keep_h = slot == 3 ? 1 : 0;
  return k;
}

// The loop body: assemble at the trial point, reduce, LM step.
// slot 0/1: FP64 / FP32 assembly; slot 2: FP32 assembly for H, then the FP64
// gradient pass for S~, T~, J~ (the LM runs with the FP64 constants); slot 3: as
// slot 2, the FP32 pass skipped while H is kept (the finishing stage of a mixed solve).
ift_status enqueue_body(ift_ctx* c, int slot, cudaStream_t s, unsigned long long handle, int use_cond) {
  double* trial = (double*)((char*)c->d_lm + offsetof(LMState, trial));
  const int* done = (const int*)((char*)c->d_lm + offsetof(LMState, done));
  const int* hkeep = (const int*)((char*)c->d_lm + offsetof(LMState, hkeep));
  ift_status st = launch_eval(c, slot, trial, trial + c->ku, c->d_mu, c->d_res, done, s, hkeep, c->d_lm);
  if (st != IFT_OK) return st;
  lm_step_kernel<<<1, 32, 0, s>>>(c->d_lm, c->d_res, slot_consts(c, slot), handle, use_cond);
  CK(cudaGetLastError(), "LM step launch");
  return IFT_OK;
}

// A while-loop graph whose body is produced by enqueue(stream, handle).
template <class F>
ift_status build_while_graph(ift_ctx* c, cudaGraph_t* out_graph, cudaGraphExec_t* out_exec, F enqueue) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0), "graph create");
  *out_graph = g;
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault), "conditional handle");
  // the parameter struct holds a union without a default constructor: build it in zeroed storage
  alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
  std::memset(pbuf, 0, sizeof(pbuf));
  cudaGraphNodeParams* p = reinterpret_cast<cudaGraphNodeParams*>(pbuf);
  p->type = cudaGraphNodeTypeConditional;
  p->conditional.handle = h;
  p->conditional.type = cudaGraphCondTypeWhile;
  p->conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, p), "while node");
  cudaGraph_t body = p->conditional.phGraph_out[0];
  cudaStream_t cs = nullptr;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return c->cuda_fail(e, "begin capture");
  }
  ift_status st = enqueue(cs, (unsigned long long)h);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cs, &captured);
  cudaStreamDestroy(cs);
  if (st != IFT_OK) return st;
  if (e != cudaSuccess) return c->cuda_fail(e, "end capture");
  CK(cudaGraphInstantiate(out_exec, g, 0), "graph instantiate");
  return IFT_OK;
}

// Build (once per configuration) the solve graph of working precision wp: one while
// node whose body is the loop body above, the LM step kernel setting the condition.
ift_status build_graph(ift_ctx* c, int wp) {
  if (c->graph_exec[wp]) cudaGraphExecDestroy(c->graph_exec[wp]);
  if (c->graph[wp]) cudaGraphDestroy(c->graph[wp]);
  c->graph_exec[wp] = nullptr;
  c->graph[wp] = nullptr;
  for (int tp = 0; tp < 2; ++tp) {
    if ((tp == wp || wp >= 2) && c->plan_epoch[tp] != c->epoch) {
      ift_status st = plan_launch(c, tp);
      if (st != IFT_OK) return st;
    }
  }
  ift_status st = build_while_graph(c, &c->graph[wp], &c->graph_exec[wp], [&](cudaStream_t cs, unsigned long long h) {
    return enqueue_body(c, wp, cs, h, 1);
  });
  if (st != IFT_OK) return st;
  c->graph_epoch[wp] = c->epoch;
  return IFT_OK;
}

// Host-driven loop over the same body (no graph): used when IFT_SOLVE_NO_GRAPH is set,
// e.g. so that a profiler that does not enter conditional graph nodes sees every launch.
// Bodies are enqueued in groups of 8; after a group the done flag is read back.
ift_status run_solve_loop(ift_ctx* c, int wp, cudaStream_t s) {
  const LMConsts k = lm_consts(c, stage_tol(c, wp >= 2 ? 0 : wp));
  const int* done = (const int*)((char*)c->d_lm + offsetof(LMState, done));
  for (int b = 0; b <= k.body_limit; b += 8) {
    for (int j = 0; j < 8; ++j) {
      ift_status st = enqueue_body(c, wp, s, 0ull, 0);
      if (st != IFT_OK) return st;
    }
    int h = 0;
    CK(cudaMemcpyAsync(&h, done, sizeof(int), cudaMemcpyDeviceToHost, s), "read done flag");
    CK(cudaStreamSynchronize(s), "solve loop");
    if (h) return IFT_OK;
  }
  return IFT_OK;
}

ift_status run_stage(ift_ctx* c, int wp, cudaStream_t s) {
  static const bool no_graph = getenv("IFT_SOLVE_NO_GRAPH") != nullptr;
  if (no_graph) return run_solve_loop(c, wp, s);
  if (c->graph_epoch[wp] != c->epoch || !c->graph_exec[wp]) {
    ift_status st = build_graph(c, wp);
    if (st != IFT_OK) return st;
  }
  CK(cudaGraphLaunch(c->graph_exec[wp], s), "graph launch");
  return IFT_OK;
}

// The whole solve after the prologue: one stage in the context's precision, or for
// mixed precision an FP32 stage to the stage-1 tolerance followed by an FP64 stage
// restarted (joint phase) at the FP32 stage's final point.
ift_status run_solve(ift_ctx* c, cudaStream_t s) {
  if (c->cfg.precision == IFT_FP64) return run_stage(c, 0, s);
  if (c->cfg.precision == IFT_FP32_JACOBIAN) return run_stage(c, 2, s);
  ift_status st = run_stage(c, 1, s);
  if (st != IFT_OK || c->cfg.precision == IFT_FP32) return st;
  lm_restart_kernel<<<1, 64, 0, s>>>(c->d_lm, 1, c->ku, c->kx);
  CK(cudaGetLastError(), "stage restart");
  // the finishing stage: FP64 residual, gradient and objective, H from FP32 (kept
  // across full steps)
  return run_stage(c, 3, s);
}

void fill_info(const LMState& st, ift_solve_info* info, int ku, int kx) {
  if (!info) return;
  info->status = st.status;
  info->init_iters = st.iters[0];
  info->iters = st.iters[1];
  info->trials = st.trials;
  info->shifts = st.shifts;
  info->J = st.J;
  double ns = 0.0, nt = 0.0;
  for (int i = 0; i < ku; ++i) ns += st.g[i] * st.g[i];
  for (int i = 0; i < kx; ++i) nt += st.g[ku + i] * st.g[ku + i];
  info->normS = std::sqrt(ns);
  info->normT = std::sqrt(nt);
  info->g0 = st.g0;
  info->fp32_iters = st.iters32;
  info->fp32_trials = st.trials32;
  info->h_evals = st.hevals;
}

}  // namespace

extern "C" {

ift_status ift_solve_rom(ift_ctx* c, const double* mu, double* y, double* z, ift_solve_info* info) {
  NvtxRange nvtx_range("ift_solve_rom");
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (!mu || !y || (c->kx > 0 && !z)) return c->fail(IFT_ERR_ARG, "null argument");
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(c->d_mu, mu, (c->dim == 1 ? 1 : 2) * 8, cudaMemcpyHostToDevice, s), "copy mu");
  if (c->cfg.lm_init == IFT_INIT_GIVEN) {
    CK(cudaMemcpyAsync(c->d_w, y, c->ku * 8, cudaMemcpyHostToDevice, s), "copy y");
    if (c->kx > 0) CK(cudaMemcpyAsync(c->d_tau, z, c->kx * 8, cudaMemcpyHostToDevice, s), "copy z");
  }
  st = solve_prologue(c, c->d_mu, c->d_w, c->d_tau, s);
  if (st != IFT_OK) return st;
  st = run_solve(c, s);
  if (st != IFT_OK) return st;
  LMState hs;
  CK(cudaMemcpyAsync(&hs, c->d_lm, sizeof(LMState), cudaMemcpyDeviceToHost, s), "copy state");
  CK(cudaStreamSynchronize(s), "solve");
  for (int i = 0; i < c->ku; ++i) y[i] = hs.z[i];
  for (int i = 0; i < c->kx; ++i) z[i] = hs.z[c->ku + i];
  fill_info(hs, info, c->ku, c->kx);
  st = tc_status_check(c);
  if (st != IFT_OK) return st;
  return (ift_status)hs.status;
}

ift_status ift_solve_rom_dev(ift_ctx* c, const double* mu, double* y, double* z, ift_solve_info* info_host,
                             void* stream) {
  NvtxRange nvtx_range("ift_solve_rom_dev");
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (!mu || !y || (c->kx > 0 && !z)) return c->fail(IFT_ERR_ARG, "null argument");
  cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
  CK(cudaMemcpyAsync(c->d_mu, mu, (c->dim == 1 ? 1 : 2) * 8, cudaMemcpyDeviceToDevice, s), "copy mu");
  if (c->cfg.lm_init == IFT_INIT_GIVEN) {
    CK(cudaMemcpyAsync(c->d_w, y, c->ku * 8, cudaMemcpyDeviceToDevice, s), "copy y");
    if (c->kx > 0) CK(cudaMemcpyAsync(c->d_tau, z, c->kx * 8, cudaMemcpyDeviceToDevice, s), "copy z");
  }
  st = solve_prologue(c, c->d_mu, c->d_w, c->d_tau, s);
  if (st != IFT_OK) return st;
  st = run_solve(c, s);
  if (st != IFT_OK) return st;
  const double* zsrc = (const double*)((char*)c->d_lm + offsetof(LMState, z));
  CK(cudaMemcpyAsync(y, zsrc, c->ku * 8, cudaMemcpyDeviceToDevice, s), "copy y");
  if (c->kx > 0) CK(cudaMemcpyAsync(z, zsrc + c->ku, c->kx * 8, cudaMemcpyDeviceToDevice, s), "copy z");
  if (info_host) {
    LMState hs;
    CK(cudaMemcpyAsync(&hs, c->d_lm, sizeof(LMState), cudaMemcpyDeviceToHost, s), "copy state");
    CK(cudaStreamSynchronize(s), "solve");
    fill_info(hs, info_host, c->ku, c->kx);
    st = tc_status_check(c);
    if (st != IFT_OK) return st;
    return (ift_status)hs.status;
  }
  return IFT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched queries: many parameter values, each with its own sparse weight set,
// assembled by one launch over query chunks and solved by one graph.
// ---------------------------------------------------------------------------
namespace {

ift_status plan_batched(ift_ctx* c, int wp) {
  const KernelSet& ks = c->ks[wp];
  const int bwpc = c->bwpc[wp], block = 32 * bwpc;
  for (int j = 0; j < 2; ++j) {
    const bool jac = j == 1;
    const size_t smem = ks.smem_bytes_fused(jac, c->ku, c->kx, bwpc);
    if (smem > (size_t)c->smem_optin)
      return c->fail(IFT_ERR_ARG, "%d warps per CTA need %zu bytes of shared memory (at most %d)", bwpc, smem,
                     c->smem_optin);
    cudaError_t e = ks.prepare_batched(jac, smem);
    if (e != cudaSuccess) return c->cuda_fail(e, "batched kernel attributes");
    const int bps = ks.blocks_per_sm_batched(jac, block, smem);
    if (bps < 1) return c->fail(IFT_ERR_CUDA, "batched kernel does not fit on an SM (%zu bytes shared)", smem);
    long grid = (long)c->sm_count * bps;
    const long need = (c->n_chunks + bwpc - 1) / bwpc;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    c->bplan_grid[wp][j] = (int)grid;
    c->bplan_smem[wp][j] = smem;
  }
  if (ks.smem_bytes_grad) {
    const size_t smem = ks.smem_bytes_grad(c->ku, c->kx, bwpc);
    const int bps = smem <= (size_t)c->smem_optin ? ks.blocks_per_sm_grad(true, block, smem) : 0;
    if (bps < 1) return c->fail(IFT_ERR_CUDA, "batched gradient kernel does not fit on an SM (%zu bytes shared)", smem);
    long grid = (long)c->sm_count * bps;
    const long need = (c->n_chunks + bwpc - 1) / bwpc;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    c->bplan_grid_grad = (int)grid;
    c->bplan_smem_grad = smem;
  }
  c->bplan_epoch[wp] = c->epoch;
  return IFT_OK;
}

// Batched element pass over all chunks of unfinished queries, then the per-query reduction.
ift_status launch_batched(ift_ctx* c, int wp, bool jac, const double* w, long wstride, const int* done,
                          long donestride, const LMState* states, cudaStream_t s, int skip_kept = 0) {
  if (c->bplan_epoch[wp] != c->epoch) {
    ift_status st = plan_batched(c, wp);
    if (st != IFT_OK) return st;
  }
  const KernelSet& ks = c->ks[wp];
  const int block = 32 * c->bwpc[wp];
  const int j = jac ? 1 : 0;
  BatchArgs b;
  b.chunk_start = c->d_chunk_start;
  b.chunk_query = c->d_chunk_query;
  b.n_chunks = c->n_chunks;
  b.w = w;
  b.wstride = wstride;
  b.mu = c->d_bmu;
  b.mustride = 2;
  b.done = done;
  b.donestride = donestride;
  cudaError_t e;
  if (wp == 1) {
    AsmArgs<float> a = make_args<float>(c, c->d_Phi32, w, w + c->ku, c->d_bmu, false, nullptr);
    a.elems = c->d_belems;
    a.rho = c->d_brho;
    a.partial = c->d_bpartial;
    e = ks.assemble_batched(&a, &b, jac, c->bplan_grid[wp][j], block, c->bplan_smem[wp][j], s);
  } else {
    AsmArgs<double> a = make_args<double>(c, c->d_Phi, w, w + c->ku, c->d_bmu, false, nullptr);
    a.elems = c->d_belems;
    a.rho = c->d_brho;
    a.partial = c->d_bpartial;
    e = ks.assemble_batched(&a, &b, jac, c->bplan_grid[wp][j], block, c->bplan_smem[wp][j], s);
  }
  if (e != cudaSuccess) return c->cuda_fail(e, "batched kernel launch");
  reduce_chunks_kernel<<<c->B, 128, 0, s>>>(c->d_bpartial, c->d_qchunk, c->nacc(), states, c->d_bres, skip_kept);
  CK(cudaGetLastError(), "chunk reduction launch");
  return IFT_OK;
}

// The FP64 gradient pass of every unfinished query at its trial point: chunk rows
// of [g | J | count], summed per query and merged into the query's result row.
ift_status launch_batched_grad(ift_ctx* c, const double* w, long wstride, const int* done, long donestride,
                               const LMState* states, cudaStream_t s) {
  if (c->bplan_epoch[0] != c->epoch) {
    ift_status st = plan_batched(c, 0);
    if (st != IFT_OK) return st;
  }
  const int k = c->ku + c->kx;
  BatchArgs b;
  b.chunk_start = c->d_chunk_start;
  b.chunk_query = c->d_chunk_query;
  b.n_chunks = c->n_chunks;
  b.w = w;
  b.wstride = wstride;
  b.mu = c->d_bmu;
  b.mustride = 2;
  b.done = done;
  b.donestride = donestride;
  AsmArgs<double> a = make_args<double>(c, c->d_Phi, w, w + c->ku, c->d_bmu, false, nullptr);
  a.elems = c->d_belems;
  a.rho = c->d_brho;
  a.partial = c->d_bpartial;
  cudaError_t e = c->ks[0].assemble_batched_grad(&a, &b, c->bplan_grid_grad, 32 * c->bwpc[0],
                                                  c->bplan_smem_grad, s);
  if (e != cudaSuccess) return c->cuda_fail(e, "batched gradient pass launch");
  reduce_chunks_kernel<<<c->B, 128, 0, s>>>(c->d_bpartial, c->d_qchunk, k + 2, states, c->d_bgres, 0);
  merge_grad_kernel<<<c->B, 64, 0, s>>>(c->d_bgres, k, c->nacc(), c->d_bres, states);
  CK(cudaGetLastError(), "batched gradient reduce launch");
  return IFT_OK;
}

// The batched loop body in working precision wp: assemble every unfinished query,
// reduce per query, one LM step per query, loop condition.
// slot 0/1: FP64 / FP32 batched assembly; slot 2: FP32 assembly for H, then the FP64
// gradient pass for S~, T~, J~ of every unfinished query; slot 3: as slot 2, the
// FP32 pass skipped for the queries that keep H.
ift_status enqueue_batched_body(ift_ctx* c, int slot, cudaStream_t s, unsigned long long handle, int use_cond) {
  const double* trial = (const double*)((char*)c->d_blm + offsetof(LMState, trial));
  const int* done = (const int*)((char*)c->d_blm + offsetof(LMState, done));
  const int* hkeep = (const int*)((char*)c->d_blm + offsetof(LMState, hkeep));
  const long wstride = (long)(sizeof(LMState) / sizeof(double)), istride = (long)(sizeof(LMState) / sizeof(int));
  const int wp = slot >= 2 ? 1 : slot;
  ift_status st = launch_batched(c, wp, true, trial, wstride, slot == 3 ? hkeep : done, istride, c->d_blm, s,
                                 slot == 3 ? 1 : 0);
  if (st != IFT_OK) return st;
  if (slot >= 2) {
    st = launch_batched_grad(c, trial, wstride, done, istride, c->d_blm, s);
    if (st != IFT_OK) return st;
  }
  lm_step_batched_kernel<<<c->B, 32, 0, s>>>(c->d_blm, c->d_bres, c->nacc(), slot_consts(c, slot));
  batch_condition_kernel<<<1, 256, 0, s>>>(c->d_blm, c->B, c->d_active, handle, use_cond);
  CK(cudaGetLastError(), "batched LM launch");
  return IFT_OK;
}

ift_status build_batched_graph(ift_ctx* c, int wp) {
  if (c->bgraph_exec[wp]) cudaGraphExecDestroy(c->bgraph_exec[wp]);
  if (c->bgraph[wp]) cudaGraphDestroy(c->bgraph[wp]);
  c->bgraph_exec[wp] = nullptr;
  c->bgraph[wp] = nullptr;
  for (int tp = 0; tp < 2; ++tp) {
    if ((tp == wp || wp >= 2) && c->bplan_epoch[tp] != c->epoch) {
      ift_status st = plan_batched(c, tp);
      if (st != IFT_OK) return st;
    }
  }
  ift_status st = build_while_graph(c, &c->bgraph[wp], &c->bgraph_exec[wp],
                                    [&](cudaStream_t cs, unsigned long long h) {
                                      return enqueue_batched_body(c, wp, cs, h, 1);
                                    });
  if (st != IFT_OK) return st;
  c->bgraph_epoch[wp] = c->epoch;
  return IFT_OK;
}

ift_status run_batched_stage(ift_ctx* c, int wp, cudaStream_t s) {
  static const bool no_graph = getenv("IFT_SOLVE_NO_GRAPH") != nullptr;
  if (no_graph) {
    const LMConsts k = lm_consts(c, stage_tol(c, wp >= 2 ? 0 : wp));
    for (int b = 0; b <= k.body_limit; b += 8) {
      for (int j = 0; j < 8; ++j) {
        ift_status st = enqueue_batched_body(c, wp, s, 0ull, 0);
        if (st != IFT_OK) return st;
      }
      int active = 0;
      CK(cudaMemcpyAsync(&active, c->d_active, sizeof(int), cudaMemcpyDeviceToHost, s), "read active count");
      CK(cudaStreamSynchronize(s), "batched solve loop");
      if (!active) return IFT_OK;
    }
    return IFT_OK;
  }
  if (c->bgraph_epoch[wp] != c->epoch || !c->bgraph_exec[wp]) {
    ift_status st = build_batched_graph(c, wp);
    if (st != IFT_OK) return st;
  }
  CK(cudaGraphLaunch(c->bgraph_exec[wp], s), "batched graph launch");
  return IFT_OK;
}

// Mixed solves run the FP32 stage of every query, then the FP64 stage of every
// query. (Moving each query to FP64 on its own, with both kernels in every loop
// body, measured slower on the hyperreduced batch: the second launch and chunk
// scan per body cost more than the overlap of the two stages' tails saved.)
ift_status run_batched_solve(ift_ctx* c, cudaStream_t s) {
  if (c->cfg.precision == IFT_FP64) return run_batched_stage(c, 0, s);
  if (c->cfg.precision == IFT_FP32_JACOBIAN) return run_batched_stage(c, 2, s);
  ift_status st = run_batched_stage(c, 1, s);
  if (st != IFT_OK || c->cfg.precision == IFT_FP32) return st;
  lm_restart_kernel<<<c->B, 64, 0, s>>>(c->d_blm, c->B, c->ku, c->kx);
  CK(cudaGetLastError(), "stage restart");
  // the finishing stage: FP64 residual, gradient and objective, H from FP32 (kept
  // across full steps)
  return run_batched_stage(c, 3, s);
}

// Split every query's items into chunks of c->chunk elements (one warp each) and size
// the chunk partials; called when the weights or the chunk size change.
ift_status rechunk(ift_ctx* c) {
  const int B = c->B;
  std::vector<int> cstart, cquery, qchunk(B + 1);
  for (int q = 0; q < B; ++q) {
    qchunk[q] = (int)cquery.size();
    for (int64_t i = c->h_offsets[q]; i < c->h_offsets[q + 1]; i += c->chunk) {
      cstart.push_back((int)i);
      cquery.push_back(q);
    }
  }
  qchunk[B] = (int)cquery.size();
  cstart.push_back((int)c->h_offsets[B]);
  CK(dalloc(c->d_chunk_start, cstart.size()), "alloc chunks");
  CK(dalloc(c->d_chunk_query, cquery.size()), "alloc chunks");
  CK(dalloc(c->d_qchunk, qchunk.size()), "alloc chunks");
  CK(dalloc(c->d_bpartial, cquery.size() * (size_t)c->nacc()), "alloc chunk partials");
  CK(cudaMemcpy(c->d_chunk_start, cstart.data(), cstart.size() * 4, cudaMemcpyHostToDevice), "copy chunks");
  CK(cudaMemcpy(c->d_chunk_query, cquery.data(), cquery.size() * 4, cudaMemcpyHostToDevice), "copy chunks");
  CK(cudaMemcpy(c->d_qchunk, qchunk.data(), qchunk.size() * 4, cudaMemcpyHostToDevice), "copy chunks");
  c->n_chunks = (int)cquery.size();
  c->epoch++;
  return IFT_OK;
}

ift_status check_batched(ift_ctx* c) {
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (c->B < 1) return c->fail(IFT_ERR_STATE, "ift_set_eq_weights_batched must come first");
  return IFT_OK;
}

// mu rows of the host (B x n_mu) packed as B x 2 on the device
ift_status upload_mu_rows(ift_ctx* c, const double* mu, cudaStream_t s) {
  const int nmu = (c->dim == 1) ? 1 : 2;
  std::vector<double> m2((size_t)c->B * 2, 0.0);
  for (int q = 0; q < c->B; ++q)
    for (int i = 0; i < nmu; ++i) m2[(size_t)q * 2 + i] = mu[(size_t)q * nmu + i];
  CK(cudaMemcpyAsync(c->d_bmu, m2.data(), m2.size() * 8, cudaMemcpyHostToDevice, s), "copy mu");
  CK(cudaStreamSynchronize(s), "copy mu");
  return IFT_OK;
}

}  // namespace

extern "C" {

ift_status ift_set_eq_weights_batched(ift_ctx* c, int B, const int64_t* offsets, const int32_t* elem,
                                      const double* rho) {
  if (!c) return IFT_ERR_ARG;
  if (!c->have_mesh || !c->have_bases) return c->fail(IFT_ERR_STATE, "set_mesh and set_bases must come first");
  if (B < 1 || !offsets || !elem || !rho) return c->fail(IFT_ERR_ARG, "need B >= 1 and non-null arrays");
  if (offsets[0] != 0) return c->fail(IFT_ERR_ARG, "offsets[0] must be 0");
  for (int q = 0; q < B; ++q)
    if (offsets[q + 1] <= offsets[q]) return c->fail(IFT_ERR_ARG, "query %d has no elements", q);
  const int64_t total = offsets[B];
  if (total > ((int64_t)1 << 31) - 1) return c->fail(IFT_ERR_ARG, "too many weight entries");
  std::vector<int> stamp(c->n_elems, -1);
  for (int q = 0; q < B; ++q)
    for (int64_t i = offsets[q]; i < offsets[q + 1]; ++i) {
      if (elem[i] < 0 || elem[i] >= c->n_elems) return c->fail(IFT_ERR_ARG, "weight element out of range");
      if (stamp[elem[i]] == q) return c->fail(IFT_ERR_ARG, "element %d listed twice in query %d", elem[i], q);
      stamp[elem[i]] = q;
      if (!(rho[i] > 0.0) || !std::isfinite(rho[i])) return c->fail(IFT_ERR_ARG, "weights must be positive and finite");
    }
  const int nacc = c->nacc(), k = c->ku + c->kx;
  drop_graph(c);
  c->B = 0;
  CK(dalloc(c->d_belems, (size_t)total), "alloc batched weights");
  CK(dalloc(c->d_brho, (size_t)total), "alloc batched weights");
  CK(dalloc(c->d_bmu, (size_t)B * 2), "alloc mu");
  CK(dalloc(c->d_bw, (size_t)B * k), "alloc points");
  CK(dalloc(c->d_bres, (size_t)B * nacc), "alloc results");
  CK(dalloc(c->d_bgres, (size_t)B * (c->ku + c->kx + 2)), "alloc gradient results");
  CK(dalloc(c->d_blm, (size_t)B), "alloc solver states");
  CK(dalloc(c->d_active, 1), "alloc active count");
  CK(cudaMemcpy(c->d_belems, elem, (size_t)total * 4, cudaMemcpyHostToDevice), "copy weights");
  CK(cudaMemcpy(c->d_brho, rho, (size_t)total * 8, cudaMemcpyHostToDevice), "copy weights");
  CK(cudaMemset(c->d_blm, 0, (size_t)B * sizeof(LMState)), "clear states");
  c->h_offsets.assign(offsets, offsets + B + 1);
  c->B = B;
  return rechunk(c);
}

ift_status ift_reduced_residual_jacobian_batched(ift_ctx* c, const double* mu, const double* y, const double* z,
                                                 double* S, double* T, double* H, double* J) {
  NvtxRange nvtx_range("ift_reduced_residual_jacobian_batched");
  ift_status st = check_batched(c);
  if (st != IFT_OK) return st;
  if (!mu || !y || (c->kx > 0 && !z)) return c->fail(IFT_ERR_ARG, "null input pointer");
  const int B = c->B, ku = c->ku, kx = c->kx, k = ku + kx, nacc = c->nacc();
  cudaStream_t s = c->stream;
  std::vector<double> w((size_t)B * k);
  for (int q = 0; q < B; ++q) {
    for (int i = 0; i < ku; ++i) w[(size_t)q * k + i] = y[(size_t)q * ku + i];
    for (int i = 0; i < kx; ++i) w[(size_t)q * k + ku + i] = z[(size_t)q * kx + i];
  }
  st = upload_mu_rows(c, mu, s);
  if (st != IFT_OK) return st;
  CK(cudaMemcpyAsync(c->d_bw, w.data(), w.size() * 8, cudaMemcpyHostToDevice, s), "copy points");
  st = launch_batched(c, c->eval_wp(), true, c->d_bw, k, nullptr, 0, nullptr, s);
  if (st == IFT_OK && c->eval_slot() == 2) st = launch_batched_grad(c, c->d_bw, k, nullptr, 0, nullptr, s);
  if (st != IFT_OK) return st;
  std::vector<double> res((size_t)B * nacc);
  CK(cudaMemcpyAsync(res.data(), c->d_bres, res.size() * 8, cudaMemcpyDeviceToHost, s), "copy results");
  CK(cudaStreamSynchronize(s), "batched assembly");
  bool bad = false;
  for (int q = 0; q < B; ++q) {
    const double* r = &res[(size_t)q * nacc];
    if (H) std::memcpy(H + (size_t)q * k * k, r, (size_t)k * k * 8);
    if (S) std::memcpy(S + (size_t)q * ku, r + k * k, ku * 8);
    if (T && kx > 0) std::memcpy(T + (size_t)q * kx, r + k * k + ku, kx * 8);
    const bool bq = r[k * k + k + 1] > 0.0;
    if (J) J[q] = bq ? INFINITY : r[k * k + k];
    bad = bad || bq;
  }
  if (bad) return c->fail(IFT_ERR_NONPHYSICAL, "some queries are non-physical at their points");
  return IFT_OK;
}

ift_status ift_solve_rom_batched(ift_ctx* c, const double* mu, double* y, double* z, ift_solve_info* info) {
  NvtxRange nvtx_range("ift_solve_rom_batched");
  ift_status st = check_batched(c);
  if (st != IFT_OK) return st;
  if (!mu || !y || (c->kx > 0 && !z)) return c->fail(IFT_ERR_ARG, "null argument");
  const int B = c->B, ku = c->ku, kx = c->kx;
  cudaStream_t s = c->stream;
  st = upload_mu_rows(c, mu, s);
  if (st != IFT_OK) return st;
  const bool given = c->cfg.lm_init == IFT_INIT_GIVEN;
  if (given) {
    CK(cudaMemcpyAsync(c->d_bw, y, (size_t)B * ku * 8, cudaMemcpyHostToDevice, s), "copy y");
    if (kx > 0) CK(cudaMemcpyAsync(c->d_bw + (size_t)B * ku, z, (size_t)B * kx * 8, cudaMemcpyHostToDevice, s), "copy z");
  }
  lm_init_batched_kernel<<<B, 64, 0, s>>>(c->d_blm, B, ku, kx, c->m, c->cfg.problem, c->cfg.gamma, c->d_bmu, 2,
                                          c->d_colsum, c->d_bw, c->d_bw + (size_t)B * ku, given ? 1 : 0);
  CK(cudaGetLastError(), "batched init");
  st = run_batched_solve(c, s);
  if (st != IFT_OK) return st;
  std::vector<LMState> hs(B);
  CK(cudaMemcpyAsync(hs.data(), c->d_blm, (size_t)B * sizeof(LMState), cudaMemcpyDeviceToHost, s), "copy states");
  CK(cudaStreamSynchronize(s), "batched solve");
  // overall status: OK if every query converged, else the first error, else the first warning
  int first_err = IFT_OK, first_warn = IFT_OK;
  for (int q = 0; q < B; ++q) {
    for (int i = 0; i < ku; ++i) y[(size_t)q * ku + i] = hs[q].z[i];
    for (int i = 0; i < kx; ++i) z[(size_t)q * kx + i] = hs[q].z[ku + i];
    if (info) fill_info(hs[q], &info[q], ku, kx);
    if (hs[q].status < 0 && first_err == IFT_OK) first_err = hs[q].status;
    if (hs[q].status > 0 && first_warn == IFT_OK) first_warn = hs[q].status;
  }
  return (ift_status)(first_err != IFT_OK ? first_err : first_warn);
}

ift_status ift_solve_rom_batched_dev(ift_ctx* c, const double* mu, double* y, double* z, int32_t* status,
                                     void* stream) {
  NvtxRange nvtx_range("ift_solve_rom_batched_dev");
  ift_status st = check_batched(c);
  if (st != IFT_OK) return st;
  if (!mu || !y || (c->kx > 0 && !z)) return c->fail(IFT_ERR_ARG, "null argument");
  const int B = c->B, ku = c->ku, kx = c->kx;
  cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
  const int nmu = (c->dim == 1) ? 1 : 2;
  CK(cudaMemcpy2DAsync(c->d_bmu, 2 * 8, mu, nmu * 8, nmu * 8, B, cudaMemcpyDeviceToDevice, s), "copy mu");
  const bool given = c->cfg.lm_init == IFT_INIT_GIVEN;
  if (given) {
    CK(cudaMemcpyAsync(c->d_bw, y, (size_t)B * ku * 8, cudaMemcpyDeviceToDevice, s), "copy y");
    if (kx > 0) CK(cudaMemcpyAsync(c->d_bw + (size_t)B * ku, z, (size_t)B * kx * 8, cudaMemcpyDeviceToDevice, s), "copy z");
  }
  lm_init_batched_kernel<<<B, 64, 0, s>>>(c->d_blm, B, ku, kx, c->m, c->cfg.problem, c->cfg.gamma, c->d_bmu, 2,
                                          c->d_colsum, c->d_bw, c->d_bw + (size_t)B * ku, given ? 1 : 0);
  CK(cudaGetLastError(), "batched init");
  st = run_batched_solve(c, s);
  if (st != IFT_OK) return st;
  const size_t stride = sizeof(LMState);
  const char* base = (const char*)c->d_blm;
  CK(cudaMemcpy2DAsync(y, ku * 8, base + offsetof(LMState, z), stride, ku * 8, B, cudaMemcpyDeviceToDevice, s),
     "copy y");
  if (kx > 0)
    CK(cudaMemcpy2DAsync(z, kx * 8, base + offsetof(LMState, z) + ku * 8, stride, kx * 8, B,
                         cudaMemcpyDeviceToDevice, s),
       "copy z");
  if (status)
    CK(cudaMemcpy2DAsync(status, sizeof(int), base + offsetof(LMState, status), stride, sizeof(int), B,
                         cudaMemcpyDeviceToDevice, s),
       "copy status");
  return IFT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// HDM residual norms at many points: the greedy-search indicator (Eq. greedy0).
// ---------------------------------------------------------------------------
namespace {

constexpr int kNormChunk = 64;  // elements per warp work item

ift_status launch_residual_norms(ift_ctx* c, int B, const double* d_pts, const double* d_mu, double* d_norms,
                                 cudaStream_t s) {
  const int wp = c->eval_wp();
  const KernelSet& ks = c->ks[wp];
  const int warps = 4, block = 32 * warps;
  const size_t smem = ks.smem_bytes(false, c->ku, c->kx, warps);
  if (smem > (size_t)c->smem_optin) return c->fail(IFT_ERR_ARG, "residual-norm kernel does not fit (%zu bytes)", smem);
  cudaError_t e = ks.prepare_norms(smem);
  if (e != cudaSuccess) return c->cuda_fail(e, "norm kernel attributes");
  const int bps = ks.blocks_per_sm_norms(block, smem);
  if (bps < 1) return c->fail(IFT_ERR_CUDA, "residual-norm kernel does not fit on an SM");
  const int nchunk = (int)((c->n_elems + kNormChunk - 1) / kNormChunk);
  const size_t parts = (size_t)B * nchunk;
  if (parts > c->rn_cap_parts) {
    CK(dalloc(c->d_rn_part, parts), "alloc norm partials");
    c->rn_cap_parts = parts;
  }
  long grid = (long)c->sm_count * bps;
  const long need = ((long)parts + warps - 1) / warps;
  if (grid > need) grid = need;
  const int k = c->ku + c->kx;
  if (wp == 1) {
    AsmArgs<float> a = make_args<float>(c, c->d_Phi32, d_pts, d_pts + c->ku, d_mu, true, nullptr);
    e = ks.residual_norms(&a, d_pts, k, d_mu, 2, B, nchunk, kNormChunk, c->d_rn_part, (int)grid, block, smem, s);
  } else {
    AsmArgs<double> a = make_args<double>(c, c->d_Phi, d_pts, d_pts + c->ku, d_mu, true, nullptr);
    e = ks.residual_norms(&a, d_pts, k, d_mu, 2, B, nchunk, kNormChunk, c->d_rn_part, (int)grid, block, smem, s);
  }
  if (e != cudaSuccess) return c->cuda_fail(e, "residual-norm kernel launch");
  residual_norms_finish_kernel<<<(B + 127) / 128, 128, 0, s>>>(c->d_rn_part, B, nchunk, d_norms);
  CK(cudaGetLastError(), "residual-norm finish");
  return IFT_OK;
}

}  // namespace

extern "C" ift_status ift_hdm_residual_norms(ift_ctx* c, int B, const double* mu, const double* y, const double* z,
                                             double* norms) {
  NvtxRange nvtx_range("ift_hdm_residual_norms");
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (B < 1 || !mu || !y || (c->kx > 0 && !z) || !norms) return c->fail(IFT_ERR_ARG, "bad argument");
  const int ku = c->ku, kx = c->kx, k = ku + kx, nmu = (c->dim == 1) ? 1 : 2;
  cudaStream_t s = c->stream;
  if ((size_t)B > c->rn_cap_B) {
    CK(dalloc(c->d_rn_pts, (size_t)B * k), "alloc norm points");
    CK(dalloc(c->d_rn_mu, (size_t)B * 2), "alloc norm parameters");
    CK(dalloc(c->d_rn_norms, (size_t)B), "alloc norms");
    c->rn_cap_B = (size_t)B;
  }
  std::vector<double> pts((size_t)B * k), mus((size_t)B * 2, 0.0);
  for (int q = 0; q < B; ++q) {
    for (int i = 0; i < ku; ++i) pts[(size_t)q * k + i] = y[(size_t)q * ku + i];
    for (int i = 0; i < kx; ++i) pts[(size_t)q * k + ku + i] = z[(size_t)q * kx + i];
    for (int i = 0; i < nmu; ++i) mus[(size_t)q * 2 + i] = mu[(size_t)q * nmu + i];
  }
  CK(cudaMemcpyAsync(c->d_rn_pts, pts.data(), pts.size() * 8, cudaMemcpyHostToDevice, s), "copy points");
  CK(cudaMemcpyAsync(c->d_rn_mu, mus.data(), mus.size() * 8, cudaMemcpyHostToDevice, s), "copy parameters");
  st = launch_residual_norms(c, B, c->d_rn_pts, c->d_rn_mu, c->d_rn_norms, s);
  if (st != IFT_OK) return st;
  CK(cudaMemcpyAsync(norms, c->d_rn_norms, (size_t)B * 8, cudaMemcpyDeviceToHost, s), "copy norms");
  CK(cudaStreamSynchronize(s), "residual norms");
  return IFT_OK;
}

// ---------------------------------------------------------------------------
// Per-element reduced-residual contributions: columns of the EQP linear program.
// ---------------------------------------------------------------------------
extern "C" ift_status ift_element_gradients(ift_ctx* c, const double* mu, const double* y, const double* z,
                                            int64_t n, const int32_t* elems, double* out) {
  NvtxRange nvtx_range("ift_element_gradients");
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (!mu || !y || (c->kx > 0 && !z) || !out || n < -1 || n == 0 || (n > 0 && !elems))
    return c->fail(IFT_ERR_ARG, "bad argument");
  const int64_t items = (n < 0) ? c->n_elems : n;
  if (n > 0)
    for (int64_t i = 0; i < n; ++i)
      if (elems[i] < 0 || elems[i] >= c->n_elems) return c->fail(IFT_ERR_ARG, "element index out of range");
  const int wp = c->eval_wp(), k = c->ku + c->kx, nmu = (c->dim == 1) ? 1 : 2;
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(c->d_mu, mu, nmu * 8, cudaMemcpyHostToDevice, s), "copy mu");
  CK(cudaMemcpyAsync(c->d_w, y, c->ku * 8, cudaMemcpyHostToDevice, s), "copy y");
  if (c->kx > 0) CK(cudaMemcpyAsync(c->d_tau, z, c->kx * 8, cudaMemcpyHostToDevice, s), "copy z");
  int* d_el = nullptr;
  double* d_out = nullptr;
  auto cleanup = [&]() {
    dfree(d_el);
    dfree(d_out);
  };
  if (n > 0 && dalloc(d_el, (size_t)n) != cudaSuccess) return c->fail(IFT_ERR_OOM, "element list");
  if (dalloc(d_out, (size_t)items * (k + 1)) != cudaSuccess) {
    cleanup();
    return c->fail(IFT_ERR_OOM, "output rows");
  }
  if (n > 0) cudaMemcpyAsync(d_el, elems, (size_t)n * 4, cudaMemcpyHostToDevice, s);
  const KernelSet& ks = c->ks[wp];
  const int warps = c->wpc[wp], block = 32 * warps;
  const size_t smem = ks.smem_bytes(true, c->ku, c->kx, warps);
  const long grid = std::min<long>((items + warps - 1) / warps, (long)c->sm_count * 8);
  cudaError_t e;
  if (wp == 1) {
    AsmArgs<float> a = make_args<float>(c, c->d_Phi32, c->d_w, c->d_tau, c->d_mu, true, nullptr);
    a.elems = d_el;
    a.n_items = items;
    e = ks.element_gradients(&a, d_out, (int)grid, block, smem, s);
  } else {
    AsmArgs<double> a = make_args<double>(c, c->d_Phi, c->d_w, c->d_tau, c->d_mu, true, nullptr);
    a.elems = d_el;
    a.n_items = items;
    e = ks.element_gradients(&a, d_out, (int)grid, block, smem, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, (size_t)items * (k + 1) * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return c->cuda_fail(e, "element gradients");
  for (int64_t i = 0; i < items; ++i)
    if (std::isinf(out[i * (k + 1) + k])) return c->fail(IFT_ERR_NONPHYSICAL, "non-physical element at (y, z)");
  return IFT_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the launch shapes.
// ---------------------------------------------------------------------------
namespace {

// Median of reps timed runs of fn (after one warm-up); +inf if a launch fails.
template <class F>
float time_launch(ift_ctx* c, cudaStream_t s, int reps, F fn) {
  if (fn() != IFT_OK) return INFINITY;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> t;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, s);
    ift_status st = fn();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (st != IFT_OK) ms = INFINITY;
    t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::sort(t.begin(), t.end());
  (void)c;
  return t[t.size() / 2];
}

}  // namespace

extern "C" ift_status ift_autotune(ift_ctx* c, const double* mu, const double* y, const double* z, int32_t* chosen) {
  NvtxRange nvtx_range("ift_autotune");
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (!mu || !y || (c->kx > 0 && !z)) return c->fail(IFT_ERR_ARG, "null input pointer");
  cudaStream_t s = c->stream;
  const int wp = c->eval_wp();
  const int nmu = (c->dim == 1) ? 1 : 2, k = c->ku + c->kx;
  CK(cudaMemcpy(c->d_mu, mu, nmu * 8, cudaMemcpyHostToDevice), "copy mu");
  CK(cudaMemcpy(c->d_w, y, c->ku * 8, cudaMemcpyHostToDevice), "copy y");
  if (c->kx > 0) CK(cudaMemcpy(c->d_tau, z, c->kx * 8, cudaMemcpyHostToDevice), "copy z");
  const int cand_w[3] = {1, 2, 4};
  // single-query fused assembly: warps per CTA, for each precision the context runs
  for (int tp = 0; tp < 2; ++tp) {
    if (!c->ks[tp].valid) continue;
    float best = INFINITY;
    int best_w = c->wpc[tp];
    for (int w : cand_w) {
      c->wpc[tp] = w;
      c->epoch++;
      const float t = time_launch(c, s, 3, [&]() {
        return launch_assemble(c, tp, true, c->d_w, c->d_tau, c->d_mu, c->d_res, nullptr, s);
      });
      if (t < best) {
        best = t;
        best_w = w;
      }
    }
    c->wpc[tp] = best_w;
    c->epoch++;
  }
  if (c->B > 0) {
    // batched assembly: chunk size x warps per CTA, scored on a full batch plus a tail
    // in which only every 50th query is still running (weight 8: tails have more bodies).
    // The chunk size is tuned on the precision that dominates a solve (FP64 for mixed
    // contexts: its stage evaluates at the full cost), then the other precision's warps.
    std::vector<double> wrep((size_t)c->B * k), mrep((size_t)c->B * 2, 0.0);
    for (int q = 0; q < c->B; ++q) {
      for (int i = 0; i < c->ku; ++i) wrep[(size_t)q * k + i] = y[i];
      for (int i = 0; i < c->kx; ++i) wrep[(size_t)q * k + c->ku + i] = z[i];
      for (int i = 0; i < nmu; ++i) mrep[(size_t)q * 2 + i] = mu[i];
    }
    std::vector<int> tail(c->B);
    for (int q = 0; q < c->B; ++q) tail[q] = (q % 50 == 0) ? 0 : 1;
    int* d_tail = nullptr;
    CK(dalloc(d_tail, (size_t)c->B), "alloc tail flags");
    CK(cudaMemcpy(d_tail, tail.data(), tail.size() * 4, cudaMemcpyHostToDevice), "copy tail flags");
    CK(cudaMemcpy(c->d_bw, wrep.data(), wrep.size() * 8, cudaMemcpyHostToDevice), "copy points");
    CK(cudaMemcpy(c->d_bmu, mrep.data(), mrep.size() * 8, cudaMemcpyHostToDevice), "copy mu");
    auto score_of = [&](int tp) {
      const float tf = time_launch(c, s, 3, [&]() {
        return launch_batched(c, tp, true, c->d_bw, k, nullptr, 0, nullptr, s);
      });
      const float tt = time_launch(c, s, 3, [&]() {
        return launch_batched(c, tp, true, c->d_bw, k, d_tail, 1, nullptr, s);
      });
      return tf + 8.0f * tt;
    };
    const int primary = (c->cfg.precision == IFT_FP32) ? 1 : 0;
    const int cand_c[4] = {4, 8, 16, 32};
    float bscore = INFINITY;
    int bc = c->chunk, bw = c->bwpc[primary];
    for (int ch : cand_c) {
      c->chunk = ch;
      st = rechunk(c);
      if (st != IFT_OK) {
        dfree(d_tail);
        return st;
      }
      for (int w : cand_w) {
        c->bwpc[primary] = w;
        c->epoch++;
        const float score = score_of(primary);
        if (score < bscore) {
          bscore = score;
          bc = ch;
          bw = w;
        }
      }
    }
    c->chunk = bc;
    c->bwpc[primary] = bw;
    st = rechunk(c);
    if (st != IFT_OK) {
      dfree(d_tail);
      return st;
    }
    const int other = 1 - primary;
    if (c->ks[other].valid) {
      float best = INFINITY;
      int best_w = c->bwpc[other];
      for (int w : cand_w) {
        c->bwpc[other] = w;
        c->epoch++;
        const float score = score_of(other);
        if (score < best) {
          best = score;
          best_w = w;
        }
      }
      c->bwpc[other] = best_w;
    }
    dfree(d_tail);
  }
  c->err.clear();
  c->epoch++;
  if (chosen) {
    chosen[0] = c->wpc[wp];
    chosen[1] = c->bwpc[wp];
    chosen[2] = c->chunk;
  }
  CK(cudaStreamSynchronize(s), "autotune");
  return IFT_OK;
}

extern "C" ift_status ift_set_launch_shapes(ift_ctx* c, int warps, int batched_warps, int chunk) {
  if (!c) return IFT_ERR_ARG;
  auto ok_w = [](int w) { return w == 1 || w == 2 || w == 4; };
  if (!ok_w(warps) || !ok_w(batched_warps) || !(chunk == 4 || chunk == 8 || chunk == 16 || chunk == 32))
    return c->fail(IFT_ERR_ARG, "launch shapes must be warps in {1,2,4} and chunk in {4,8,16,32}");
  // each precision the context runs takes these warps, or the most that fit its shared memory
  int w1[2], w2[2];
  for (int tp = 0; tp < 2; ++tp) {
    w1[tp] = warps;
    w2[tp] = batched_warps;
    if (c->have_bases) {
      while (w1[tp] > 1 && shapes_smem(c, tp, w1[tp]) > (size_t)c->smem_optin) w1[tp] /= 2;
      while (w2[tp] > 1 && shapes_smem(c, tp, w2[tp]) > (size_t)c->smem_optin) w2[tp] /= 2;
    }
  }
  const int ewp = c->eval_wp();
  if (w1[ewp] != warps || w2[ewp] != batched_warps)
    return c->fail(IFT_ERR_ARG, "these warps per CTA need more shared memory than a CTA may have for these bases");
  for (int tp = 0; tp < 2; ++tp) {
    c->wpc[tp] = w1[tp];
    c->bwpc[tp] = w2[tp];
  }
  if (chunk != c->chunk) {
    c->chunk = chunk;
    if (c->B > 0) {
      ift_status st = rechunk(c);
      if (st != IFT_OK) return st;
    }
  }
  c->err.clear();
  c->epoch++;
  return IFT_OK;
}

// ---------------------------------------------------------------------------
// Snapshot alignment (Eq. align0): min over (w, x) of (1/2)|F(Phi w, x; mu)|^2,
// F = [R; N] over every element (rho = 1), with the free mesh coordinates x
// unknowns. Levenberg-Marquardt on the full space. At each accepted point one
// element pass stores every element's share of the Gauss-Newton system, M_e =
// A_e^T A_e (+ the distortion term) and g_e = A_e^T R_e (+ dN_e N_e), with
// A_e = [dR_e/dw | dR_e/dx_e], in HBM: the blocks that touch the element's mesh
// coordinates per element, the state block summed over the elements (H_ww, the
// state coefficients being shared) (align_jac_kernel). The normal equations are
// then solved by Jacobi-preconditioned conjugate gradients whose products J^T J v
// read those blocks once each (align_apply_kernel, align_wrows_kernel), the whole
// solve one CUDA graph with a device-side loop. The line search evaluates F alone
// (align_kernel mode 0).
// ---------------------------------------------------------------------------
namespace {

constexpr int kDotBlocks = 120;
static_assert(kDotBlocks >= LM_KMAX, "align_finish_kernel forms one w row per block");

struct AlignWork {
  long Nu = 0, Ne = 0, Nx = 0;
  int ku = 0, nfree = 0, nu = 0, nxe = 0, agrid = 1, awarps = 1, jgrid = 1, jwarps = 1;
  double *w = nullptr, *x = nullptr, *F = nullptr, *dU = nullptr, *dx = nullptr, *dF = nullptr, *gU = nullptr,
         *gx = nullptr, *wt = nullptr, *xt = nullptr, *Ft = nullptr, *part = nullptr, *nbad = nullptr;
  double *g = nullptr, *d = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr, *z = nullptr,
         *diag = nullptr;                                  // unknowns' space
  double *M = nullptr, *ge = nullptr, *apart = nullptr;  // element systems, CTA partials of the w rows
  double *H = nullptr, *hpart = nullptr;                 // H_ww (packed) and its CTA partials
  double* part2 = nullptr;                               // CG partials of r . r and r . z
  double* yslot = nullptr;                               // a product's mesh rows per element coordinate
  int *efree = nullptr, *soff = nullptr, *slots = nullptr;  // element coordinates' free indices; free -> slots
  double* xdir = nullptr;                                  // a mesh direction in element order
  CGState* cg = nullptr;
  int* free_idx = nullptr;  // the free coordinates
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~AlignWork() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (double** q : {&w, &x, &F, &dU, &dx, &dF, &gU, &gx, &wt, &xt, &Ft, &part, &nbad, &g, &d, &r, &p, &Ap, &z,
                       &diag, &M, &ge, &apart, &xdir, &H, &hpart, &part2, &yslot})
      dfree(*q);
    dfree(cg);
    dfree(free_idx);
    dfree(efree);
    dfree(soff);
    dfree(slots);
  }
  // stored: the buffers of the Levenberg-Marquardt solve as well
  cudaError_t alloc(bool stored) {
    const long n = ku + nfree;
    cudaError_t e = cudaSuccess;
    auto B = [&](double*& q, long m) {
      if (e == cudaSuccess) e = dalloc(q, (size_t)(m > 0 ? m : 1));
    };
    B(w, LM_KMAX);
    B(wt, LM_KMAX);
    B(x, Nx);
    B(xt, Nx);
    B(F, Nu + Ne);
    B(Ft, Nu + Ne);
    B(dF, Nu + Ne);
    B(dU, Nu);
    B(gU, Nu);
    B(dx, Nx);
    B(gx, Nx);
    B(part, 2 * kDotBlocks);
    B(nbad, 1);
    if (stored) {
      B(g, n);
      B(d, n);
      B(r, n);
      B(p, n);
      B(Ap, n);
      B(z, n);
      B(diag, n);
      B(M, Ne * (long)(ku * nxe + nxe * nxe));
      B(ge, Ne * (long)(ku + nxe));
      B(H, (long)ku * (ku + 1) / 2);
      B(part2, 2 * kDotBlocks);
      B(yslot, Ne * nxe);
      if (e == cudaSuccess) e = dalloc(efree, (size_t)(Ne * nxe > 0 ? Ne * nxe : 1));
      if (e == cudaSuccess) e = dalloc(soff, (size_t)nfree + 1);
      if (e == cudaSuccess) e = dalloc(slots, (size_t)(Ne * nxe > 0 ? Ne * nxe : 1));
      B(hpart, (long)jgrid * ku * (ku + 1) / 2);
      B(apart, (long)agrid * ku);
      B(xdir, Ne * nxe);
      if (e == cudaSuccess) e = dalloc(cg, 1);
    }
    if (e == cudaSuccess) e = dalloc(free_idx, (size_t)(nfree > 0 ? nfree : 1));
    return e;
  }
};

// Sum of the block partials in block order (deterministic for a fixed grid).
double align_dot(const AlignWork& W, const double* a, const double* b, long n, cudaStream_t s) {
  dot_partial_kernel<<<kDotBlocks, 256, 0, s>>>(a, b, n, W.part);
  double h[kDotBlocks];
  cudaMemcpyAsync(h, W.part, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  double t = 0.0;
  for (int i = 0; i < kDotBlocks; ++i) t += h[i];
  return t;
}

int vec_grid(long n) {
  long g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 1024 ? 1024 : g));
}

// FP64 kernel arguments of the alignment passes at (w, x): the current mesh in
// place of the reference nodes, no mesh basis, face-normal Jacobians formed.
AsmArgs<double> align_args(ift_ctx* c, const double* w, const double* x) {
  AsmArgs<double> a = make_args<double>(c, c->d_Phi, w, c->d_tau, c->d_mu, true, nullptr);
  a.X = x;
  a.kx = 0;
  a.Psi = nullptr;
  a.need_hn = 1;
  return a;
}

// One element pass of align_kernel in FP64 at (w, x): mode 0 F, 1 J v, 2 J^T v.
ift_status align_pass(ift_ctx* c, int mode, const double* w, const double* x, const double* vU, const double* vx,
                      const double* vN, double* outU, double* outX, cudaStream_t s) {
  const KernelSet& ks = c->ks[0];
  if (!ks.align) return c->fail(IFT_ERR_NOTIMPL, "snapshot alignment kernels are not built");
  AsmArgs<double> a = align_args(c, w, x);
  const int warps = mode == 0 ? 4 : 2, block = 32 * warps;
  const size_t smem = ks.smem_bytes(mode != 0, c->ku, 0, warps);
  if (smem > (size_t)c->smem_optin) return c->fail(IFT_ERR_ARG, "alignment pass needs too much shared memory");
  long grid = (c->n_elems + warps - 1) / warps;
  if (grid > (long)c->sm_count * 8) grid = (long)c->sm_count * 8;
  cudaError_t e = ks.align(mode, &a, c->d_X, vU, vx, vN, outU, outX, (int)grid, block, smem, s);
  if (e != cudaSuccess) return c->cuda_fail(e, "alignment pass");
  return IFT_OK;
}

ift_status align_setup(ift_ctx* c, AlignWork& W, const double* mu, const double* w, const double* x,
                       bool stored = false) {
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (!mu || !w || !x) return c->fail(IFT_ERR_ARG, "null input pointer");
  W.Nu = c->n_elems * (long)c->nu;
  W.Ne = c->n_elems;
  W.Nx = c->n_verts * (long)c->dim;
  W.ku = c->ku;
  W.nu = c->nu;
  W.nxe = c->nxe;
  if (stored) {
    if (!c->ks[0].align_apply_plan) return c->fail(IFT_ERR_NOTIMPL, "snapshot alignment kernels are not built");
    CK(c->ks[0].align_apply_plan(W.ku, W.Ne, c->sm_count, &W.awarps, &W.agrid), "alignment product shape");
    CK(c->ks[0].align_jac_plan(W.ku, W.Ne, c->sm_count, &W.jwarps, &W.jgrid), "alignment Jacobian pass shape");
  }
  CK(W.alloc(stored), "alignment buffers");
  const int nmu = (c->dim == 1) ? 1 : 2;
  // host or device inputs (unified addressing tells them apart)
  CK(cudaMemcpy(c->d_mu, mu, nmu * 8, cudaMemcpyDefault), "copy mu");
  CK(cudaMemcpy(W.w, w, W.ku * 8, cudaMemcpyDefault), "copy w");
  CK(cudaMemcpy(W.x, x, W.Nx * 8, cudaMemcpyDefault), "copy x");
  return IFT_OK;
}

// The element systems, F and the non-physical count at (W.w, W.x); J = (1/2)|F|^2
// (+inf where an element is non-physical).
ift_status align_form(ift_ctx* c, AlignWork& W, double& J, cudaStream_t s) {
  const KernelSet& ks = c->ks[0];
  if (!ks.align_jac) return c->fail(IFT_ERR_NOTIMPL, "snapshot alignment kernels are not built");
  if (ks.align_jac_smem(c->ku, W.jwarps) > (size_t)c->smem_optin)
    return c->fail(IFT_ERR_ARG, "alignment Jacobian pass needs too much shared memory");
  AsmArgs<double> a = align_args(c, W.w, W.x);
  CK(cudaMemsetAsync(W.nbad, 0, 8, s), "zero count");
  CK(ks.align_jac(&a, c->d_X, W.M, W.ge, W.F, W.nbad, W.hpart, W.jwarps, W.jgrid, s), "alignment Jacobian pass");
  const int nh = W.ku * (W.ku + 1) / 2;
  reduce_partials_kernel<<<(nh + 31) / 32, 1024, 0, s>>>(W.hpart, W.jgrid, nh, W.H, nullptr);
  CK(cudaGetLastError(), "H_ww");
  J = 0.5 * align_dot(W, W.F, W.F, W.Nu + W.Ne, s);
  double nb = 0.0;
  CK(cudaMemcpy(&nb, W.nbad, 8, cudaMemcpyDeviceToHost), "read count");
  if (nb > 0.0) J = INFINITY;
  return IFT_OK;
}

// out (unknowns' space) from the element systems: mode 1 J^T F, 2 diag(J^T J)
// (the CG body forms mode 0, J^T J v, itself).
ift_status align_apply(ift_ctx* c, AlignWork& W, int mode, double* out, cudaStream_t s) {
  const KernelSet& ks = c->ks[0];
  CK(ks.align_apply(mode, W.M, W.ge, W.efree, W.xdir, W.Ne, W.ku, nullptr, W.apart, W.yslot, W.agrid, W.awarps, s),
     "alignment product");
  align_wrows_kernel<<<(W.ku + 7) / 8, 256, 0, s>>>(W.apart, W.agrid, W.ku, W.H, nullptr, mode, out);
  if (W.nfree > 0)
    take_free_kernel<<<vec_grid(W.nfree), 256, 0, s>>>(W.nfree, W.yslot, W.soff, W.slots, out + W.ku);
  CK(cudaGetLastError(), "alignment product");
  return IFT_OK;
}

// The CG loop body: Ap = (J^T J + lam D) p with the partials of p . Ap, then one
// preconditioned CG update (the r partials in a second buffer).
ift_status align_cg_body(ift_ctx* c, AlignWork& W, cudaStream_t s, unsigned long long handle, int use_cond) {
  const KernelSet& ks = c->ks[0];
  const long n = W.ku + W.nfree;
  CK(ks.align_apply(0, W.M, W.ge, W.efree, W.xdir, W.Ne, W.ku, W.p, W.apart, W.yslot, W.agrid, W.awarps, s),
     "alignment product");
  align_finish_kernel<<<kDotBlocks, 256, 0, s>>>(W.apart, W.agrid, W.ku, W.H, W.p, W.nfree, W.yslot, W.soff, W.slots,
                                                 W.cg, W.Ap, W.part);
  cg_update_kernel<<<kDotBlocks, 256, 0, s>>>(n, W.ku, W.part, kDotBlocks, W.cg, W.p, W.Ap, W.diag, W.d, W.r, W.z,
                                              W.part2);
  cg_beta_kernel<<<1, 32, 0, s>>>(W.part2, kDotBlocks, W.cg, handle, use_cond);
  cg_dir_kernel<<<vec_grid(n), 256, 0, s>>>(n, W.ku, W.cg, W.z, W.p, W.soff, W.slots, W.xdir);
  CK(cudaGetLastError(), "conjugate-gradient step");
  return IFT_OK;
}

}  // namespace

extern "C" ift_status ift_align_residual(ift_ctx* c, const double* mu, const double* w, const double* x, double* F) {
  AlignWork W;
  ift_status st = align_setup(c, W, mu, w, x);
  if (st != IFT_OK) return st;
  if (!F) return c->fail(IFT_ERR_ARG, "null output pointer");
  cudaStream_t s = c->stream;
  st = align_pass(c, 0, W.w, W.x, nullptr, nullptr, nullptr, W.F, nullptr, s);
  if (st != IFT_OK) return st;
  CK(cudaMemcpyAsync(F, W.F, (W.Nu + W.Ne) * 8, cudaMemcpyDeviceToHost, s), "copy F");
  CK(cudaStreamSynchronize(s), "alignment residual");
  return IFT_OK;
}

extern "C" ift_status ift_align_jvp(ift_ctx* c, const double* mu, const double* w, const double* x, const double* dU,
                                    const double* dx, double* dF) {
  AlignWork W;
  ift_status st = align_setup(c, W, mu, w, x);
  if (st != IFT_OK) return st;
  if (!dU || !dx || !dF) return c->fail(IFT_ERR_ARG, "null pointer");
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(W.dU, dU, W.Nu * 8, cudaMemcpyHostToDevice, s), "copy dU");
  CK(cudaMemcpyAsync(W.dx, dx, W.Nx * 8, cudaMemcpyHostToDevice, s), "copy dx");
  st = align_pass(c, 1, W.w, W.x, W.dU, W.dx, nullptr, W.dF, nullptr, s);
  if (st != IFT_OK) return st;
  CK(cudaMemcpyAsync(dF, W.dF, (W.Nu + W.Ne) * 8, cudaMemcpyDeviceToHost, s), "copy dF");
  CK(cudaStreamSynchronize(s), "alignment J v");
  return IFT_OK;
}

extern "C" ift_status ift_align_vjp(ift_ctx* c, const double* mu, const double* w, const double* x, const double* v,
                                    double* gU, double* gx) {
  AlignWork W;
  ift_status st = align_setup(c, W, mu, w, x);
  if (st != IFT_OK) return st;
  if (!v || !gU || !gx) return c->fail(IFT_ERR_ARG, "null pointer");
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(W.dF, v, (W.Nu + W.Ne) * 8, cudaMemcpyHostToDevice, s), "copy v");
  CK(cudaMemsetAsync(W.gU, 0, W.Nu * 8, s), "zero gU");
  CK(cudaMemsetAsync(W.gx, 0, W.Nx * 8, s), "zero gx");
  st = align_pass(c, 2, W.w, W.x, W.dF, nullptr, W.dF + W.Nu, W.gU, W.gx, s);
  if (st != IFT_OK) return st;
  CK(cudaMemcpyAsync(gU, W.gU, W.Nu * 8, cudaMemcpyDeviceToHost, s), "copy gU");
  CK(cudaMemcpyAsync(gx, W.gx, W.Nx * 8, cudaMemcpyDeviceToHost, s), "copy gx");
  CK(cudaStreamSynchronize(s), "alignment J^T v");
  return IFT_OK;
}

namespace {

// ift_align and ift_align_dev: mu, w, x and free_mask host or device pointers (the
// copies use unified addressing), the work on stream s, which is synchronised.
ift_status align_run(ift_ctx* c, const double* mu, double* w, double* x, const uint8_t* free_mask, double tol,
                     int max_iters, ift_align_info* info, cudaStream_t s) {
  AlignWork W;
  ift_status st = check_ready(c);
  if (st != IFT_OK) return st;
  if (!free_mask) return c->fail(IFT_ERR_ARG, "null free-coordinate mask");
  // device inputs may still be in flight on the caller's stream: the copies below
  // read them after it
  CK(cudaStreamSynchronize(s), "caller's stream");
  std::vector<uint8_t> hmask((size_t)c->n_verts * c->dim);
  CK(cudaMemcpy(hmask.data(), free_mask, hmask.size(), cudaMemcpyDefault), "copy free-coordinate mask");
  for (uint8_t m : hmask) W.nfree += m ? 1 : 0;
  if (c->ku + c->nxe > 96) return c->fail(IFT_ERR_ARG, "alignment supports k_u + n_xe <= 96");
  st = align_setup(c, W, mu, w, x, true);
  if (st != IFT_OK) return st;
  if (!(tol >= 0.0) || max_iters < 0) return c->fail(IFT_ERR_ARG, "tol >= 0 and max_iters >= 0 required");
  {
    // free coordinates; per element coordinate its free index (-1: fixed); per free
    // coordinate the element slots that hold it (CSR), for the element-order direction
    std::vector<int> idx, pos((size_t)W.Nx, -1);
    for (long i = 0; i < W.Nx; ++i)
      if (hmask[(size_t)i]) {
        pos[(size_t)i] = (int)idx.size();
        idx.push_back((int)i);
      }
    const long ns = W.Ne * W.nxe;
    std::vector<int> ev((size_t)W.Ne * c->nv), efree((size_t)ns), off((size_t)W.nfree + 1, 0), slots;
    CK(cudaMemcpy(ev.data(), c->d_ev, ev.size() * 4, cudaMemcpyDeviceToHost), "read elements");
    for (long t = 0; t < ns; ++t) {
      const long e = t / W.nxe;
      const int r = (int)(t - e * W.nxe);
      const int q = pos[(size_t)ev[(size_t)e * c->nv + r / c->dim] * c->dim + r % c->dim];
      efree[(size_t)t] = q;
      if (q >= 0) ++off[(size_t)q + 1];
    }
    for (int j = 0; j < W.nfree; ++j) off[(size_t)j + 1] += off[(size_t)j];
    slots.resize((size_t)off[(size_t)W.nfree] > 0 ? (size_t)off[(size_t)W.nfree] : 1);
    {
      std::vector<int> fill(off.begin(), off.end() - 1);
      for (long t = 0; t < ns; ++t)
        if (efree[(size_t)t] >= 0) slots[(size_t)fill[(size_t)efree[(size_t)t]]++] = (int)t;
    }
    if (!idx.empty()) CK(cudaMemcpy(W.free_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice), "copy idx");
    CK(cudaMemcpy(W.efree, efree.data(), efree.size() * 4, cudaMemcpyHostToDevice), "copy free indices");
    CK(cudaMemcpy(W.soff, off.data(), off.size() * 4, cudaMemcpyHostToDevice), "copy slot offsets");
    CK(cudaMemcpy(W.slots, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice), "copy slots");
  }
  const long n = W.ku + W.nfree;
  // the fixed coordinates' slots of the element-order direction stay zero
  CK(cudaMemsetAsync(W.xdir, 0, (W.Ne * W.nxe > 0 ? W.Ne * W.nxe : 1) * 8, s), "zero direction");
  // readings of Sec. 3.2.3 as for the reduced solve: lambda_0 = 1e-4, /10 after a
  // full step, x10 after a shortened one, Armijo 1e-4, at most 30 halvings; damping
  // on the mesh block only (Eq. levmarq-step)
  const double c1 = 1e-4, round_tol = 16.0 * 2.220446049250313e-16;
  double lam = 1e-4;
  CGState cg0{};
  cg0.tol = c->cfg.align_cg_tol > 0.0 ? c->cfg.align_cg_tol : 1e-12;
  cg0.max_iters = (int)std::min<long>(4 * n + 20, 2000);
  cg0.done = 1;
  // (1/2)|F|^2 at (ww, xx) by the residual-only pass; +inf where an element is
  // non-physical (such a trial is rejected, as in the reduced solve)
  auto objective = [&](const double* ww, const double* xx, double* FF, double& Jv) -> ift_status {
    CK(cudaMemsetAsync(W.nbad, 0, 8, s), "zero count");
    ift_status q = align_pass(c, 0, ww, xx, nullptr, nullptr, nullptr, FF, W.nbad, s);
    if (q != IFT_OK) return q;
    Jv = 0.5 * align_dot(W, FF, FF, W.Nu + W.Ne, s);
    double nb = 0.0;
    CK(cudaMemcpy(&nb, W.nbad, 8, cudaMemcpyDeviceToHost), "read count");
    if (nb > 0.0) Jv = INFINITY;
    return IFT_OK;
  };
  // at an accepted point: the stored blocks, F, the gradient and the preconditioner
  auto form = [&](double& Jv, double& gn) -> ift_status {
    ift_status q = align_form(c, W, Jv, s);
    if (q != IFT_OK) return q;
    if (!std::isfinite(Jv)) return IFT_OK;
    q = align_apply(c, W, 1, W.g, s);
    if (q != IFT_OK) return q;
    q = align_apply(c, W, 2, W.diag, s);
    if (q != IFT_OK) return q;
    gn = std::sqrt(align_dot(W, W.g, W.g, n, s));
    return IFT_OK;
  };
  cg0.lam = lam;
  CK(cudaMemcpy(W.cg, &cg0, sizeof(CGState), cudaMemcpyHostToDevice), "copy solve scalars");
  // one conjugate-gradient solve = one launch of a while-loop graph (or, with
  // IFT_SOLVE_NO_GRAPH set, the same body enqueued from the host in groups of 8)
  static const bool no_graph = getenv("IFT_SOLVE_NO_GRAPH") != nullptr;
  if (!no_graph) {
    st = build_while_graph(c, &W.graph, &W.exec, [&](cudaStream_t cs, unsigned long long h) {
      return align_cg_body(c, W, cs, h, 1);
    });
    if (st != IFT_OK) return st;
  }
  auto run_cg = [&]() -> ift_status {
    if (!no_graph) {
      CK(cudaGraphLaunch(W.exec, s), "conjugate-gradient graph");
      return IFT_OK;
    }
    for (int b = 0; b <= cg0.max_iters; b += 8) {
      for (int j = 0; j < 8; ++j) {
        ift_status q = align_cg_body(c, W, s, 0ull, 0);
        if (q != IFT_OK) return q;
      }
      int dn = 0;
      CK(cudaMemcpyAsync(&dn, (const char*)W.cg + offsetof(CGState, done), sizeof(int), cudaMemcpyDeviceToHost, s),
         "read done flag");
      CK(cudaStreamSynchronize(s), "conjugate-gradient loop");
      if (dn) break;
    }
    return IFT_OK;
  };
  // device time of the phases (CUDA events on the solve's stream)
  cudaEvent_t ev[2];
  CK(cudaEventCreate(&ev[0]), "event");
  CK(cudaEventCreate(&ev[1]), "event");
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      cudaEventDestroy(e[0]);
      cudaEventDestroy(e[1]);
    }
  } ev_guard{ev};
  double ms_form = 0.0, ms_cg = 0.0, ms_search = 0.0;
  auto lap = [&](double& acc) -> ift_status {
    CK(cudaEventRecord(ev[1], s), "event");
    CK(cudaEventSynchronize(ev[1]), "event");
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, ev[0], ev[1]), "event time");
    acc += t;
    return IFT_OK;
  };
  double J = 0.0, gnorm = 0.0;
  CK(cudaEventRecord(ev[0], s), "event");
  st = form(J, gnorm);
  if (st != IFT_OK) return st;
  if (!std::isfinite(J)) return c->fail(IFT_ERR_NONPHYSICAL, "the starting point is not physical");
  if ((st = lap(ms_form)) != IFT_OK) return st;
  const double g0 = gnorm, thresh = tol * std::max(1.0, g0);
  int status = IFT_NOT_CONVERGED, iters = 0, cg_total = 0, trials = 0;
  for (;;) {
    if (gnorm <= thresh) {
      status = IFT_OK;
      break;
    }
    if (iters >= max_iters) break;
    // (J^T J + lam D) d = -g by preconditioned CG from d = 0, on the device
    cg0.lam = lam;
    CK(cudaEventRecord(ev[0], s), "event");
    CK(cudaMemcpyAsync(W.cg, &cg0, sizeof(CGState), cudaMemcpyHostToDevice, s), "copy solve scalars");
    cg_start_kernel<<<kDotBlocks, 256, 0, s>>>(n, W.ku, W.g, W.diag, W.cg, W.d, W.r, W.z, W.p, W.part, W.soff,
                                               W.slots, W.xdir);
    cg_start_finish_kernel<<<1, 32, 0, s>>>(W.part, kDotBlocks, W.cg);
    CK(cudaGetLastError(), "conjugate-gradient start");
    if ((st = run_cg()) != IFT_OK) return st;
    CGState cgr{};
    CK(cudaMemcpyAsync(&cgr, W.cg, sizeof(CGState), cudaMemcpyDeviceToHost, s), "read solve scalars");
    const double slope = align_dot(W, W.g, W.d, n, s);  // synchronises the stream
    if ((st = lap(ms_cg)) != IFT_OK) return st;
    cg_total += cgr.iters;
    CK(cudaEventRecord(ev[0], s), "event");
    // backtracking line search on (1/2)|F|^2
    double alpha = 1.0, Jt = 0.0;
    int h = 0;
    bool accepted = false;
    for (;;) {
      CK(cudaMemcpyAsync(W.wt, W.w, W.ku * 8, cudaMemcpyDeviceToDevice, s), "wt = w");
      axpy_kernel<<<1, 64, 0, s>>>(W.ku, alpha, W.d, W.wt);
      CK(cudaMemsetAsync(W.gx, 0, W.Nx * 8, s), "zero step");
      if (W.nfree > 0) scatter_free_kernel<<<vec_grid(W.nfree), 256, 0, s>>>(W.free_idx, W.nfree, W.d + W.ku, W.gx);
      CK(cudaMemcpyAsync(W.xt, W.x, W.Nx * 8, cudaMemcpyDeviceToDevice, s), "xt = x");
      axpy_kernel<<<vec_grid(W.Nx), 256, 0, s>>>(W.Nx, alpha, W.gx, W.xt);
      st = objective(W.wt, W.xt, W.Ft, Jt);
      if (st != IFT_OK) return st;
      ++trials;
      if (std::isfinite(Jt) && Jt <= J + c1 * alpha * slope + round_tol * std::fabs(J)) {
        accepted = true;
        break;
      }
      if (++h > 30) break;
      alpha *= 0.5;
    }
    if ((st = lap(ms_search)) != IFT_OK) return st;
    if (!accepted) {
      status = IFT_LINESEARCH_FAILED;
      break;
    }
    lam = (h == 0) ? std::max(lam / 10.0, 1e-12) : std::min(lam * 10.0, 1e8);
    std::swap(W.w, W.wt);
    std::swap(W.x, W.xt);
    ++iters;
    double Jf = 0.0;
    CK(cudaEventRecord(ev[0], s), "event");
    st = form(Jf, gnorm);
    if (st != IFT_OK) return st;
    if ((st = lap(ms_form)) != IFT_OK) return st;
    J = Jt;
  }
  CK(cudaMemcpyAsync(w, W.w, W.ku * 8, cudaMemcpyDefault, s), "copy w");
  CK(cudaMemcpyAsync(x, W.x, W.Nx * 8, cudaMemcpyDefault, s), "copy x");
  CK(cudaStreamSynchronize(s), "alignment");
  if (info) {
    info->status = status;
    info->iters = iters;
    info->cg_iters = cg_total;
    info->trials = trials;
    info->J = J;
    info->gnorm = gnorm;
    info->g0 = g0;
    info->ms_form = ms_form;
    info->ms_cg = ms_cg;
    info->ms_search = ms_search;
  }
  return (ift_status)status;
}

}  // namespace

extern "C" ift_status ift_align(ift_ctx* c, const double* mu, double* w, double* x, const uint8_t* free_mask,
                                double tol, int max_iters, ift_align_info* info) {
  NvtxRange nvtx_range("ift_align");
  return align_run(c, mu, w, x, free_mask, tol, max_iters, info, c ? c->stream : nullptr);
}

extern "C" ift_status ift_align_dev(ift_ctx* c, const double* mu, double* w, double* x, const uint8_t* free_mask,
                                    double tol, int max_iters, ift_align_info* info_host, void* stream) {
  NvtxRange nvtx_range("ift_align_dev");
  return align_run(c, mu, w, x, free_mask, tol, max_iters, info_host,
                   stream ? (cudaStream_t)stream : (c ? c->stream : nullptr));
}
