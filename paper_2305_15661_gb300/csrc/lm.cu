// Levenberg-Marquardt step kernel and small helper kernels of the solve.
#include <cuda_runtime.h>

#include "../../include/ift.h"
#include "elem.cuh"
#include "lm.cuh"

namespace ift {

namespace {

// Constants of the line search and damping rule (readings of Sec. 3.2.3):
// lambda_0 = 1e-4, lambda/10 (>= 1e-12) after a full step, 10 lambda (<= 1e8)
// after a shortened step; Armijo constant 1e-4 with an allowance of 16 machine
// epsilons of |J| for rounding in J; at most 30 halvings; on a failed Cholesky
// the diagonal is shifted by 1e-14 trace/k, times 10 per retry, at most 10 times.
constexpr double kLam0 = 1e-4, kLamMin = 1e-12, kLamMax = 1e8, kC1 = 1e-4;
constexpr double kRound = 16.0 * 2.220446049250313e-16;
constexpr int kMaxShifts = 10;

__device__ double active_norm(const LMState& s, int ku, int kx, bool full) {
  double t = 0.0;
  for (int c = 0; c < ku; ++c) t += s.g[c] * s.g[c];
  if (full)
    for (int c = 0; c < kx; ++c) t += s.g[ku + c] * s.g[ku + c];
  return sqrt(t);
}

// Cholesky of the n x n matrix in shared memory A (row-major, lower triangle used),
// done by one warp, right-looking. On return the strict lower triangle holds L and
// the diagonal holds 1 / L_jj (the solve below multiplies by it). An FP64 warp
// instruction costs the same with one active lane as with 32, so each column takes
// one reciprocal square root for its pivot, one scaling of the column below it
// and then the trailing lower triangle, all m (m + 1) / 2 of its entries spread
// over the 32 lanes (m = n - 1 - j): entry t of that triangle is (i, l) with
// l = n - 1 - a, i = l + b, t = a (a + 1) / 2 + b, 0 <= b <= a.
__device__ bool warp_cholesky(double* A, int n, int lane) {
  for (int j = 0; j < n; ++j) {
    __syncwarp();
    const double d = A[j * n + j];
    if (!(d > 0.0)) return false;
    const double inv = rsqrt(d);
    __syncwarp();
    for (int i = j + 1 + lane; i < n; i += 32) A[i * n + j] *= inv;
    if (lane == 0) A[j * n + j] = inv;
    __syncwarp();
    const int m = n - 1 - j;
    const int tri = m * (m + 1) / 2;
    for (int t = lane; t < tri; t += 32) {
      int a = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      if ((a + 1) * (a + 2) / 2 <= t) ++a;
      if (a * (a + 1) / 2 > t) --a;
      const int l = n - 1 - a;
      const int i = l + (t - a * (a + 1) / 2);
      A[i * n + l] -= A[i * n + j] * A[l * n + j];
    }
  }
  __syncwarp();
  return true;
}

// Solves L L^T x = b in place in rhs (n values, shared memory) with the factor of
// warp_cholesky (strict lower triangle L, diagonal 1 / L_jj), by one warp:
// column-oriented forward and backward substitution (one pivot per step,
// lane-parallel updates of the remaining rows).
__device__ void warp_cholesky_solve(const double* L, int n, double* rhs, int lane) {
  for (int j = 0; j < n; ++j) {  // L y = b
    __syncwarp();
    const double yj = rhs[j] * L[j * n + j];
    __syncwarp();
    if (lane == 0) rhs[j] = yj;
    for (int i = j + 1 + lane; i < n; i += 32) rhs[i] -= L[i * n + j] * yj;
  }
  for (int i = n - 1; i >= 0; --i) {  // L^T x = y
    __syncwarp();
    const double xi = rhs[i] * L[i * n + i];
    __syncwarp();
    if (lane == 0) rhs[i] = xi;
    for (int j = lane; j < i; j += 32) rhs[j] -= L[i * n + j] * xi;
  }
  __syncwarp();
}

// The LM state of one query, copied between global and shared memory by one warp.
__device__ void copy_state(LMState& dst, const LMState& src, int lane) {
  static_assert(sizeof(LMState) % 8 == 0, "LMState is copied in 8-byte words");
  auto* d = reinterpret_cast<unsigned long long*>(&dst);
  const auto* v = reinterpret_cast<const unsigned long long*>(&src);
  for (int w = lane; w < (int)(sizeof(LMState) / 8); w += 32) d[w] = v[w];
  __syncwarp();
}

}  // namespace

// Lane-0 logic of the iteration, in the order of the oracle's loop:
//   at the current iterate: stop if |g| <= thresh (converged), else stop if the
//   phase has taken max_iters steps, else solve for a step.
// end_phase(): phase 0 hands over to phase 1 at the same point (the joint
// iteration restarts there with lambda_0 and its own reference norm);
// phase 1 finishes the solve.
__device__ void begin_phase(LMState& s, const LMConsts& c) {
  s.g0 = active_norm(s, c.ku, c.kx, s.phase == 1);
  s.thresh = c.tol * fmax(1.0, s.g0);
  s.lam = kLam0;
}

// Returns true if a step must be solved for, false if the solve finished.
__device__ bool decide(LMState& s, const LMConsts& c) {
  for (;;) {
    const bool full = s.phase == 1;
    int st = -100;
    if (active_norm(s, c.ku, c.kx, full) <= s.thresh) st = IFT_OK;
    else if (s.iters[s.phase] >= c.max_iters) st = IFT_NOT_CONVERGED;
    if (st == -100) return true;
    if (!full) {
      s.init_status = st;
      s.phase = 1;
      begin_phase(s, c);
      continue;
    }
    s.status = st;
    s.done = 1;
    return false;
  }
}

// One LM step of one query by one warp. res = [H (k*k) | g (k) | J | nonphysical count]
// at s.trial; s is the query's state in shared memory (the scalar logic runs on
// lane 0 and would wait on global memory at every field); Ms (LM_KMAX^2), rhs
// (LM_KMAX) and gs (LM_KMAX + 2) are the warp's shared buffers.
__device__ void lm_step_warp(LMState& s, const double* res, const LMConsts& c, double* Ms, double* rhs, double* gs,
                             int lane) {
  const int ku = c.ku, kx = c.kx, k = ku + kx;
  const double* Hr = res;
  for (int i = lane; i < k + 2; i += 32) gs[i] = res[k * k + i];
  __syncwarp();
  const double* gr = gs;
  const double Jr = gs[k];
  const double npr = gs[k + 1];
  int need_solve = 0;
  bool refresh_h = false;  // the next evaluation recomputes H (after a shortened step)
  if (lane == 0 && !s.done) {
    s.bodies += 1;
    s.res_at_z = 0;
    if (c.keep_h && !s.hkeep) s.hevals += 1;
    if (s.bodies > c.body_limit) {
      s.status = IFT_ERR_TIMEOUT;
      s.done = 1;
    } else if (s.state == 0) {
      // result at the starting point of the solve
      if (npr > 0.0 || !isfinite(Jr)) {
        s.status = IFT_ERR_NONPHYSICAL;
        s.done = 1;
      } else {
        for (int i = 0; i < k; ++i) {
          s.z[i] = s.trial[i];
          s.g[i] = gr[i];
        }
        s.J = Jr;
        s.state = 1;
        s.res_at_z = 1;
        begin_phase(s, c);
        need_solve = decide(s, c);
      }
    } else {
      const bool ok = npr == 0.0 && isfinite(Jr) && Jr <= s.J + kC1 * s.alpha * s.slope + kRound * fabs(s.J);
      if (ok) {
        refresh_h = s.h != 0;
        s.lam = (s.h == 0) ? fmax(s.lam / 10.0, kLamMin) : fmin(s.lam * 10.0, kLamMax);
        for (int i = 0; i < k; ++i) {
          s.z[i] = s.trial[i];
          s.g[i] = gr[i];
        }
        s.J = Jr;
        s.iters[s.phase] += 1;
        s.res_at_z = 1;
        need_solve = decide(s, c);
      } else if (s.h + 1 > c.max_halvings) {
        // line search failed: this phase ends at the current iterate
        if (s.phase == 0) {
          s.init_status = IFT_LINESEARCH_FAILED;
          s.phase = 1;
          begin_phase(s, c);
          need_solve = decide(s, c);
        } else {
          s.status = IFT_LINESEARCH_FAILED;
          s.done = 1;
        }
      } else {
        refresh_h = true;
        s.h += 1;
        s.alpha *= 0.5;
        const int ka = (s.phase == 1) ? k : ku;
        for (int i = 0; i < ka; ++i) s.trial[i] = s.z[i] + s.alpha * s.dz[i];
        s.trials += 1;
      }
    }
  }
  need_solve = __shfl_sync(0xffffffffu, need_solve, 0);
  while (need_solve) {
    __syncwarp();
    // (H + diag(0, lambda I)) dz = -g on the active block
    const int ka = (s.phase == 1) ? k : ku;
    const double lam = s.lam;
    const bool damp = s.phase == 1;
    for (int i = lane; i < ka * ka; i += 32) {
      const int r = i / ka, cc = i % ka;
      double v = Hr[r * k + cc];
      if (damp && r == cc && r >= ku) v += lam;
      Ms[i] = v;
    }
    __syncwarp();
    bool ok = warp_cholesky(Ms, ka, lane);
    // the diagonal shift of a failed factorisation: 1e-14 trace / k of the damped matrix
    double sh = 0.0;
    if (!ok) {
      double tr = 0.0;
      for (int i = 0; i < ka; ++i) tr += Hr[i * k + i] + ((damp && i >= ku) ? lam : 0.0);
      sh = 1e-14 * tr / ka;
    }
    int nsh = 0;
    while (!ok && nsh < kMaxShifts) {
      __syncwarp();
      for (int i = lane; i < ka * ka; i += 32) {
        const int r = i / ka, cc = i % ka;
        double v = Hr[r * k + cc];
        if (damp && r == cc && r >= ku) v += lam;
        if (r == cc) v += sh;
        Ms[i] = v;
      }
      __syncwarp();
      ok = warp_cholesky(Ms, ka, lane);
      sh *= 10.0;
      ++nsh;
    }
    __syncwarp();
    if (ok) {
      for (int i = lane; i < ka; i += 32) rhs[i] = -s.g[i];
      warp_cholesky_solve(Ms, ka, rhs, lane);
    }
    int again = 0;
    if (lane == 0) {
      s.shifts += nsh;
      if (ok) {
        double slope = 0.0;
        for (int i = 0; i < ka; ++i) {
          s.dz[i] = rhs[i];
          slope += s.g[i] * rhs[i];
        }
        for (int i = ka; i < k; ++i) s.dz[i] = 0.0;
        s.slope = slope;
        s.alpha = 1.0;
        s.h = 0;
        for (int i = 0; i < k; ++i) s.trial[i] = s.z[i] + s.dz[i];
        s.trials += 1;
      } else if (s.phase == 0) {
        s.init_status = IFT_LINESEARCH_FAILED;
        s.phase = 1;
        begin_phase(s, c);
        again = decide(s, c);
      } else {
        s.status = IFT_LINESEARCH_FAILED;
        s.done = 1;
      }
    }
    need_solve = __shfl_sync(0xffffffffu, again, 0);
  }
  // Finishing stage of a mixed solve: H only steers the step, so after a full step
  // the next evaluation keeps the H it has (the FP64 gradient, objective and
  // tests are recomputed at every point); a rejected or shortened step refreshes
  // it, and a finished query skips the FP32 pass.
  if (lane == 0 && c.keep_h) s.hkeep = (s.done || !refresh_h) ? 1 : 0;
  __syncwarp();
}

// A finished query's step changes nothing but the kept-H flag (set, as the step
// itself would set it); its state is then not copied at all. Returns true if the
// query is finished.
__device__ bool lm_step_finished(LMState& g, const LMConsts& c, int lane) {
  const bool done = g.done != 0;
  if (done && lane == 0 && c.keep_h) g.hkeep = 1;
  return done;
}

// One LM step, single warp (the single-query solve).
__global__ void lm_step_kernel(LMState* sp, const double* res, LMConsts c, unsigned long long cond_handle,
                               int use_cond) {
  __shared__ double Ms[LM_KMAX * LM_KMAX];
  __shared__ double rhs[LM_KMAX];
  __shared__ double gs[LM_KMAX + 2];
  __shared__ LMState st;
  const int lane = threadIdx.x;
  if (lm_step_finished(*sp, c, lane)) {
    if (use_cond && lane == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, 0u);
    return;
  }
  copy_state(st, *sp, lane);
  lm_step_warp(st, res, c, Ms, rhs, gs, lane);
  copy_state(*sp, st, lane);
  // inside the solve graph: keep looping while the solve is not finished
  if (use_cond && lane == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, st.done ? 0u : 1u);
}

// One LM step for each of B queries: block q (one warp) steps query q with its
// reduced result res + q * nacc.
__global__ void lm_step_batched_kernel(LMState* states, const double* res, int nacc, LMConsts c) {
  __shared__ double Ms[LM_KMAX * LM_KMAX];
  __shared__ double rhs[LM_KMAX];
  __shared__ double gs[LM_KMAX + 2];
  __shared__ LMState st;
  const int q = blockIdx.x, lane = threadIdx.x;
  if (lm_step_finished(states[q], c, lane)) return;
  copy_state(st, states[q], lane);
  lm_step_warp(st, res + (size_t)q * nacc, c, Ms, rhs, gs, lane);
  copy_state(states[q], st, lane);
}

// Loop condition of the batched solve: keep looping while any query is unfinished.
__global__ void batch_condition_kernel(const LMState* states, int B, int* active, unsigned long long cond_handle,
                                       int use_cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int q = threadIdx.x; q < B; q += blockDim.x) mine += states[q].done ? 0 : 1;
  if (mine) atomicAdd(&any, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    *active = any;
    if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, any ? 1u : 0u);
  }
}

// Per-query sum of the chunk partials: res[q][i] = sum over the chunks of q (in order).
// Finished queries are skipped, and with skip_kept also those whose H is kept.
__global__ void reduce_chunks_kernel(const double* partial, const int* qchunk, int nacc, const LMState* states,
                                     double* res, int skip_kept) {
  const int q = blockIdx.x;
  if (states != nullptr && (states[q].done || (skip_kept && states[q].hkeep))) return;
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) {
    double t = 0.0;
    for (int ch = qchunk[q]; ch < qchunk[q + 1]; ++ch) t += partial[(size_t)ch * nacc + i];
    res[(size_t)q * nacc + i] = t;
  }
}

// Starting states of B queries: w0 = sum_a U_inf,a(mu_q) colsum[a][c] (= Phi^T U_guess(mu_q)),
// tau0 = 0, phase 0 (paper) ; or the given (y, z) rows, phase 1.
__global__ void lm_init_batched_kernel(LMState* states, int B, int ku, int kx, int m, int problem, double gamma,
                                       const double* mu, int mustride, const double* colsum, const double* y0,
                                       const double* z0, int phase);

// Starting state: z = trial = (w0, tau0), phase 0 (paper initialisation) or 1 (given start).
__global__ void lm_init_kernel(LMState* sp, const double* w0, const double* tau0, int ku, int kx, int phase) {
  LMState& s = *sp;
  const int k = ku + kx;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double v = (i < ku) ? w0[i] : (tau0 ? tau0[i - ku] : 0.0);
    s.z[i] = v;
    s.trial[i] = v;
    s.dz[i] = 0.0;
    s.g[i] = 0.0;
  }
  if (threadIdx.x == 0) {
    s.phase = phase;
    s.state = 0;
    s.status = IFT_NOT_CONVERGED;
    s.init_status = IFT_OK;
    s.iters[0] = s.iters[1] = 0;
    s.trials = 0;
    s.shifts = 0;
    s.h = 0;
    s.bodies = 0;
    s.done = 0;
    s.iters32 = 0;
    s.trials32 = 0;
    s.hkeep = 0;
    s.hevals = 0;
    s.res_at_z = 0;
    s.lam = kLam0;
    s.alpha = 1.0;
    s.J = 0.0;
    s.slope = 0.0;
    s.g0 = 0.0;
    s.thresh = 0.0;
  }
}

__global__ void lm_init_batched_kernel(LMState* states, int B, int ku, int kx, int m, int problem, double gamma,
                                       const double* mu, int mustride, const double* colsum, const double* y0,
                                       const double* z0, int phase) {
  const int q = blockIdx.x;
  if (q >= B) return;
  LMState& s = states[q];
  const int k = ku + kx;
  double Ug[4] = {1.0, 0.0, 0.0, 0.0};
  if (phase == 0 && problem == 2) euler_farfield(gamma, mu[(size_t)q * mustride], mu[(size_t)q * mustride + 1], Ug);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double v;
    if (phase == 0) {
      v = 0.0;
      if (i < ku)
        for (int a = 0; a < m; ++a) v += Ug[a] * colsum[a * ku + i];
    } else {
      v = (i < ku) ? y0[(size_t)q * ku + i] : z0[(size_t)q * kx + (i - ku)];
    }
    s.z[i] = v;
    s.trial[i] = v;
    s.dz[i] = 0.0;
    s.g[i] = 0.0;
  }
  if (threadIdx.x == 0) {
    s.phase = phase;
    s.state = 0;
    s.status = IFT_NOT_CONVERGED;
    s.init_status = IFT_OK;
    s.iters[0] = s.iters[1] = 0;
    s.trials = 0;
    s.shifts = 0;
    s.h = 0;
    s.bodies = 0;
    s.done = 0;
    s.iters32 = 0;
    s.trials32 = 0;
    s.hkeep = 0;
    s.hevals = 0;
    s.res_at_z = 0;
    s.lam = kLam0;
    s.alpha = 1.0;
    s.J = 0.0;
    s.slope = 0.0;
    s.g0 = 0.0;
    s.thresh = 0.0;
  }
}

// The FP32 edge table of straight-sided triangles: per element e, 1 + kx groups of
// four floats, first the reference edges (x_1 - x_0, x_2 - x_0) as (e1x, e1y, e2x, e2y),
// then for each mesh column c the same differences of its vertex rows of Psi. The
// differences are taken in FP64 and rounded once, so the FP32 element pass forms
// the current edges (reference + sum_c tau_c column differences) without FP64 work.
__global__ void geo32_kernel(const double* X, const int* ev, const double* Psi, int kx, long n_elems, float4* out) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n_elems; e += (long)gridDim.x * blockDim.x) {
    const long v0 = ev[e * 3], v1 = ev[e * 3 + 1], v2 = ev[e * 3 + 2];
    float4* o = out + e * (1 + kx);
    o[0] = make_float4((float)(X[v1 * 2] - X[v0 * 2]), (float)(X[v1 * 2 + 1] - X[v0 * 2 + 1]),
                       (float)(X[v2 * 2] - X[v0 * 2]), (float)(X[v2 * 2 + 1] - X[v0 * 2 + 1]));
    for (int c = 0; c < kx; ++c)
      o[1 + c] = make_float4((float)(Psi[(v1 * 2) * kx + c] - Psi[(v0 * 2) * kx + c]),
                             (float)(Psi[(v1 * 2 + 1) * kx + c] - Psi[(v0 * 2 + 1) * kx + c]),
                             (float)(Psi[(v2 * 2) * kx + c] - Psi[(v0 * 2) * kx + c]),
                             (float)(Psi[(v2 * 2 + 1) * kx + c] - Psi[(v0 * 2 + 1) * kx + c]));
  }
}

// colsum[a][c] = sum over the rows r of Phi with r mod m = a of Phi[r][c] (one block per column).
__global__ void phi_colsum_kernel(const double* Phi, long Nu, int ku, int m, double* colsum) {
  __shared__ double red[4][256];
  const int c = blockIdx.x;
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  for (long r = threadIdx.x; r < Nu; r += blockDim.x) t[r % m] += Phi[r * ku + c];
  for (int a = 0; a < 4; ++a) red[a][threadIdx.x] = t[a];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int a = 0; a < 4; ++a) red[a][threadIdx.x] += red[a][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int a = 0; a < m; ++a) colsum[a * ku + c] = red[a][0];
}

// Hand a query over from the FP32 stage of a mixed solve to the FP64 stage: the
// joint iteration restarts at the FP32 stage's last iterate with lambda_0 and a new
// reference norm (taken from the first FP64 assembly there); the FP32 stage's
// joint-phase counts are kept in iters32 / trials32. tid/nthreads: the calling
// threads of one query.
__device__ void restart_fp64(LMState& s, int k, int tid, int nthreads) {
  for (int i = tid; i < k; i += nthreads) {
    s.trial[i] = s.z[i];
    s.dz[i] = 0.0;
  }
  if (tid == 0) {
    // the FP32 stage's last result was evaluated at its final point (it ended on an
    // accepted step or at its start, not on a rejected trial): the H of the result
    // row is H there, which the first FP64-stage evaluation would recompute bit for
    // bit (the same FP32 pass at the same point), so that evaluation keeps it
    s.hkeep = s.res_at_z ? 1 : 0;
    s.iters32 = s.iters[1];
    s.trials32 = s.trials;
    s.iters[1] = 0;
    s.trials = 0;
    // a query stopped by a non-physical start stays stopped
    if (s.status != IFT_ERR_NONPHYSICAL) {
      s.phase = 1;
      s.state = 0;
      s.status = IFT_NOT_CONVERGED;
      s.h = 0;
      s.bodies = 0;
      s.done = 0;
      s.lam = kLam0;
      s.alpha = 1.0;
    }
  }
}

// The hand-over for B queries, one block each.
__global__ void lm_restart_kernel(LMState* states, int B, int ku, int kx) {
  const int q = blockIdx.x;
  if (q >= B) return;
  restart_fp64(states[q], ku + kx, threadIdx.x, blockDim.x);
}

// Block q: the FP64 gradient pass's [g | J | count] of query q (rows of k + 2 at g)
// into the [g | J | count] part of its full result row (res + q nacc); the
// non-physical counts of the two passes add up (the FP64 count alone when the FP32
// pass was skipped because H is kept). Finished queries are skipped.
__global__ void merge_grad_kernel(const double* g, int k, int nacc, double* res, const LMState* states) {
  const int q = blockIdx.x;
  if (states != nullptr && states[q].done) return;
  const bool kept = states != nullptr && states[q].hkeep;
  const double* src = g + (size_t)q * (k + 2);
  double* dst = res + (size_t)q * nacc + (size_t)k * k;
  for (int i = threadIdx.x; i < k + 2; i += blockDim.x) {
    if (i <= k || kept) dst[i] = src[i];
    else dst[i] += src[i];
  }
}

__global__ void residual_norms_finish_kernel(const double* part, int B, int nchunk, double* norms) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)q * nchunk + c];
  norms[q] = sqrt(s);
}

// Block b sums columns [32 b, 32 b + 32) of the partials: each of its warps (up to
// 32) sums one contiguous segment of the rows (coalesced 32-column reads, eight rows
// in flight per lane), then warp 0 adds the segment sums in segment order (the
// order is fixed for a launch shape).
// skip (optional): a device flag; when non-zero the block returns at once and out is
// left as it is (a finished solve, or an evaluation that keeps H).
__global__ void __launch_bounds__(1024) reduce_partials_kernel(const double* partial, int nparts, int nacc,
                                                              double* out, const int* skip) {
  if (skip != nullptr && *skip) return;
  __shared__ double seg[32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int per = (nparts + nw - 1) / nw, c0 = w * per, c1 = min(nparts, c0 + per);
  double s = 0.0;
  if (i < nacc) {
    int c = c0;
    for (; c + 8 <= c1; c += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = partial[(size_t)(c + u) * nacc + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; c < c1; ++c) s += partial[(size_t)c * nacc + i];
  }
  seg[w][lane] = s;
  __syncthreads();
  if (w == 0 && i < nacc) {
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += seg[k][lane];
    out[i] = t;
  }
}

// w_guess = Phi^T U_guess, U_guess the constant state (Burgers u = 1, Euler U_inf(mu))
// at every node. Block b sums rows [b*chunk, (b+1)*chunk) into part[b][c].
__global__ void phit_u_partial_kernel(const double* Phi, long Nu, int ku, int m, int problem, double gamma,
                                      const double* mu, long chunk, double* part) {
  extern __shared__ double sh[];
  double Ug[4];
  if (problem == 2) {
    euler_farfield(gamma, mu[0], mu[1], Ug);
  } else {
    Ug[0] = 1.0;
  }
  const long r0 = (long)blockIdx.x * chunk;
  const long r1 = (r0 + chunk < Nu) ? r0 + chunk : Nu;
  const int lanes_per_col = blockDim.x / ku;  // >= 1 (blockDim >= ku)
  const int c = threadIdx.x % ku, sub = threadIdx.x / ku;
  double s = 0.0;
  if (sub < lanes_per_col)
    for (long r = r0 + sub; r < r1; r += lanes_per_col) s += Phi[r * ku + c] * Ug[r % m];
  sh[threadIdx.x] = (sub < lanes_per_col) ? s : 0.0;
  __syncthreads();
  if (threadIdx.x < ku) {
    double t = 0.0;
    for (int j = 0; j < lanes_per_col; ++j) t += sh[j * ku + threadIdx.x];
    part[(size_t)blockIdx.x * ku + threadIdx.x] = t;
  }
}

__global__ void sum_columns_kernel(const double* part, int nparts, int ku, double* w) {
  const int c = threadIdx.x;
  if (c >= ku) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += part[(size_t)b * ku + c];
  w[c] = s;
}

// ---------------------------------------------------------------------------
// Vector kernels of the snapshot alignment's conjugate-gradient solve.
// ---------------------------------------------------------------------------

// Block b: the partial dot product of a and b over its grid-stride share, into part[b]
// (summed on the host in block order).
__global__ void dot_partial_kernel(const double* a, const double* b, long n, double* part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// y = y + alpha x
__global__ void axpy_kernel(long n, double alpha, const double* x, double* y) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] += alpha * x[i];
}

// x[idx[j]] = v[j] (the free mesh coordinates of a step in the unknowns' space)
__global__ void scatter_free_kernel(const int* idx, int nfree, const double* v, double* x) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nfree; j += gridDim.x * blockDim.x) x[idx[j]] = v[j];
}

// The w rows of the alignment products: out[c] = sum_b part[b][c] (block order) plus
// mode 0: (H_ww dw)_c, mode 2: H_ww[c][c], mode 1: nothing (H packed upper, acc_h
// order); one warp per row.
__global__ void align_wrows_kernel(const double* part, int nparts, int ku, const double* H, const double* dw,
                                   int mode, double* out) {
  const int lane = threadIdx.x & 31, c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ku) return;
  double s = 0.0;
  for (int b = lane; b < nparts; b += 32) s += part[(size_t)b * ku + c];
  if (mode == 0) {
    for (int j = lane; j < ku; j += 32) {
      const int r = j < c ? j : c, b = j < c ? c : j;
      s += H[r * ku - (r * (r - 1)) / 2 + (b - r)] * dw[j];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    if (mode == 2) s += H[c * ku - (c * (c - 1)) / 2];
    out[c] = s;
  }
}

// Preconditioned conjugate gradients on (J^T J + lam D) d = -g with the Jacobi
// preconditioner m = diag(J^T J) + lam D (D = 1 on the mesh rows, the first ku
// rows are the state coefficients). The scalars stay on the device; once done is
// set an iteration changes nothing, and cg_beta_kernel ends the graph's loop.
__device__ __forceinline__ double cg_precond(const double* diag, const CGState* st, long i, int ku) {
  const double m = diag[i] + (i >= ku ? st->lam : 0.0);
  return m > 0.0 ? 1.0 / m : 1.0;
}

// Block partial sums of (a . a, a . b) into part[2 blk], part[2 blk + 1]
__device__ __forceinline__ void block_dot2(double s0, double s1, double* part) {
  __shared__ double sh[2][256];
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sh[0][0];
    part[2 * blockIdx.x + 1] = sh[1][0];
  }
}

// p's free mesh entry j into its element slots (CSR: slots[off[j] .. off[j + 1]) of
// the element-order direction xdir)
__device__ __forceinline__ void scatter_slots(const int* off, const int* slots, long j, double v, double* xdir) {
  for (int q = off[j]; q < off[j + 1]; ++q) xdir[slots[q]] = v;
}

// d = 0, r = -g, z = M^{-1} r, p = z (its mesh part also into xdir); partials of
// r . r and r . z (256 threads per block)
__global__ void cg_start_kernel(long n, int ku, const double* g, const double* diag, const CGState* st, double* d,
                                double* r, double* z, double* p, double* part, const int* off, const int* slots,
                                double* xdir) {
  double s0 = 0.0, s1 = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double ri = -g[i], zi = ri * cg_precond(diag, st, i, ku);
    d[i] = 0.0;
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
    if (i >= ku) scatter_slots(off, slots, i - ku, zi, xdir);
    s0 += ri * ri;
    s1 += ri * zi;
  }
  block_dot2(s0, s1, part);
}

// Sums of the pair partials (a . a, a . b) by one warp in a fixed order
__device__ __forceinline__ void warp_sum2(const double* part, int nblk, double& s0, double& s1) {
  const int lane = threadIdx.x & 31;
  s0 = 0.0;
  s1 = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    s0 += part[2 * b];
    s1 += part[2 * b + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
}

// Ap = (J^T J + lam D) p from the product kernel's outputs, and the partials of
// p . Ap (block b into dotpart[b]; 256 threads, gridDim >= ku): the free mesh rows
// Ap[ku + j] = sum of yslot over the coordinate's slots (CSR order) + lam p[ku + j],
// and block c < ku the w row Ap[c] = sum_b part[b][c] + (H_ww p_w)_c (H packed upper,
// acc_h order). Every sum runs in a fixed order.
__device__ __forceinline__ double block_sum256(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double t = sh[0];
  __syncthreads();
  return t;
}

__global__ void align_finish_kernel(const double* part, int nparts, int ku, const double* H, const double* p,
                                    int nfree, const double* yslot, const int* off, const int* slots,
                                    const CGState* st, double* Ap, double* dotpart) {
  __shared__ double sh[256];
  const double lam = st->lam;
  double s = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nfree; j += gridDim.x * blockDim.x) {
    double a = lam * p[ku + j];
    for (int q = off[j]; q < off[j + 1]; ++q) a += yslot[slots[q]];
    Ap[ku + j] = a;
    s += p[ku + j] * a;
  }
  double wrow = 0.0;
  if (blockIdx.x < ku) {
    const int c = blockIdx.x;
    double t = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) t += part[(size_t)b * ku + c];
    for (int j = threadIdx.x; j < ku; j += blockDim.x) {
      const int r = j < c ? j : c, q = j < c ? c : j;
      t += H[r * ku - (r * (r - 1)) / 2 + (q - r)] * p[j];
    }
    wrow = block_sum256(t, sh);
    if (threadIdx.x == 0) Ap[c] = wrow;
  }
  const double tot = block_sum256(s, sh);
  if (threadIdx.x == 0) dotpart[blockIdx.x] = tot + (blockIdx.x < ku ? p[blockIdx.x] * wrow : 0.0);
}

// (one warp)
__global__ void cg_start_finish_kernel(const double* part, int nblk, CGState* st) {
  double rr, rz;
  warp_sum2(part, nblk, rr, rz);
  if (threadIdx.x != 0) return;
  st->rr0 = rr;
  st->rz = rz;
  st->alpha = 0.0;
  st->beta = 0.0;
  st->iters = 0;
  st->done = (rr > 0.0 && rz > 0.0) ? 0 : 1;
}

// alpha = r.z / p.Ap from the partials of p . Ap (pap_part: nblk values, reduced
// by every block in the same order, so that all blocks take the same decision;
// block 0 records the iteration), then d += alpha p, r -= alpha Ap,
// z = M^{-1} r and the partials of r . r and r . z into part (256 threads)
__global__ void cg_update_kernel(long n, int ku, const double* pap_part, int nblk, CGState* st, const double* p,
                                 const double* Ap, const double* diag, double* d, double* r, double* z,
                                 double* part) {
  __shared__ double sp;
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) v += pap_part[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sp = v;
  }
  __syncthreads();
  const double pap = sp;
  const bool was_done = st->done != 0;
  const bool live = !was_done && pap > 0.0;
  const double a = live ? st->rz / pap : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && !was_done) {
    ++st->iters;
    if (!live) st->done = 1;
  }
  double s0 = 0.0, s1 = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double ri = r[i];
    if (live) {
      d[i] += a * p[i];
      ri -= a * Ap[i];
      r[i] = ri;
      const double zi = ri * cg_precond(diag, st, i, ku);
      z[i] = zi;
      s1 += ri * zi;
    }
    s0 += ri * ri;
  }
  block_dot2(s0, s1, part);
}

// convergence test and beta; inside the solve's graph (use_cond) sets its loop
// condition: continue while not done (one warp)
__global__ void cg_beta_kernel(const double* part, int nblk, CGState* st, unsigned long long cond_handle,
                               int use_cond) {
  double rr, rz;
  warp_sum2(part, nblk, rr, rz);
  if (threadIdx.x != 0) return;
  st->beta = 0.0;
  if (!st->done) {
    if (!(rr <= st->tol * st->tol * st->rr0) && rr == rr && rz > 0.0 && st->iters < st->max_iters) {
      st->beta = rz / st->rz;
      st->rz = rz;
    } else {
      st->done = 1;
    }
  }
  if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, st->done ? 0u : 1u);
}

// p = z + beta p (its mesh part also into xdir)
__global__ void cg_dir_kernel(long n, int ku, const CGState* st, const double* z, double* p, const int* off,
                              const int* slots, double* xdir) {
  if (st->done) return;
  const double b = st->beta;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double v = z[i] + b * p[i];
    p[i] = v;
    if (i >= ku) scatter_slots(off, slots, i - ku, v, xdir);
  }
}

// out[j] = the sum of yslot over free coordinate j's slots in CSR order (the free
// mesh rows of a product)
__global__ void take_free_kernel(int nfree, const double* yslot, const int* off, const int* slots, double* out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nfree; j += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int q = off[j]; q < off[j + 1]; ++q) a += yslot[slots[q]];
    out[j] = a;
  }
}

}  // namespace ift
