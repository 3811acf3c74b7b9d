// Levenberg-Marquardt driver of the hyperreduced problem on the device (Sec. 3.2.3).
//
// The solve is a loop of identical bodies [assemble at the trial point ->
// reduce -> lm_step]; lm_step reads the assembled (H, g, J) at the trial point,
// accepts or rejects it by the sufficient-decrease test, updates lambda, checks
// the stopping test, and on acceptance solves (H + diag(0, lambda I)) dz = -g by
// Cholesky and writes the next trial point z + dz. A rejected trial halves the
// step. Because the assembly at an accepted trial point is the assembly at the
// new iterate, every LM iteration costs one fused assembly pass in the common
// case (full step accepted).
#pragma once
#include <cuda_runtime.h>

namespace ift {

constexpr int LM_KMAX = 64;

struct LMConsts {
  double tol;
  int max_iters;
  int ku, kx;
  int body_limit;   // hard bound on loop bodies (then IFT_ERR_TIMEOUT)
  int max_halvings; // line-search halvings before the phase ends (30; fewer in the FP32 stage of a mixed solve)
  int keep_h;       // 1: after a full step, the next evaluation keeps H (the finishing stage of a mixed solve)
};

// Device-resident solver state (one per query).
struct LMState {
  int phase;        // 0: w only (tau frozen), 1: joint (w, tau), 2: finished
  int state;        // 0: the pending assembly is at the starting point, 1: at a trial point
  int status;       // ift_status
  int init_status;  // status at the end of phase 0
  int iters[2];     // accepted steps per phase
  int trials, shifts, h, bodies, done;
  int iters32, trials32;  // joint-phase steps and trials of the FP32 stage of a mixed solve
  int hkeep;        // 1: the next evaluation leaves H as it is (no FP32 Jacobian pass)
  int hevals;       // evaluations with keep_h that recomputed H
  int res_at_z;     // 1: the result the last step read was evaluated at the current iterate z
  double lam, alpha, J, slope, g0, thresh;
  double z[LM_KMAX];      // current iterate (w | tau)
  double dz[LM_KMAX];     // step
  double g[LM_KMAX];      // gradient [S; T] at the current iterate
  double trial[LM_KMAX];  // point of the next assembly (w | tau)
};

// Device-resident scalars of the snapshot alignment's preconditioned conjugate-
// gradient solve (one CUDA graph per Levenberg-Marquardt step; see cg_*_kernel).
struct CGState {
  double lam;    // damping of the mesh rows
  double tol;    // stop when |r| <= tol |r_0|
  double rz;     // r . z of the current iterate
  double rr0;    // |r_0|^2
  double alpha;  // step length of the current iteration (0 once done)
  double beta;   // direction update of the current iteration
  int done;      // converged, broken down or out of iterations: later iterations change nothing
  int iters;     // products with the normal matrix taken
  int max_iters;
  int pad;
};

}  // namespace ift
