/*
 * ift.h -- C ABI of the GB300 implementation of the EQP-IFT online hot path
 * (implicit feature tracking with empirical quadrature, arXiv 2305.15661).
 *
 * The library evaluates, on one GPU, the weighted reduced residuals and
 * Gauss-Newton system of the hyperreduced implicit-feature-tracking model and
 * solves it with Levenberg-Marquardt:
 *   state U = Phi w, mesh x = X + Psi tau                      (Sec. 3.1)
 *   S~ = sum_e rho_e (Phi_e^T dR_e/dU_e^T + Phi_e'^T dR_e/dU_e'^T) R_e
 *   T~ = sum_e rho_e Psi_e^T (dR_e/dx_e^T R_e + dN_e/dx_e^T N_e)  (Eqs. ift-eqp-res0, ift-res-elem2)
 *   H  = sum_e rho_e [A_w A_t]^T [A_w A_t] (+ distortion block)  (Eq. levmarq-elem)
 *   J~ = sum_e rho_e (|R_e|^2 + N_e^2) / 2                         (Eq. ift-opt-eqp2)
 * with A_w = dR_e/dU_e Phi_e + dR_e/dU_e' Phi_e', A_t = dR_e/dx_e Psi_e.
 * The paper's notation w, tau is written y, z in the argument names.
 *
 * Conventions for every call:
 *  - All pointers are HOST pointers unless the function name ends in "_dev";
 *    host inputs are copied in and the caller keeps ownership. "_dev" calls take
 *    device pointers and run on the stream given at ift_create (or the stream
 *    argument), asynchronously, and write their outputs to caller buffers.
 *  - Floating-point inputs and outputs are IEEE double, integers int32/int64,
 *    all arrays dense and row-major (C order).
 *  - Degrees of freedom are element-major: DOF index = e*n_u + node*m + var, with
 *    n_u = n_b*m (m = 1 Burgers, m = 4 Euler); nodal order per element as
 *    ift_reference_nodes() reports. Mesh coordinates are vertex-major:
 *    x[v*dim + c].
 *  - Call order: ift_create -> ift_set_mesh -> ift_set_bases -> (ift_set_eq_weights)
 *    -> evaluate / solve. Out-of-order calls return IFT_ERR_STATE. Without
 *    ift_set_eq_weights every element has weight 1 (the unweighted ROM,
 *    Remark rom-eqp-ones).
 *  - Errors are returned as status codes; ift_last_error() gives the message.
 *    No call aborts, traps or prints. A failed call leaves the context usable.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef IFT_H
#define IFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ift_ctx ift_ctx;

typedef enum {
  IFT_OK = 0,
  IFT_NOT_CONVERGED = 1,     /* solver hit max_iters; outputs are the last iterate */
  IFT_LINESEARCH_FAILED = 2, /* no step length in 1, 1/2, ..., 2^-30 gave sufficient decrease */
  IFT_ERR_ARG = -1,          /* bad argument (size, pointer, degree, mesh orientation) */
  IFT_ERR_STATE = -2,        /* call out of order */
  IFT_ERR_CUDA = -3,         /* CUDA runtime error (message in ift_last_error) */
  IFT_ERR_OOM = -4,          /* device allocation failed */
  IFT_ERR_NONPHYSICAL = -5,  /* evaluation point has g <= 0, rho <= 0 or P <= 0, or non-finite R */
  IFT_ERR_TIMEOUT = -6,      /* a bounded device wait ran out */
  IFT_ERR_NOTIMPL = -7       /* combination of options not built */
} ift_status;

enum { IFT_BURGERS1D = 1, IFT_EULER2D = 2 };
/* Arithmetic of the element evaluation and contraction. IFT_FP64: all FP64.
   IFT_FP32: FP32 element kernels and contraction, FP32 sums within a warp's
   elements, FP64 sums across warps and CTAs. IFT_MIXED: evaluation calls as
   IFT_FP32; solves run the LM with FP32 assemblies to a relative optimality of
   1e-6 (or tol if larger), or until a line search needs more than one halving
   (FP32 rounding in J~ ends the FP32 stage), then continue from that point to
   tol with the IFT_FP32_JACOBIAN evaluation (H from FP32, S~, T~, J~ in FP64),
   where H is recomputed only at the first point of that stage and after a
   rejected or shortened step (a full step keeps it: H only steers the step).
   The LM normal equations, line search and stopping test are FP64 in every mode. */
enum { IFT_FP64 = 0, IFT_FP32 = 1, IFT_MIXED = 2, IFT_FP32_JACOBIAN = 3 };
/* IFT_FP32_JACOBIAN: every LM iteration (and every evaluation call) takes the
   Gauss-Newton matrix H from the FP32 element Jacobians and contraction (tensor
   cores with IFT_CONTRACT_TF32 / _3XTF32) and S~, T~, J~ from an FP64 pass that
   evaluates R_e and applies the transposed element Jacobian to it (no Jacobian
   columns formed). The optimality test, the line search and the normal
   equations are FP64, so a solve converges to the FP64 optimum; H only steers the
   step. */
/* How FP32 evaluations form H += rho A_e^T A_e (Eq. levmarq-elem): FP = FP32
   fused multiply-adds; TF32 = tensor cores with TF32 inputs (10-bit mantissa)
   and FP32 accumulation, H to about 1e-3 relative; 3XTF32 = tensor cores with
   each operand split into two TF32 parts (three products), H to about FP32
   accuracy; BF16 = tensor cores with BF16 inputs (7-bit mantissa) and FP32
   accumulation, H to a few 1e-3 relative. S~, T~ and J~ are FP32 fused
   multiply-adds in every mode, so the optimum of a solve does not depend on this
   choice (H only steers the step). With BF16, the single-query FP32 evaluations
   (ift_reduced_residual_jacobian, ift_solve_rom) form H with tcgen05 products from
   a stack of the rows of sqrt(rho_e) A_e in BF16, which takes (k_u + k_x) x
   (items x n_u) x 2 bytes of device memory (items: the elements with nonzero
   weight; 307 MB for 80,000 p = 3 elements at k = 48), allocated when the weights
   are set or first used; a bounded wait there that runs out makes the evaluation
   or the solve return IFT_ERR_TIMEOUT (ift_solve_rom_dev: when it is given
   info_host). The batched calls keep warp-level tensor-core tiles. */
enum { IFT_CONTRACT_FP = 0, IFT_CONTRACT_TF32 = 1, IFT_CONTRACT_3XTF32 = 2, IFT_CONTRACT_BF16 = 3 };
/* LM start: PAPER = w from Phi^T U_guess then LM on w with tau = 0, then joint
   LM (Remark rem:solver); GIVEN = start the joint LM at the caller's (y, z). */
enum { IFT_INIT_PAPER = 0, IFT_INIT_GIVEN = 1 };

typedef struct {
  int problem;        /* IFT_BURGERS1D or IFT_EULER2D */
  int p;              /* DG degree: Burgers 1..3, Euler 1..3 */
  int precision;      /* IFT_FP64, IFT_FP32 or IFT_MIXED */
  double gamma;       /* ratio of specific heats (Euler) */
  double kappa;       /* distortion weight kappa of Eq. dist_elem0 (>= 0) */
  double eps_g;       /* epsilon of Eq. dist_elem1 (the paper uses 1e-8) */
  double tol;         /* stop when |[S~;T~]| <= tol * max(1, |[S~;T~]| at phase start) */
  int max_iters;      /* per LM phase */
  int lm_init;        /* IFT_INIT_PAPER or IFT_INIT_GIVEN */
  int contraction;    /* IFT_CONTRACT_FP, _TF32, _3XTF32 or _BF16 (all but FP need a precision other than IFT_FP64) */
  int q;              /* geometry degree: 1 straight-sided, 2 curved six-node triangles (IFT_EULER2D only;
                         ift_set_mesh then takes the three vertices and the midpoint nodes of edges
                         0-1, 1-2, 2-0 of every element, and the mesh modes act on all those nodes) */
  double align_cg_tol; /* ift_align: relative residual at which each conjugate-gradient solve stops,
                          in [0, 1); 0 selects 1e-12, where every step is the exact Levenberg-Marquardt
                          step (within rounding); larger values take inexact steps (fewer CG iterations,
                          the same stopping test on |J^T F|) */
  int max_loop_bodies; /* bound on the LM loop bodies a solve (or a batched solve) runs on the device, each
                          body one evaluation at a trial point and one LM step; 0 selects
                          (2 max_iters + 4) * 34, which no solve within max_iters per phase reaches. When
                          the bound is reached the solve ends with IFT_ERR_TIMEOUT, the last accepted
                          point in y, z, and the context stays usable. The bound is a count kept by the
                          LM step kernel: nothing on the device waits or spins. */
} ift_config;

/* Fills cfg with the defaults: gamma 1.4, kappa 0, eps_g 1e-8, tol 1e-8,
   max_iters 200, FP64, IFT_INIT_PAPER, IFT_CONTRACT_FP, align_cg_tol 1e-12,
   max_loop_bodies 0. */
void ift_config_default(ift_config* cfg);

/* Creates a context on the current CUDA device. stream: a cudaStream_t to run on
   (NULL = a stream owned by the context). Returns IFT_ERR_ARG for a bad problem
   or degree, IFT_ERR_CUDA if no device is usable. */
ift_status ift_create(const ift_config* cfg, void* stream, ift_ctx** out);
ift_status ift_destroy(ift_ctx* ctx);
const char* ift_last_error(const ift_ctx* ctx);
/* Message for a failed ift_create (thread-local). */
const char* ift_create_error(void);

/* Reference element of the context: nodes (n_b x dim master coordinates:
   [0,1] for Burgers, triangle (0,0),(1,0),(0,1) for Euler) and, per face, its
   p+1 trace nodes in the face's direction (n_face x n_trace). Sizes come from
   ift_sizes. */
ift_status ift_reference_nodes(const ift_ctx* ctx, double* nodes, int32_t* face_nodes);

/* sizes[0..7] = n_b, n_u, n_u' (neighbour trace DOFs per element), n_x per element,
   n_face, n_trace, n_q (volume points), n_fq (points per face). */
ift_status ift_sizes(const ift_ctx* ctx, int64_t* sizes);

/* Mesh (Sec. 2.3, Eq. hdm_elem): reference nodes X (n_verts x dim) and simplices
   elem_verts (n_elems x (dim+1)), counter-clockwise (Burgers: left to right).
   Faces are matched by shared vertices; unmatched faces are boundary faces:
   Euler far field U_inf(mu); Burgers inflow u = 1 on the face with outward
   normal -x, outflow (exterior = interior state) on the other.
   Returns IFT_ERR_ARG for an inverted element or a face shared three times. */
ift_status ift_set_mesh(ift_ctx* ctx, int64_t n_verts, const double* X, int64_t n_elems,
                        const int32_t* elem_verts);

/* Bases of the implicit-feature-tracking manifold (Sec. 3.1): Phi (N_u x k_u),
   Psi (N_x x k_x), N_u = n_elems*n_u, N_x = n_verts*dim. k_u >= 1, k_x >= 0,
   k_u + k_x <= 64. */
ift_status ift_set_bases(ift_ctx* ctx, int64_t N_u, int k_u, const double* Phi, int64_t N_x, int k_x,
                         const double* Psi);

/* Empirical-quadrature weights (Eq. ift-eqp-res0): nnz pairs (elem[i], rho[i]),
   elements distinct, rho > 0. nnz = -1 restores rho = 1 on every element.
   Only the listed elements (and their neighbours' trace rows of Phi) are read by
   the evaluation (the hyperreduced gather, Sec. 3.2.1). */
ift_status ift_set_eq_weights(ift_ctx* ctx, int64_t nnz, const int32_t* elem, const double* rho);

/* Weighted reduced residuals, Gauss-Newton matrix and objective at (y, z) = (w, tau):
   S (k_u), T (k_x), H ((k_u+k_x)^2, full symmetric), J (1). mu: problem
   parameters (Burgers: mu[0]; Euler: mu = (Mach, angle in radians)).
   Any output pointer may be NULL. Returns IFT_ERR_NONPHYSICAL (outputs written,
   J = +inf) when an element with non-zero weight is non-physical at (y, z). */
ift_status ift_reduced_residual_jacobian(ift_ctx* ctx, const double* mu, const double* y, const double* z,
                                         double* S, double* T, double* H, double* J);
ift_status ift_reduced_residual_jacobian_dev(ift_ctx* ctx, const double* mu, const double* y, const double* z,
                                             double* S, double* T, double* H, double* J, void* stream);

/* Per-element residuals and Jacobians at a full state (inspection of the
   element kernel): for each of the n listed elements, R_e (n_u), dR_e/dU_e
   (n_u x n_u), dR_e/dU_e' (n_u x n_u'), dR_e/dx_e (n_u x n_x), N_e and dN_e/dx_e
   (n_x), at global state U (N_u) and mesh x (N_x). U_e' is the neighbours'
   trace nodes, face by face, ordered along this element's face direction,
   m variables each (zero on boundary faces). Output pointers may be NULL. */
ift_status ift_element_eval(ift_ctx* ctx, const double* mu, const double* U, const double* x, int64_t n,
                            const int32_t* elems, double* R, double* JU, double* JUp, double* Jx, double* N,
                            double* dN);

typedef struct {
  int status;          /* ift_status of the solve */
  int init_iters;      /* accepted LM steps of the w-only initialisation */
  int iters;           /* accepted LM steps of the joint iteration */
  int trials;          /* objective evaluations in line searches */
  int shifts;          /* Cholesky diagonal shifts */
  double J;            /* final objective */
  double normS, normT; /* final |S~|, |T~| */
  double g0;           /* |[S~;T~]| at the start of the joint iteration */
  int fp32_iters;      /* mixed precision: joint-phase steps of the FP32 stage (iters counts the FP64 stage) */
  int fp32_trials;     /* mixed precision: objective evaluations of the FP32 stage */
  int h_evals;         /* mixed precision: evaluations of the FP64 stage that recomputed H (FP32
                          Jacobian pass); the others kept the H of an earlier one (at the
                          stage's first point, the FP32 stage's last H when it was evaluated
                          there) */
} ift_solve_info;

/* Levenberg-Marquardt solve of the hyperreduced problem (Sec. 3.2.3):
   (H + diag(0, lambda I)) dz = -[S~; T~], Armijo backtracking on J~,
   lambda_0 = 1e-4, lambda/10 after a full step, 10 lambda after a shortened one.
   With IFT_INIT_PAPER y and z are outputs only; with IFT_INIT_GIVEN they are
   also the start. Returns the final status (also in info->status). */
ift_status ift_solve_rom(ift_ctx* ctx, const double* mu, double* y, double* z, ift_solve_info* info);
ift_status ift_solve_rom_dev(ift_ctx* ctx, const double* mu, double* y, double* z, ift_solve_info* info_host,
                             void* stream);

/* Many queries (Sec. 3.2.1 for each parameter value): query q has its own
   sparse weight set, elements elem[offsets[q] .. offsets[q+1]) with weights rho
   (offsets has B+1 entries, offsets[0] = 0, every query non-empty, elements
   distinct within a query, rho > 0). Only the listed elements and their
   neighbours' trace rows are read (the hyperreduced gather). Replaces an earlier
   batched set; ift_set_bases clears it. */
ift_status ift_set_eq_weights_batched(ift_ctx* ctx, int B, const int64_t* offsets, const int32_t* elem,
                                      const double* rho);

/* S~, T~, H, J~ of every query at its own point: mu (B x n_mu), y (B x k_u),
   z (B x k_x) in; S (B x k_u), T (B x k_x), H (B x k x k), J (B) out (host).
   IFT_ERR_NONPHYSICAL if any query is non-physical (its J is +inf). */
ift_status ift_reduced_residual_jacobian_batched(ift_ctx* ctx, const double* mu, const double* y, const double* z,
                                                 double* S, double* T, double* H, double* J);

/* LM solves of all B queries in one CUDA graph: every loop body assembles all
   unfinished queries in one launch, reduces per query, steps each query's LM
   and tests whether any query is still running. Same iteration as
   ift_solve_rom per query. y (B x k_u), z (B x k_x) out (and in with
   IFT_INIT_GIVEN); info (B). Returns IFT_OK if every query converged, else the
   first error, else the first warning (each query's status is in info). */
ift_status ift_solve_rom_batched(ift_ctx* ctx, const double* mu, double* y, double* z, ift_solve_info* info);
/* Device-pointer variant: mu, y, z and status (B int32, may be NULL) are device
   pointers; asynchronous on stream (NULL: the context's stream). */
ift_status ift_solve_rom_batched_dev(ift_ctx* ctx, const double* mu, double* y, double* z, int32_t* status,
                                     void* stream);

/* Launch-shape autotuner (not part of the paper's method). Times the fused
   assembly of this context's workload at (mu, y, z) for 1, 2 and 4 warps per CTA,
   separately for each precision the context runs (mixed contexts run FP32 and
   FP64 kernels) and, when batched weights are set, the batched assembly for chunk
   sizes 4, 8, 16, 32 elements x 1, 2, 4 warps per CTA (scored on a full batch plus
   a tail with 2% of the queries running; the chunk size on the precision that
   dominates a solve, FP64 for mixed contexts), keeps the fastest shapes in the
   context and writes the evaluation precision's to chosen[0..2] = (warps per CTA,
   batched warps per CTA, chunk size). Shapes that need more shared memory than a
   CTA may have are skipped. Results change only by reduction order (all shapes
   compute the same sums). Default shapes without tuning: 2, 2, 8, fewer warps
   where the bases need more shared memory. */
ift_status ift_autotune(ift_ctx* ctx, const double* mu, const double* y, const double* z, int32_t* chosen);
/* Sets the launch shapes directly (for instance, shapes an earlier ift_autotune
   chose for the same workload): warps and batched_warps in {1, 2, 4}, chunk in
   {4, 8, 16, 32}; anything else, or warps whose shared memory does not fit the
   evaluation precision's kernels, is IFT_ERR_ARG. The FP64 kernels of a mixed
   context take the most warps up to these that fit. Results change only by
   reduction order. */
ift_status ift_set_launch_shapes(ift_ctx* ctx, int warps, int batched_warps, int chunk);

/* HDM residual norms at B points (the greedy-search indicator of Eq. greedy0):
   norms[q] = |R(Phi y_q, X + Psi z_q; mu_q)|_2, the full DG residual (every
   element, no empirical-quadrature weights, no distortion term) at the state and
   mesh of query q. mu (B x n_mu), y (B x k_u), z (B x k_x) in, norms (B) out; host
   pointers. A non-physical point gives +inf. FP64 contexts evaluate in FP64,
   FP32 and mixed contexts in FP32 (sums of squares in FP64). The greedy search
   takes the argmax over candidates of these norms at their hyperreduced solutions. */
ift_status ift_hdm_residual_norms(ift_ctx* ctx, int B, const double* mu, const double* y, const double* z,
                                  double* norms);

/* Per-element contributions to the reduced residuals (the columns of the EQP
   linear program, Eq. eqp-con): at (y, z) = (w, tau) and mu, for each of the n
   listed elements (n = -1: every element, in order) one row of k + 1 values,
   [S^(e) (k_u) | T^(e) (k_x) | J^(e)], such that the weighted residuals of
   Eq. ift-eqp-res0 are S~ = sum_e rho_e S^(e), T~ = sum_e rho_e T^(e) and
   J~ = sum_e rho_e J^(e) for any weights rho. out: host, n x (k + 1) (n_elems x
   (k + 1) for n = -1). The weights set on the context are not used. Returns
   IFT_ERR_NONPHYSICAL (rows of non-physical elements NaN, J^(e) = +inf) when an
   element is non-physical at (y, z). */
ift_status ift_element_gradients(ift_ctx* ctx, const double* mu, const double* y, const double* z, int64_t n,
                                 const int32_t* elems, double* out);

/* Allocation-free variant of ift_reduced_residual_jacobian_dev, for callers that
   cannot call cudaMalloc when they need the reduced system: code that owns all
   device memory through its own pool or arena and forbids other allocators,
   programs that reserve their whole memory budget at start-up, and
   latency-critical loops where an allocation would synchronise the device. It
   has no counterpart in the paper: it computes the same S~, T~, H, J~ (FP64) as
   the context-based call, without a context.

   Every pointer is a caller-owned DEVICE pointer: X (n_verts x dim),
   elem_verts (n_elems x (dim+1)), the face connectivity nbr / nbr_face
   (n_elems x n_face: neighbour element and its local face, -1 on boundary
   faces) and bc (n_elems x n_face: 0 interior, 1 far field (Euler) or inflow
   u = 1 (Burgers, the face with outward normal -x), 2 outflow (Burgers)),
   Phi (N_u x k_u), Psi (N_x x k_x), the weights (nnz pairs elem/rho, or
   nnz = -1 for rho = 1 on every element; repeated elements are each counted),
   mu, y, z, and the outputs S, T, H, J as in ift_reduced_residual_jacobian (any
   output may be NULL). stream: a cudaStream_t or NULL for the default stream.

   The call is asynchronous: its status covers only the host-side checks, and
   two outcomes show only in the outputs once the stream has reached them.
   - A non-physical state at some element (g <= 0, density or pressure <= 0)
     gives J = +inf with status IFT_OK (the context-based call returns
     IFT_ERR_NONPHYSICAL there, because it waits for the result).
   - The device checks, before any assembly, every index the element kernel
     will use for the listed elements (all elements when nnz = -1): the element
     ids, their vertex ids (< n_verts) and neighbour ids (< n_elems), and that
     every rho is finite and >= 0. On a violation no element is evaluated and
     every output is NaN.

   The call allocates nothing: its scratch (reference tables, an error flag,
   per-CTA partial sums, the reduced result) lives in an 8 MiB array in the
   library's device memory, held on every GPU that loads the library until the
   process exits. Limits: k_u + k_x <= 64, p in 1..3; larger sizes, bad
   pointers, nnz = 0 or nnz < -1 return IFT_ERR_ARG, CUDA failures IFT_ERR_CUDA
   (no message is stored: there is no context). The partial sums take
   k^2 + k + 2 doubles per CTA, so the grid is at most
   (1,048,576 - 1,504 - (k^2 + k + 2 rounded up to 32)) / (k^2 + k + 2) CTAs:
   about 250 at k = 64, still more than one per SM on a 152-SM GPU. The array is
   shared by all calls and keeps the last call's contents (each call clears the
   flag and overwrites what it reads); calls whose GPU work overlaps on one
   device (other streams or host threads) race on it and must be serialised by
   the caller. The first call on each device looks up the array's device
   address and copies the reference tables into it with a synchronous
   cudaMemcpy; later calls only launch kernels. */
ift_status ift_reduced_residual_jacobian_static(
    int problem, int p, int64_t n_verts, const double* X, int64_t n_elems, const int32_t* elem_verts,
    const int32_t* nbr, const int32_t* nbr_face, const int8_t* bc, const double* Phi, int k_u,
    const double* Psi, int k_x, int64_t nnz, const int32_t* elems, const double* rho, const double* mu,
    const double* y, const double* z, double gamma, double kappa, double eps_g, double* S, double* T,
    double* H, double* J, void* stream);

/* ---- Learned warm start of the LM solve --------------------------------------
   The paper starts every LM solve from the projected guess (Remark rem:solver).
   The calls below add an optional learned start: a fully connected network
   x (n_in) -> width (x depth hidden layers, GELU(z) = z (1 + erf(z / sqrt 2)) / 2)
   -> n_out (linear), trained on pairs (mu, [w; tau]) from converged solves and
   evaluated at new mu to give the (y, z) of an IFT_INIT_GIVEN solve. All
   network arithmetic runs in FP32 on the device (forward, backward, loss,
   Adam); host arrays are FP64 and are converted at the boundary.

   Parameters are flattened layer by layer as W_l (in x out, row-major, so a
   row of inputs times W_l gives the layer's pre-activation) followed by b_l. */
typedef struct ift_mlp ift_mlp;

/* Creates a network on the current device with W ~ N(0, 1/in) (splitmix64 and
   Box-Muller draws from seed) and b = 0. stream: cudaStream_t or NULL.
   IFT_ERR_ARG unless n_in, n_out >= 1, 0 <= depth <= 16, width >= 1 when depth > 0. */
ift_status ift_mlp_create(int n_in, int width, int depth, int n_out, uint64_t seed, void* stream, ift_mlp** out);
ift_status ift_mlp_destroy(ift_mlp* net);
ift_status ift_mlp_num_params(const ift_mlp* net, int64_t* count);
/* Host copies of the parameters (FP64 in, FP64 out; stored as FP32). */
ift_status ift_mlp_get_params(const ift_mlp* net, double* params);
ift_status ift_mlp_set_params(ift_mlp* net, const double* params);

/* Per-column standardisation of inputs and targets (set by ift_mlp_train, used by
   ift_mlp_predict; identity after ift_mlp_create): means and standard deviations,
   n_in and n_out values each. set: standard deviations must be positive, means
   finite, else IFT_ERR_ARG. With the parameters they restore a trained network. */
ift_status ift_mlp_get_scaling(const ift_mlp* net, double* x_mean, double* x_std, double* t_mean, double* t_std);
ift_status ift_mlp_set_scaling(ift_mlp* net, const double* x_mean, const double* x_std, const double* t_mean,
                               const double* t_std);

/* Mean-squared-error loss L = sum (Y - t)^2 / (count n_out) of the network on
   count rows x (count x n_in) against t (count x n_out), both taken as the
   network's own inputs and targets (no normalisation), and its gradient with
   respect to the flattened parameters (grad may be NULL). 1 <= count <= 2^20. */
ift_status ift_mlp_loss_grad(ift_mlp* net, int64_t count, const double* x, const double* t, double* loss,
                             double* grad);

/* Trains on count pairs (x, t): inputs and targets are first standardised per
   column (mean 0, standard deviation 1, kept in the network for predict), then
   `epochs` passes of Adam (beta 0.9 / 0.999, eps 1e-8) over mini-batches of
   `batch` rows in a seeded random order (the last partial batch of an epoch is
   dropped); the step of update t of T is lr (0.01 + 0.99 (1 + cos(pi t / T)) / 2),
   from lr down to lr / 100. final_loss (may be NULL): the loss over all pairs in
   the standardised variables after training. */
ift_status ift_mlp_train(ift_mlp* net, int64_t count, const double* x, const double* t, int epochs, int batch,
                         double lr, uint64_t seed, double* final_loss);

/* out (count x n_out) = the network at x (count x n_in), in the caller's
   variables (standardisation applied and undone). */
ift_status ift_mlp_predict(ift_mlp* net, int64_t count, const double* x, double* out);

/* The same evaluation as ift_mlp_predict with every product of width inputs (the
   hidden-to-hidden layers and the output layer) on the tensor cores: BF16
   operands (the FP32 parameters and the GELU outputs rounded to BF16), FP32
   accumulation and FP32 bias and GELU; the first layer (n_in inputs) stays FP32.
   One CTA evaluates 128 queries through every layer. Outputs agree with
   ift_mlp_predict to the BF16 rounding of the operands (about 1e-2 relative).
   IFT_ERR_NOTIMPL unless depth >= 1, n_in <= 32, width a multiple of 16 in
   [16, 256] and n_out <= 256; IFT_ERR_TIMEOUT if a bounded device wait for the
   tensor cores ran out. */
ift_status ift_mlp_predict_bf16(ift_mlp* net, int64_t count, const double* x, double* out);

/* The start the learned one is compared with: for each query, the outputs of
   the nearest training point, y_out[q] = y_train[argmin_t |scale (x_q - x_t)|]
   (scale: n_in per-column factors, NULL = 1; the lowest index wins ties).
   Computed on the device. */
ift_status ift_nearest_start(int64_t n_train, int n_in, const double* x_train, int n_out, const double* y_train,
                             int64_t n_query, const double* x_query, const double* scale, double* y_out);

/* ------------------------------------------------------------------------
   Snapshot alignment (Eq. align0): the full-space problem
     min over (w, x) of (1/2) |F(Phi w, x; mu)|^2,  F = [R(Phi w, x; mu); N(x)],
   every element with weight 1, the free mesh coordinates x (all nodes, N_x =
   n_verts x dim values, the coordinate entries whose free_mask byte is non-zero)
   and w (k_u) unknown. Needs set_mesh and set_bases (Psi is not used: the mesh
   moves freely); FP64 in every precision.
   ------------------------------------------------------------------------ */
typedef struct {
  int status;    /* IFT_OK, IFT_NOT_CONVERGED (max_iters), IFT_LINESEARCH_FAILED */
  int iters;     /* accepted Levenberg-Marquardt steps */
  int cg_iters;  /* conjugate-gradient iterations over all steps (one J v and one J^T v each) */
  int trials;    /* objective evaluations in line searches */
  double J;      /* final (1/2)|F|^2 */
  double gnorm;  /* final |J^T F| over the unknowns */
  double g0;     /* |J^T F| at the start */
  /* device time (ms, CUDA events on the context's stream) of the phases: forming the
     stored element blocks with F, J^T F and diag(J^T J) at each accepted point; the
     conjugate-gradient solves; the line searches */
  double ms_form, ms_cg, ms_search;
} ift_align_info;

/* F = [R (N_u); N (n_elems)] at (w, x) (host pointers; x: N_x reference-layout
   coordinates of the current mesh; the distortion compares with the mesh of
   ift_set_mesh). */
ift_status ift_align_residual(ift_ctx* ctx, const double* mu, const double* w, const double* x, double* F);

/* dF = J (dU, dx) = [dR/dU dU + dR/dx dx; dN/dx dx] at (w, x): dU (N_u), dx (N_x). */
ift_status ift_align_jvp(ift_ctx* ctx, const double* mu, const double* w, const double* x, const double* dU,
                         const double* dx, double* dF);

/* (gU, gx) = J^T v: gU = (dR/dU)^T v_R (N_u), gx = (dR/dx)^T v_R + (dN/dx)^T v_N (N_x),
   v = [v_R (N_u); v_N (n_elems)]. */
ift_status ift_align_vjp(ift_ctx* ctx, const double* mu, const double* w, const double* x, const double* v,
                         double* gU, double* gx);

/* Levenberg-Marquardt on (w, free x) from the given (w, x) (both in/out). At each
   accepted point one element pass stores every element's share of the Gauss-Newton
   system on the device (the blocks coupling its mesh coordinates, and the state
   block summed over the elements), k_u n_xe + n_xe^2 + k_u + n_xe doubles per
   element. Each step then solves (J^T J + lambda D) d = -J^T F (D = 1 on the mesh
   coordinates, 0 on w) by Jacobi-preconditioned conjugate gradients to a relative
   residual of 1e-12 (at most min(4 n + 20, 2000) iterations, n the unknowns), run as
   one CUDA graph, followed by a backtracking line search on (1/2)|F|^2; lambda rules
   as ift_solve_rom. Stops when |J^T F| <= tol max(1, |J^T F| at the start).
   free_mask: N_x bytes, non-zero for a free coordinate. Requires k_u + n_xe <= 96.
   Errors: IFT_ERR_ARG (null pointers, tol < 0, max_iters < 0, sizes),
   IFT_ERR_NONPHYSICAL (the start is not physical), IFT_ERR_CUDA / IFT_ERR_OOM.
   Returns info->status (IFT_OK, IFT_NOT_CONVERGED or IFT_LINESEARCH_FAILED). */
ift_status ift_align(ift_ctx* ctx, const double* mu, double* w, double* x, const uint8_t* free_mask, double tol,
                     int max_iters, ift_align_info* info);
/* ift_align with device pointers for mu, w, x (in/out) and free_mask, on `stream`
   (NULL: the context's). The Levenberg-Marquardt loop decides on the host, so the
   call synchronises the stream before it returns; info_host may be NULL. */
ift_status ift_align_dev(ift_ctx* ctx, const double* mu, double* w, double* x, const uint8_t* free_mask,
                         double tol, int max_iters, ift_align_info* info_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* IFT_H */
