// Element kernels of the EQP-IFT hot path (device code).
//
// One warp evaluates one element at a time (a grid-stride loop over a list of
// (element, weight) items, so the same kernel serves the full assembly with
// rho = 1 and the hyperreduced gather over the sampled elements):
//   1. gather Phi_e and Psi_e into the warp's shared memory by asynchronous
//      copies (cp.async, all in flight at once); the neighbours' trace rows
//      Phi_e' are read from global memory (mostly L2 hits) where they are used;
//   2. U_e = Phi_e w, U_e' = Phi_e' w, x_e = X_e + Psi_e tau        (Sec. 3.1)
//   3. straight-sided geometry: cofactor matrix g J^{-T} of the element map
//      and scaled face normals (Eq. p2r-flux; Nanson's formula);
//   4. lanes split the quadrature points: contravariant volume fluxes and flux
//      Jacobians, Roe fluxes and their derivatives (dual numbers) at face points;
//   5. lanes split the residual entries: R_e (Eq. hdm_elem, DG weak form);
//   6. lane c forms column c of A_e = [dR_e/dU_e Phi_e + dR_e/dU_e' Phi_e' |
//      dR_e/dx_e Psi_e] as a Jacobian-vector product (Eq. levmarq-elem);
//   7. lanes split the rows of the weighted contraction
//      H += rho A^T A, g += rho A^T R, J += rho |R|^2/2 (+ distortion terms)
//      into the warp's accumulators (Eqs. ift-eqp-res0, levmarq-elem, ift-opt-eqp2).
// At the end each CTA sums its warps' accumulators in warp order and writes one
// FP64 partial; a second kernel sums the partials in a fixed order. The result is
// deterministic for a fixed launch shape.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "physics.cuh"

namespace ift {

// Asynchronous global -> shared copies (cp.async, sm_80 and later): a lane issues
// its copies, then commit + wait; every copy of the group is in flight at once.
// 16-byte copies need both addresses 16-byte aligned; the 4- and 8-byte forms need
// their own size alignment.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// every committed group but the newest has landed (this thread's copies)
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Copy n values of T from global src to shared dst (dst 16-byte aligned) by the warp's
// lanes with cp.async: 16-byte pieces when src is 16-byte aligned and n T fill whole
// pieces, else one value per copy. The caller waits (cp_async_wait_all + __syncwarp).
template <class T>
__device__ __forceinline__ void warp_copy_async(T* dst, const T* src, int n, int lane, int step = 32) {
  constexpr int V = 16 / sizeof(T);
  if (((uintptr_t)src & 15) == 0 && n % V == 0) {
    for (int i = lane * V; i < n; i += step * V) cp_async16(dst + i, src + i);
  } else {
    for (int i = lane; i < n; i += step) {
      if (sizeof(T) == 8) cp_async8(dst + i, src + i);
      else cp_async4(dst + i, src + i);
    }
  }
}

// Lanes that work on one element: the whole warp (step 32, lane = 0..31) or, where a
// warp carries two elements (the gradient pass), the calling lane's half-warp (step 16,
// lane = 0..15 within it). Any over those lanes; every lane of the warp must call it.
__device__ __forceinline__ bool group_any(bool v, int step) {
  if (step == 32) return __any_sync(0xffffffffu, v);
  const unsigned m = __ballot_sync(0xffffffffu, v);
  return ((threadIdx.x & 16) ? (m >> 16) : (m & 0xffffu)) != 0;
}

// Per-warp accumulators: the upper triangle of H row by row (k (k + 1) / 2 entries),
// then g (k), J and the non-physical count. Position of H[r][b], r <= b:
__host__ __device__ inline int acc_h(int r, int b, int k) { return r * k - (r * (r - 1)) / 2 + (b - r); }
__host__ __device__ inline int acc_tail(int k) { return k * (k + 1) / 2; }
__host__ __device__ inline int acc_count(int k) { return k * (k + 1) / 2 + k + 2; }

// Element-list items, state and problem data shared by the element kernels.
template <class T>
struct AsmArgs {
  // mesh
  const double* X;          // n_verts x DIM
  const int* ev;            // n_elems x NV
  const int* nbr;           // n_elems x NFACE: neighbour element or -1
  const int* nbr_face;      // n_elems x NFACE: neighbour's local face
  const signed char* bc;    // n_elems x NFACE: 0 interior, 1 far field / inflow, 2 outflow
  // bases
  const T* Phi;             // N_u x ku
  const double* Psi;        // N_x x kx
  int ku, kx;
  // items: element ids and weights (elems == nullptr: item i is element i, weight 1)
  const int* elems;
  const double* rho;
  long n_items;
  // evaluation point (FP64) and parameters
  const double* w;
  const double* tau;
  const double* mu;
  // reference tables (FP64, packed: D | B | Lt | fw | qw | qxi)
  const double* tables;
  double gamma, kappa, eps;
  // output: per-CTA partial sums [H (k*k) | g (k) | J | nonphysical count]
  double* partial;
  // optional: a device flag; when non-zero the kernel returns at once (a finished solve)
  const int* skip;
  // T = float only: how H += rho A^T A is formed (0: FP32 FMA, 1: TF32 tensor cores,
  // 2: 3xTF32 tensor cores, i.e. hi/lo splits of each operand, about FP32 accuracy,
  // 3: BF16 tensor cores)
  int contraction;
  // form dH/dn at face points even without mesh columns (the snapshot alignment
  // applies dR/dx to full mesh directions)
  int need_hn;
  // FP32 straight-sided 2-D elements (may be null): per element 1 + kx groups of
  // four floats, the reference edges (x_1 - x_0, x_2 - x_0) = (e1x, e1y, e2x, e2y)
  // and the same differences of each mesh column of Psi (taken in FP64, rounded
  // once); the FP32 geometry is formed from them with no FP64 arithmetic
  const float4* geo32 = nullptr;
  // FP32 with BF16 contraction (may be null): instead of forming H in the element
  // pass, write the element's rows of sqrt(rho_e) A_e transposed in BF16 pairs,
  // At[m][item * n_u + i] (row stride at_ld values), for the tensor-core product
  // that follows the pass (syrk_tc.cu)
  uint32_t* at_out = nullptr;
  long at_ld = 0;
};

// H += rho A^T A on the tensor cores (warp-level mma.m16n8k8, TF32 inputs, FP32
// accumulation), upper triangle only. A is the warp's n_u x k row-major block in
// shared memory; rows are the contraction index. A tile covers 16 rows r (the
// columns of A read as A^T) by 8 columns b of H; only tiles that meet r <= b are
// formed. SPLIT: each operand is split as hi + lo (both TF32) and the product
// taken as hi*hi + hi*lo + lo*hi, which restores about FP32 accuracy.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int NU, bool SPLIT>
__device__ __forceinline__ void syrk_upper_tf32(const float* A, int k, int ka, float* acc, float rho, int lane) {
  const int g = lane >> 2, t = lane & 3;
  constexpr int KS = (NU + 7) / 8;
  const int mtiles = (k + 15) / 16, ntiles = (k + 7) / 8;
  auto ld = [&](int i, int col) { return (i < NU && col < k) ? A[i * ka + col] : 0.0f; };
  for (int mt = 0; mt < mtiles; ++mt) {
    const int r0 = mt * 16 + g, r1 = r0 + 8;
    for (int nt = 2 * mt; nt < ntiles; ++nt) {
      const int bc = nt * 8 + g;
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const int i0 = ks * 8 + t, i1 = i0 + 4;
        const float av[4] = {ld(i0, r0), ld(i0, r1), ld(i1, r0), ld(i1, r1)};
        const float bv[2] = {ld(i0, bc), ld(i1, bc)};
        uint32_t ah[4], bh[2];
#pragma unroll
        for (int j = 0; j < 4; ++j) ah[j] = to_tf32(av[j]);
#pragma unroll
        for (int j = 0; j < 2; ++j) bh[j] = to_tf32(bv[j]);
        if (SPLIT) {
          uint32_t al[4], bl[2];
#pragma unroll
          for (int j = 0; j < 4; ++j) al[j] = to_tf32(av[j] - __uint_as_float(ah[j]));
#pragma unroll
          for (int j = 0; j < 2; ++j) bl[j] = to_tf32(bv[j] - __uint_as_float(bh[j]));
          mma_tf32(c, al, bh);
          mma_tf32(c, ah, bl);
        }
        mma_tf32(c, ah, bh);
      }
      const int cb = nt * 8 + 2 * t;
      const int rr[4] = {r0, r0, r1, r1}, cc[4] = {cb, cb + 1, cb, cb + 1};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (rr[j] <= cc[j] && cc[j] < k) acc[acc_h(rr[j], cc[j], k)] += rho * c[j];
    }
  }
}

// The same upper-triangle product with BF16 operands (mma.m16n8k16, FP32
// accumulation): a 7-bit mantissa per operand, so H carries a relative error of
// a few 1e-3. Fragment layout as above with k = 16: each 32-bit register holds two
// consecutive contraction indices, the lower index in the lower half.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int NU>
__device__ __forceinline__ void syrk_upper_bf16(const float* A, int k, int ka, float* acc, float rho, int lane) {
  const int g = lane >> 2, t = lane & 3;
  constexpr int KS = (NU + 15) / 16;
  const int mtiles = (k + 15) / 16, ntiles = (k + 7) / 8;
  auto ld = [&](int i, int col) { return (i < NU && col < k) ? A[i * ka + col] : 0.0f; };
  for (int mt = 0; mt < mtiles; ++mt) {
    const int r0 = mt * 16 + g, r1 = r0 + 8;
    for (int nt = 2 * mt; nt < ntiles; ++nt) {
      const int bc = nt * 8 + g;
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const int i0 = ks * 16 + 2 * t, i1 = i0 + 8;
        const uint32_t av[4] = {pack_bf16x2(ld(i0, r0), ld(i0 + 1, r0)), pack_bf16x2(ld(i0, r1), ld(i0 + 1, r1)),
                                pack_bf16x2(ld(i1, r0), ld(i1 + 1, r0)), pack_bf16x2(ld(i1, r1), ld(i1 + 1, r1))};
        const uint32_t bv[2] = {pack_bf16x2(ld(i0, bc), ld(i0 + 1, bc)), pack_bf16x2(ld(i1, bc), ld(i1 + 1, bc))};
        mma_bf16(c, av, bv);
      }
      const int cb = nt * 8 + 2 * t;
      const int rr[4] = {r0, r0, r1, r1}, cc[4] = {cb, cb + 1, cb, cb + 1};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (rr[j] <= cc[j] && cc[j] < k) acc[acc_h(rr[j], cc[j], k)] += rho * c[j];
    }
  }
}

// The same BF16 upper-triangle product with its operands staged once per element:
// A (n_u x k FP32, row stride ka) is rounded to BF16 and transposed into T (k rows of
// kp = n_u rounded up to 16 entries, zero beyond n_u; rs bytes per row, 16 more than
// the data so that the eight rows of an ldmatrix phase fall on different banks),
// and each 16 x 16 (A^T) and 16 x 8 (A) fragment is one ldmatrix. Rows of a tile
// beyond k read row k - 1; their products land outside the triangle and are dropped.
// T takes rs * k bytes of shared memory the caller no longer needs (Phi_e).
__host__ __device__ constexpr int syrk_bf16_rs(int nu) { return ((nu + 15) / 16) * 32 + 16; }

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t r[2], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}

template <int NU>
__device__ __forceinline__ void syrk_upper_bf16_staged(const float* A, int k, int ka, unsigned char* Tb, float* acc,
                                                       float rho, int lane) {
  constexpr int KS = (NU + 15) / 16;  // 16-entry steps of the contraction index
  constexpr int rs = syrk_bf16_rs(NU);
  // transpose and round, one row m of T per lane: 16-byte groups of four BF16 pairs
  // (A[i][m], A[i + 1][m]), zero beyond n_u
  for (int m = lane; m < k; m += 32) {
#pragma unroll
    for (int grp = 0; grp < KS * 2; ++grp) {
      uint32_t w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i0 = grp * 8 + 2 * u, i1 = i0 + 1;
        const float lo = i0 < NU ? A[i0 * ka + m] : 0.0f, hi = i1 < NU ? A[i1 * ka + m] : 0.0f;
        w[u] = pack_bf16x2(lo, hi);
      }
      *reinterpret_cast<uint4*>(Tb + m * rs + grp * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  __syncwarp();
  const uint32_t tb = (uint32_t)__cvta_generic_to_shared(Tb);
  const int g = lane >> 2, t = lane & 3;
  const int mtiles = (k + 15) / 16, ntiles = (k + 7) / 8;
  // ldmatrix row addresses: x4 (A^T tile) lanes 8j..8j+7 give rows (j & 1) * 8 + r at
  // column (j >> 1) * 8; x2 (A tile) lanes 0..15 give rows r at column ((lane >> 3) & 1) * 8
  const int ra = ((lane >> 3) & 1) * 8 + (lane & 7), ca = (lane >> 4) * 8;
  const int rb = lane & 7, cb8 = ((lane >> 3) & 1) * 8;
  for (int mt = 0; mt < mtiles; ++mt) {
    const int r0 = mt * 16 + g, r1 = r0 + 8;
    const int rowa = min(mt * 16 + ra, k - 1);
    for (int nt = 2 * mt; nt < ntiles; ++nt) {
      const int rowb = min(nt * 8 + rb, k - 1);
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        uint32_t av[4], bv[2];
        ldsm_x4(av, tb + rowa * rs + (ks * 16 + ca) * 2);
        ldsm_x2(bv, tb + rowb * rs + (ks * 16 + cb8) * 2);
        mma_bf16(c, av, bv);
      }
      const int cb = nt * 8 + 2 * t;
      const int rr[4] = {r0, r0, r1, r1}, cc[4] = {cb, cb + 1, cb, cb + 1};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (rr[j] <= cc[j] && cc[j] < k) acc[acc_h(rr[j], cc[j], k)] += rho * c[j];
    }
  }
  __syncwarp();
}

template <class T, int PROB, int P>
struct Tabs {
  using Dd = Disc<PROB, P>;
  static constexpr int nD = Dd::DIM * Dd::NQ * Dd::NB, nB = Dd::NQ * Dd::NB, nL = Dd::NFQ * Dd::NTRACE,
                       nfw = Dd::NFQ, nqw = Dd::NQ, nqx = Dd::NQ;
  // curved elements: dN_j/dxi_c of the six geometry shape functions at the volume
  // points (NQ x 6 x 2), and dN_j/dt along each face at its points (NF x NFQ x 6)
  static constexpr int nGv = Dd::CURVED ? Dd::NQ * 12 : 0, nGt = Dd::CURVED ? Dd::NFACE * Dd::NFQ * 6 : 0;
  static constexpr int total = nD + nB + nL + nfw + nqw + nqx + nGv + nGt;
  // face coefficients fw[f] Lt[f][i] Lt[f][j] (NFQ x NT x NT), built beside the
  // staged tables (not part of the packed host tables)
  static constexpr int nC = Dd::NFQ * Dd::NTRACE * Dd::NTRACE;
  __host__ __device__ static constexpr size_t cf_offset() { return ((size_t)total * sizeof(T) + 15) / 16 * 16; }
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// FP64 elements whose volume Jacobian dR_e/dU_e (n_u x n_u) fits in 18 registers
// per lane form it explicitly in staged passes and multiply by Phi_e (fewer FP64
// operations, the bound of the FP64 kernels); larger ones (p = 3 Euler) take
// Jacobian-vector products per quadrature point. The FP32 kernels have their own
// forms (jac_state: rows in registers for p <= 2, per-column products otherwise).
__host__ __device__ constexpr bool kExplicitVolume(int nu, int word) { return word == 8 && nu * nu <= 576; }
// Entries of Jv per register pass (9 doubles per lane).
constexpr int kJvPass = 288;

// Four consecutive entries at a 16-byte aligned shared-memory address: one vector
// store in FP32 (a warp's scalar stores to per-point rows conflict on the banks;
// the vector form moves four words per bank pass), four stores in FP64.
template <class T>
__device__ __forceinline__ void st4(T* p, T a, T b, T c, T d) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  } else {
    p[0] = a;
    p[1] = b;
    p[2] = c;
    p[3] = d;
  }
}

// Row stride of the element's Jacobian columns A (n_u x k, row-major). FP32 elements
// with more rows than lanes (p = 3) pad each row by four floats: the tensor-core
// fragments read A down its columns, eight rows apart per lane group, and with
// k = 48 every such read hit one bank four times; k + 4 spreads them over the banks
// and keeps rows 16-byte aligned. Elsewhere the padding would cost occupancy.
__host__ __device__ constexpr int a_row_stride(int k, int nu, int word) { return (word == 4 && nu > 32) ? k + 4 : k; }

// Per-volume-point stride of the contravariant flux Jacobians Ahat_qr (the DIM M x M
// blocks of point q start at q * stride). FP32 Euler pads it by four floats: the
// lanes of step 4 each write their own point's 32 entries, and with a stride of 32
// words all of them hit the same bank (16-way conflicts); 36 words leaves at most
// two lanes per bank and keeps every row 16-byte aligned. FP64 keeps the dense
// stride (its shared memory is the tighter limit there).
__host__ __device__ constexpr int ah_stride(int m, int dim, int word) {
  return (word == 4 && m == 4) ? dim * m * m + 4 : dim * m * m;
}

// FP32 Euler state columns by rows of dR_e/dU_e in registers (jac_state_rows_f2):
// an even node count (packed pairs) and at most one row per lane (p <= 2); p = 3
// (40 rows) takes the per-column products, which measured faster there.
__host__ __device__ constexpr bool kStateRowsF32(int m, int nb) { return m == 4 && nb % 2 == 0 && m * nb <= 32; }

// Per-warp shared-memory layout. GRAD: the gradient pass, which for Euler forms no
// Jacobian columns, no face Jacobians and no volume flux Jacobians (the states U_q
// only), and accumulates only [g | J | count] (SLIM: those buffers shrink to what it uses).
// FUSED: the layout of the fused assembly kernels (assemble_kernel and
// assemble_batched_kernel); other kernels that carve the same buffers (inspection,
// per-element gradients, alignment) take the general layout.
template <class T, int PROB, int P, bool JAC, bool GRAD = false, bool FUSED = false>
struct WarpLayout {
  using Dd = Disc<PROB, P>;
  static constexpr int M = Dd::M, DIM = Dd::DIM, NQ = Dd::NQ, NU = Dd::NU, NUP = Dd::NUP, NXE = Dd::NXE,
                       NF = Dd::NFACE, NFQ = Dd::NFQ;
  static constexpr bool SLIM = GRAD && JAC && Dd::EULER;
  // the fused FP32 Euler Jacobian pass of p <= 2 forms the state columns by rows in
  // registers and stages only the mesh columns' sums in W
  static constexpr bool ROWS = FUSED && JAC && !GRAD && sizeof(T) == 4 && kStateRowsF32(Dd::M, Dd::NB);
  // elements a warp evaluates at once: two (one per half-warp, each with its own
  // copy of this layout) in the Euler gradient pass, else one
  static constexpr int PER_WARP = SLIM ? 2 : 1;
  // offset of g (the tail [g | J | count]) within the accumulators
  __host__ __device__ static int gacc_offset(int k) { return SLIM ? 0 : acc_tail(k); }
  size_t oxe, oPsie, odN, oPhie, oPoff, oUe, oUp, oFh, ofph, oAh, osq, oHf, oHp, oHm, oHn, oUi, oUo, oR, oA, odNt,
      oW, owq, otq, otqf, oacc, ocofq, ontq, bytes;
  __host__ __device__ WarpLayout(int ku, int kx) {
    const int k = ku + kx;
    size_t b = 0;
    auto put = [&](size_t n, size_t es) {
      size_t o = b;
      b = align16(b + n * es);
      return o;
    };
    oxe = put(NXE, 8);
    oPsie = put((size_t)NXE * (kx > 0 ? kx : 1), 8);
    odN = put(NXE + 2, 8);
    oPhie = put((size_t)NU * ku, sizeof(T));
    // neighbour trace rows are read from Phi in global memory (L1/L2): per face and
    // trace position, the offset of the row block in Phi (-1 on boundary faces)
    oPoff = put((size_t)NF * Dd::NTRACE, 8);
    oUe = put(NU, sizeof(T));
    oUp = put(NUP, sizeof(T));
    oFh = put(NQ * DIM * M, sizeof(T));
    ofph = put(NQ * DIM * M, sizeof(T));
    oAh = put(JAC ? (SLIM ? NQ * M : NQ * ah_stride(M, DIM, sizeof(T))) : 1, sizeof(T));
    osq = put(NQ, sizeof(T));
    oHf = put(NF * NFQ * M, sizeof(T));
    // curved elements: the cofactor at every volume point and the scaled normal at every face point
    ocofq = put(Dd::CURVED ? NQ * 4 : 1, sizeof(T));
    ontq = put(Dd::CURVED ? NF * NFQ * 2 : 1, sizeof(T));
    oHp = put(JAC && !SLIM ? NF * NFQ * M * M : 1, sizeof(T));
    oHm = put(JAC && !SLIM ? NF * NFQ * M * M : 1, sizeof(T));
    oHn = put(JAC && !SLIM ? NF * NFQ * M * 2 : 1, sizeof(T));
    oUi = put(NF * NFQ * M, sizeof(T));
    oUo = put(NF * NFQ * M, sizeof(T));
    oR = put(NU, sizeof(T));
    oA = put(JAC && !SLIM ? (size_t)NU * a_row_stride(k, NU, sizeof(T)) : 1, sizeof(T));
    odNt = put(kx + 1, sizeof(T));
    {
      // staging of the reduced-Jacobian passes: volume G (M ku) + F (DIM M ku), faces
      // dU (2 M ku) + dH (M ku), mesh directions E (NB M 4) + dcof (4 kx) + K (NF NT M 2)
      size_t w1 = (size_t)(DIM + 1) * M * ku, w2 = (size_t)3 * M * ku,
             w3 = (size_t)Dd::NB * M * 4 + 4 * kx + (size_t)NF * Dd::NTRACE * M * 2 + (size_t)NF * 2 * kx;
      size_t w = ROWS ? 0 : (w1 > w2 ? w1 : w2);
      if (w3 > w) w = w3;
      // curved mesh columns: dF per (volume point, column) and dH per (face point, column)
      if (Dd::CURVED) {
        const size_t wc = (size_t)NQ * (kx > 0 ? kx : 1) * 8 + (size_t)NF * NFQ * (kx > 0 ? kx : 1) * 4;
        if (wc > w) w = wc;
      }
      if (SLIM) w = 0;  // the gradient pass stages only the adjoint below
      if (!ROWS) {  // adjoint pass: t_q (NQ M), mu+ and mu- per face point (2 NF NFQ M), nu (2 NF NFQ),
         // eps per volume point (4 NQ), dU_e, dU_e' (NU + NU'), eps (4)
        const size_t wa = (size_t)NQ * M + (size_t)2 * NF * NFQ * M + (size_t)2 * NF * NFQ + (size_t)4 * NQ + NU +
                          NUP + 4;
        if (wa > w) w = wa;
      }
      if (kExplicitVolume(NU, sizeof(T)) && !SLIM) {  // T_q (RP M) and one pass of Jv rows (RP NU)
        const int np = (NU * NU + kJvPass - 1) / kJvPass, rp = NU / np;
        const size_t we = (size_t)rp * (M + NU);
        if (we > w) w = we;
      }
      oW = put(JAC ? w : 1, sizeof(T));
    }
    owq = put(ku > 0 ? ku : 1, sizeof(T));
    otq = put(kx > 0 ? kx : 1, 8);
    otqf = put(kx > 0 ? kx : 1, 4);  // the same tau in FP32 (FP32 geometry from the edge table)
    oacc = put(SLIM ? (size_t)k + 2 : (size_t)acc_count(k), sizeof(T));
    bytes = b;
  }
};

template <class T, int PROB, int P>
__host__ __device__ inline size_t cta_bytes(int ku, int kx) {
  return align16(Tabs<T, PROB, P>::total * sizeof(T)) + align16(Tabs<T, PROB, P>::nC * sizeof(T)) +
         align16((size_t)(ku > 0 ? ku : 1) * sizeof(T)) + align16((size_t)(kx > 0 ? kx : 1) * 8) +
         align16((size_t)(kx > 0 ? kx : 1) * 4);
}

// The upper-triangle pair table of the lane-owned contraction; the fused FP32
// kernels with k a multiple of 4 take 4 x 4 blocks (or tensor-core tiles) instead.
template <class T>
__host__ __device__ inline bool needs_pair_table(bool jac, bool grad, bool fused, int k) {
  return jac && !grad && !(fused && sizeof(T) == 4 && k % 4 == 0);
}

template <class T, int PROB, int P, bool JAC, bool GRAD = false, bool FUSED = false>
__host__ __device__ inline size_t assemble_smem_bytes(int ku, int kx, int warps) {
  const int k = ku + kx;
  using Lay = WarpLayout<T, PROB, P, JAC, GRAD, FUSED>;
  return cta_bytes<T, PROB, P>(ku, kx) + (size_t)warps * Lay::PER_WARP * Lay(ku, kx).bytes +
         (needs_pair_table<T>(JAC, GRAD, FUSED, k) ? align16((size_t)k * (k + 1)) : 0);
}

// Pointwise stage and residual for one element whose U_e, U_e', x_e are staged.
// Leaves Fh/fph/Ah (volume), Hf/Hp/Hm/Hn (faces), R (residual), and returns the
// non-physical flag (warp-uniform).
// Division of small non-negative ints by a divisor fixed for the whole kernel:
// q = floor(e * m / 2^32) with m = ceil(2^32 / d) is exact while e * d < 2^32
// (here e < 2^16, d <= 64), one multiply-high instead of a division sequence.
struct FastDiv {
  uint32_t d, m;
  __device__ void init(int dv) {
    d = (uint32_t)dv;
    m = (dv > 1) ? (0xFFFFFFFFu / d + 1u) : 0u;
  }
  __device__ __forceinline__ int div(int e) const { return d > 1 ? (int)__umulhi((uint32_t)e, m) : e; }
};

template <class T, int PROB, int P, bool JAC>
struct ElemCore {
  using Dd = Disc<PROB, P>;
  static constexpr int M = Dd::M, DIM = Dd::DIM, NB = Dd::NB, NQ = Dd::NQ, NU = Dd::NU, NUP = Dd::NUP,
                       NXE = Dd::NXE, NF = Dd::NFACE, NFQ = Dd::NFQ, NT = Dd::NTRACE;
  static constexpr int AQ = ah_stride(M, DIM, sizeof(T));  // point stride of Ah
  // shared tables (GdV, GtF: curved geometry shape-function derivatives)
  const T *D, *B, *Lt, *fw, *qw, *qxi, *GdV, *GtF;
  const T* Cf;  // fw[f] Lt[f][i] Lt[f][j]: the face blocks of dR_e/dU_e
  // warp buffers
  double *xe, *Psie, *dN;
  T *Phie, *Ue, *Up, *Fh, *fph, *Ah, *sq, *Hf, *Hp, *Hm, *Hn, *Ui, *Uo, *R, *A, *dNt, *W, *acc;
  T* gacc;  // [g | J | count] within acc
  T *cofq, *ntq;  // curved: cofactor per volume point (4), scaled normal per face point (2)
  // geometry (registers, identical on all lanes)
  T cof[4];      // cof[d*2 + r] = (g J^{-T})[d][r]
  T detJ;
  T nt[3][2];    // scaled face normals (2-D)
  bool g32;      // this element's geometry came from the FP32 edge table (Psie holds its rows)
  double x0d, x1d;  // 1-D end points
  const T* PhiG;     // Phi in global memory (neighbour trace rows)
  long long* poff;   // per face and trace position: row-block offset in PhiG, -1 on boundary faces
  FastDiv dku, dkx;  // division by k_u and k_x in the lane loops
  int ka;            // row stride of A (a_row_stride)

  template <bool GRAD = false, bool FUSED = false>
  __device__ void carve(unsigned char* base, int ku, int kx) {
    WarpLayout<T, PROB, P, JAC, GRAD, FUSED> L(ku, kx);
    g32 = false;
    dku.init(ku > 0 ? ku : 1);
    dkx.init(kx > 0 ? kx : 1);
    xe = (double*)(base + L.oxe);
    Psie = (double*)(base + L.oPsie);
    dN = (double*)(base + L.odN);
    Phie = (T*)(base + L.oPhie);
    poff = (long long*)(base + L.oPoff);
    Ue = (T*)(base + L.oUe);
    Up = (T*)(base + L.oUp);
    Fh = (T*)(base + L.oFh);
    fph = (T*)(base + L.ofph);
    Ah = (T*)(base + L.oAh);
    sq = (T*)(base + L.osq);
    Hf = (T*)(base + L.oHf);
    Hp = (T*)(base + L.oHp);
    Hm = (T*)(base + L.oHm);
    Hn = (T*)(base + L.oHn);
    Ui = (T*)(base + L.oUi);
    Uo = (T*)(base + L.oUo);
    W = (T*)(base + L.oW);
    R = (T*)(base + L.oR);
    A = (T*)(base + L.oA);
    ka = a_row_stride(ku + kx, NU, sizeof(T));
    dNt = (T*)(base + L.odNt);
    acc = (T*)(base + L.oacc);
    gacc = acc + L.gacc_offset(ku + kx);
    cofq = (T*)(base + L.ocofq);
    ntq = (T*)(base + L.ontq);
  }

  // Cofactor g G^{-T} (entry [d][r] at d * 2 + r) at volume point q, and the scaled
  // normal of face k at face point pt: per point for curved elements, else the
  // element's constants.
  __device__ __forceinline__ T cofv(int q, int i) const {
    if constexpr (Dd::CURVED) return cofq[q * 4 + i];
    else return cof[i];
  }
  __device__ __forceinline__ T ntv(int pt, int k, int d) const {
    if constexpr (Dd::CURVED) return ntq[pt * 2 + d];
    else return k == 0 ? nt[0][d] : (k == 1 ? nt[1][d] : nt[2][d]);  // selects: k is lane-dependent
  }

  // Curved element geometry (Eq. p2r-flux with the six-node quadratic map
  // x(xi) = sum_j N_j(xi) x_j): at every volume point the cofactor of J = dx/dxi,
  // at every face point the scaled normal, the tangent dx/dt of the face turned by
  // -90 degrees (counter-clockwise elements: outward). Lanes split the points.
  // Returns false for the lane's group if the map folds (det J <= 0 at a point).
  __device__ bool geometry_curved(int lane, int step) {
    bool ok = true;
    for (int t = lane; t < NQ + NF * NFQ; t += step) {
      if (t < NQ) {
        const T* gd = &GdV[t * 12];
        double J0 = 0.0, J1 = 0.0, J2 = 0.0, J3 = 0.0;  // J[r * 2 + c] = d x_r / d xi_c
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          J0 += xe[2 * j] * (double)gd[2 * j];
          J1 += xe[2 * j] * (double)gd[2 * j + 1];
          J2 += xe[2 * j + 1] * (double)gd[2 * j];
          J3 += xe[2 * j + 1] * (double)gd[2 * j + 1];
        }
        cofq[t * 4 + 0] = (T)J3;
        cofq[t * 4 + 1] = (T)(-J2);
        cofq[t * 4 + 2] = (T)(-J1);
        cofq[t * 4 + 3] = (T)J0;
        if (!(J0 * J3 - J1 * J2 > 0.0)) ok = false;
      } else {
        const int pt = t - NQ;
        const T* tw = &GtF[pt * 6];
        double tx = 0.0, ty = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          tx += xe[2 * j] * (double)tw[j];
          ty += xe[2 * j + 1] * (double)tw[j];
        }
        ntq[pt * 2 + 0] = (T)ty;
        ntq[pt * 2 + 1] = (T)(-tx);
      }
    }
    return !group_any(!ok, step);
  }

  // Geometry from xe (FP64). Returns false if the element is inverted.
  __device__ bool geometry() {
    if (DIM == 1) {
      x0d = xe[0];
      x1d = xe[1];
      double det = x1d - x0d;
      detJ = (T)det;
      cof[0] = T(1);
      return det > 0.0;
    } else {
      double j00 = xe[2] - xe[0], j01 = xe[4] - xe[0];
      double j10 = xe[3] - xe[1], j11 = xe[5] - xe[1];
      double det = j00 * j11 - j01 * j10;
      detJ = (T)det;
      cof[0] = (T)j11;
      cof[1] = (T)(-j10);
      cof[2] = (T)(-j01);
      cof[3] = (T)j00;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        int k1 = (k + 1) % 3;
        nt[k][0] = (T)(xe[2 * k1 + 1] - xe[2 * k + 1]);
        nt[k][1] = (T)(-(xe[2 * k1] - xe[2 * k]));
      }
      return det > 0.0;
    }
  }

  // Straight-sided 2-D geometry in FP32 from the element's rows of the edge table
  // (staged in Psie: the reference edges, then one row per mesh column): the current
  // edges x_1 - x_0 = (j00, j10) and x_2 - x_0 = (j01, j11) are the reference ones plus
  // sum_c tau_c times the column's edge differences, and the cofactor, determinant
  // and scaled normals follow as in geometry(). Returns false if the element is inverted.
  __device__ bool geometry32(const float* tauF, int kx) {
    const float4* g = reinterpret_cast<const float4*>(Psie);
    float4 j = g[0];  // (j00, j10, j01, j11)
    for (int c = 0; c < kx; ++c) {
      const float4 d = g[1 + c];
      const float t = tauF[c];
      j.x = fmaf(d.x, t, j.x);
      j.y = fmaf(d.y, t, j.y);
      j.z = fmaf(d.z, t, j.z);
      j.w = fmaf(d.w, t, j.w);
    }
    const float det = j.x * j.w - j.z * j.y;
    detJ = (T)det;
    cof[0] = (T)j.w;
    cof[1] = (T)(-j.y);
    cof[2] = (T)(-j.z);
    cof[3] = (T)j.x;
    // face k runs from vertex k to vertex k + 1: x_1 - x_0, x_2 - x_1, x_0 - x_2
    nt[0][0] = (T)j.y;
    nt[0][1] = (T)(-j.x);
    nt[1][0] = (T)(j.w - j.y);
    nt[1][1] = (T)(-(j.z - j.x));
    nt[2][0] = (T)(-j.w);
    nt[2][1] = (T)j.z;
    return det > 0.0f;
  }

  // Step 4: pointwise quantities. bcs: per-face boundary type.
  // face_jac = false: face fluxes only (the FP64 gradient pass takes their adjoint by
  // reverse mode instead of forming dH/dU+ and dH/dU-); vol_jac = false (Euler): the
  // volume flux Jacobians are not formed either, and the states U_q are kept in
  // Ah[q][0..3] for the adjoint's vector-Jacobian products.
  __device__ bool pointwise(int lane, const signed char* bcs, const double* mu, double gamma, bool need_hn,
                            bool face_jac = true, bool vol_jac = true, int step = 32) {
    const bool fj = JAC && face_jac;
    bool bad = false;
    const T g1 = (T)(gamma - 1.0);
    // volume points
    for (int q = lane; q < NQ; q += step) {
      T U[4];
#pragma unroll
      for (int a = 0; a < M; ++a) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < NB; ++j) s += B[q * NB + j] * Ue[j * M + a];
        U[a] = s;
      }
      if (Dd::EULER) {
        T fx[4], fy[4], Pq;
        euler_flux(U, g1, fx, fy, Pq);
        if (!(U[0] > T(0)) || !(Pq > T(0))) bad = true;
        st4(&fph[(q * 2 + 0) * 4], fx[0], fx[1], fx[2], fx[3]);
        st4(&fph[(q * 2 + 1) * 4], fy[0], fy[1], fy[2], fy[3]);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          T fr[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) fr[a] = fx[a] * cofv(q, 0 * 2 + r) + fy[a] * cofv(q, 1 * 2 + r);
          st4(&Fh[(q * 2 + r) * 4], fr[0], fr[1], fr[2], fr[3]);
        }
        if (JAC && vol_jac) {
          T Ax[16], Ay[16];
          euler_flux_jac(U, g1, Ax, Ay);
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              T v[4];
#pragma unroll
              for (int b = 0; b < 4; ++b) v[b] = Ax[a * 4 + b] * cofv(q, r) + Ay[a * 4 + b] * cofv(q, 2 + r);
              st4(&Ah[q * AQ + r * 16 + a * 4], v[0], v[1], v[2], v[3]);
            }
        } else if (JAC) {
          st4(&Ah[q * 4], U[0], U[1], U[2], U[3]);
        }
      } else {
        T f = T(0.5) * U[0] * U[0];
        Fh[q] = f;
        fph[q] = f;
        if (JAC) Ah[q] = U[0];
        // source s(x) = 0.5 exp(mu x) at the mapped point
        double xq = x0d + (double)qxi[q] * (x1d - x0d);
        sq[q] = (T)(0.5 * exp(mu[0] * xq));
      }
    }
    // face points: task t -> (group, face point); group 0: H and dH/dU+, group 1: dH/dU-
    const int npts = NF * NFQ;
    const int ngroups = (Dd::EULER && fj) ? 2 : 1;
    // dH/dn inside the task loop when both groups run in one trip of a whole warp
    // (every Euler degree here: at most 2 x 15 tasks); otherwise in a pass of its own
    const bool hn_fused = Dd::EULER && fj && need_hn && step == 32 && 2 * npts <= 32;
    const unsigned hn_mask = 2 * npts >= 32 ? 0xffffffffu : ((1u << (2 * npts)) - 1u);
    const bool hn_here = hn_fused && lane < 2 * npts;
    for (int t = lane; t < npts * ngroups; t += step) {
      const int grp = t / npts, pt = t % npts;
      const int k = pt / NFQ, f = pt % NFQ;
      T Uin[4], Uout[4];
#pragma unroll
      for (int a = 0; a < M; ++a) {
        T s = T(0), so = T(0);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          // face_node depends on the runtime face k: read Ue through the small switch
          int node = (k == 0) ? Dd::face_node(0, j) : ((k == 1) ? Dd::face_node(1, j) : Dd::face_node(2, j));
          s += Lt[f * NT + j] * Ue[node * M + a];
          so += Lt[f * NT + j] * Up[(k * NT + j) * M + a];
        }
        Uin[a] = s;
        Uout[a] = so;
      }
      const signed char bt = bcs[k];
      if (Dd::EULER) {
        if (bt == 1) {
          double Uf[4];
          euler_farfield(gamma, mu[0], mu[1], Uf);
#pragma unroll
          for (int a = 0; a < 4; ++a) Uout[a] = (T)Uf[a];
        }
        T* hf = &Hf[pt * 4];
        if (grp == 0) {
          // P > 0 with rho > 0 <=> rho E rho - |rho v|^2 / 2 > 0 (no division)
          const T Pi = Uin[3] * Uin[0] - T(0.5) * (Uin[1] * Uin[1] + Uin[2] * Uin[2]);
          const T Po = Uout[3] * Uout[0] - T(0.5) * (Uout[1] * Uout[1] + Uout[2] * Uout[2]);
          if (!(Uin[0] > T(0)) || !(Pi > T(0)) || !(Uout[0] > T(0)) || !(Po > T(0))) bad = true;
          st4(&Ui[pt * 4], Uin[0], Uin[1], Uin[2], Uin[3]);
          st4(&Uo[pt * 4], Uout[0], Uout[1], Uout[2], Uout[3]);
        }
        if (!fj) {
          T n2[2] = {ntv(pt, k, 0), ntv(pt, k, 1)};
          T H[4];
          euler_roe<T, T, T>(Uin, Uout, n2, g1, H);
          st4(hf, H[0], H[1], H[2], H[3]);
        } else {
          // group 0: dH/dU+ with U+ as the dual side; group 1: dH/dU- from the same
          // code on the swapped states and reversed normal (H(U+, U-; n) = -H(U-, U+; -n)),
          // so both groups run in lockstep and the other side stays plain
          const bool sw = grp != 0;
          const T sg = sw ? T(-1) : T(1);
          Dual<T, 4> dA[4], H[4];
          T B[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            dA[a] = dconst<T, 4>(sw ? Uout[a] : Uin[a]);
            dA[a].d[a] = T(1);
            B[a] = sw ? Uin[a] : Uout[a];
          }
          const T n2[2] = {sg * ntv(pt, k, 0), sg * ntv(pt, k, 1)};
          euler_roe<Dual<T, 4>, T, T>(dA, B, n2, g1, H);
          T* dst = sw ? &Hm[pt * 16] : &Hp[pt * 16];
          if (!sw) st4(hf, H[0].v, H[1].v, H[2].v, H[3].v);
#pragma unroll
          for (int a = 0; a < 4; ++a) st4(&dst[a * 4], sg * H[a].d[0], sg * H[a].d[1], sg * H[a].d[2], sg * H[a].d[3]);
          if (hn_here) {
            // dH/dn from the identities below, formed where the Jacobians are in
            // registers: each group applies its own Jacobian to G(its state) (see the
            // separate pass), and group 1 hands its part to group 0 by a shuffle
            const T* us = sw ? Uout : Uin;
            T part[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) part[a] = (sg * H[a].d[1]) * (-us[2]) + (sg * H[a].d[2]) * us[1];
            T other[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) other[a] = __shfl_down_sync(hn_mask, part[a], npts);
            if (!sw) {
              const T nx = ntv(pt, k, 0), ny = ntv(pt, k, 1);
              const T inv = T(1) / (nx * nx + ny * ny);
              const T Gh[4] = {T(0), -H[2].v, H[1].v, T(0)};
#pragma unroll
              for (int a = 0; a < 4; ++a) {
                const T K = Gh[a] - part[a] - other[a];
                Hn[pt * 8 + a * 2 + 0] = (H[a].v * nx - K * ny) * inv;
                Hn[pt * 8 + a * 2 + 1] = (H[a].v * ny + K * nx) * inv;
              }
            }
          }
        }
      } else {
        // Burgers: inflow u- = 1 on the face with normal -x, outflow u- = u+
        T n = (k == 0) ? T(-1) : T(1);
        if (bt == 1) Uout[0] = T(1);
        if (bt == 2) Uout[0] = Uin[0];
        T H, Hi, Ho;
        burgers_roe(Uin[0], Uout[0], n, H, Hi, Ho);
        Hf[pt] = H;
        if (JAC) {
          Hp[pt] = Hi;
          Hm[pt] = Ho;
        }
      }
    }
    if (Dd::EULER && fj && need_hn && !hn_fused) {
      __syncwarp();
      // dH/dn from two identities of the Roe flux: homogeneity, dH/dn . n = H, and
      // rotational invariance, dH/dn . (J n) = G(H) - dH/dU+ G(U+) - dH/dU- G(U-),
      // with J the 90-degree rotation and G(V) = (0, -V_2, V_1, 0) its action on a state.
      for (int pt = lane; pt < npts; pt += step) {
        const int k = pt / NFQ;
        const T nx = ntv(pt, k, 0), ny = ntv(pt, k, 1);
        const T inv = T(1) / (nx * nx + ny * ny);
        const T* h = &Hf[pt * 4];
        const T* hp = &Hp[pt * 16];
        const T* hm = &Hm[pt * 16];
        const T* ui = &Ui[pt * 4];
        const T* uo = &Uo[pt * 4];
        T Gh[4] = {T(0), -h[2], h[1], T(0)};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          // K = G(H) - Hp G(Ui) - Hm G(Uo); G(V) has entries 1 -> -V2, 2 -> V1
          T K = Gh[a] - (hp[a * 4 + 1] * (-ui[2]) + hp[a * 4 + 2] * ui[1]) -
                (hm[a * 4 + 1] * (-uo[2]) + hm[a * 4 + 2] * uo[1]);
          // [Hn n, Hn Jn] = [H, K]  with  [n, Jn] = [[nx, -ny], [ny, nx]]
          Hn[pt * 8 + a * 2 + 0] = (h[a] * nx - K * ny) * inv;
          Hn[pt * 8 + a * 2 + 1] = (h[a] * ny + K * nx) * inv;
        }
      }
    }
    return group_any(bad, step);
  }

  // Adjoint of steps 4-5 (the transposed element Jacobian applied to R_e):
  // dUe = (dR_e/dU_e)^T R_e (n_u values) and dUp = (dR_e/dU_e')^T R_e (n_u'), from the
  // pointwise flux Jacobians of step 4. Volume: dR[i][a] = -sum_q sum_r D_r[q][i]
  // (Ahat_qr dU_q)[a] with dU_q = B_q dU_e, so the adjoint is dUe[j][b] -= sum_q B_q[j]
  // t_q[b], t_q = sum_r Ahat_qr^T (D_r[q]^T R). Faces: dR[node][a] += fw Lt (Hp dU+ +
  // Hm dU-)[a]; with lam_pt = sum_j fw Lt[j] R[node_j] the adjoint lifts Hp^T lam onto
  // the interior trace nodes and Hm^T lam onto the neighbour's (or, on outflow faces,
  // where U- = U+, onto the interior ones too). dUe and dUp live in W after the staging.
  __device__ void adj_state(int lane, const signed char* bcs, T*& dUe, T*& dUp) {
    constexpr int NPT = NF * NFQ;
    T* tq = W;                  // [NQ][M]
    T* mp = W + NQ * M;         // [NPT][M]: Hp^T lam
    T* mm = mp + NPT * M;       // [NPT][M]: Hm^T lam
    dUe = mm + NPT * M;         // [NU]
    dUp = dUe + NU;             // [NUP]
    for (int t = lane; t < NQ + NPT; t += 32) {
      if (t < NQ) {
        const int q = t;
        T sr[DIM][M];
#pragma unroll
        for (int r = 0; r < DIM; ++r)
#pragma unroll
          for (int a = 0; a < M; ++a) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < NB; ++i) v += D[(r * NQ + q) * NB + i] * R[i * M + a];
            sr[r][a] = v;
          }
#pragma unroll
        for (int b = 0; b < M; ++b) {
          T v = T(0);
#pragma unroll
          for (int r = 0; r < DIM; ++r)
#pragma unroll
            for (int a = 0; a < M; ++a) v += Ah[q * AQ + (r * M + a) * M + b] * sr[r][a];
          tq[q * M + b] = v;
        }
      } else {
        const int pt = t - NQ, kf = pt / NFQ, f = pt - kf * NFQ;
        T lam[M];
#pragma unroll
        for (int a = 0; a < M; ++a) {
          T v = T(0);
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            const int node = (kf == 0) ? Dd::face_node(0, j) : ((kf == 1) ? Dd::face_node(1, j) : Dd::face_node(2, j));
            v += Lt[f * NT + j] * R[node * M + a];
          }
          lam[a] = fw[f] * v;
        }
#pragma unroll
        for (int b = 0; b < M; ++b) {
          T vp = T(0), vm = T(0);
#pragma unroll
          for (int a = 0; a < M; ++a) {
            vp += Hp[(pt * M + a) * M + b] * lam[a];
            vm += Hm[(pt * M + a) * M + b] * lam[a];
          }
          mp[pt * M + b] = vp;
          mm[pt * M + b] = vm;
        }
      }
    }
    __syncwarp();
    for (int e = lane; e < NU + NUP; e += 32) {
      T v = T(0);
      if (e < NU) {
        const int j = e / M, b = e - j * M;
#pragma unroll
        for (int q = 0; q < NQ; ++q) v -= B[q * NB + j] * tq[q * M + b];
#pragma unroll
        for (int kf = 0; kf < NF; ++kf) {
          const int jj = face_pos(kf, j);
          if (jj < 0) continue;
          const bool outflow = bcs[kf] == 2;
#pragma unroll
          for (int f = 0; f < NFQ; ++f) {
            const int pt = kf * NFQ + f;
            v += Lt[f * NT + jj] * (mp[pt * M + b] + (outflow ? mm[pt * M + b] : T(0)));
          }
        }
        dUe[e] = v;
      } else {
        const int i = e - NU, kj = i / M, b = i - kj * M, kf = kj / NT, jj = kj - kf * NT;
        if (bcs[kf] == 0) {
#pragma unroll
          for (int f = 0; f < NFQ; ++f) v += Lt[f * NT + jj] * mm[(kf * NFQ + f) * M + b];
        }
        dUp[i] = v;
      }
    }
    __syncwarp();
  }

  // The adjoint for Euler elements with the face Jacobians left out of step 4: at
  // each face point one forward and one reverse sweep of the Roe flux give
  // mup = Hp^T lam and mum = Hm^T lam directly, and with them the normal derivative
  // lam^T dH/dn from the homogeneity and rotation identities; the volume part is as in
  // adj_state and also gives eps[r][d] = sum_q sum_a (D_r[q]^T R)_a f_d(U_q)_a, the
  // volume term of R_e^T dR_e/dx_e. Outputs (in W): dUe, dUp, eps (4), nu (n_face n_fq x 2).
  __device__ void adj_state_vjp(int lane, const signed char* bcs, double gamma, T*& dUe, T*& dUp, T*& eps,
                                T*& nu, int step = 32, T** eq_out = nullptr) {
    constexpr int NPT = NF * NFQ;
    const T g1 = (T)(gamma - 1.0);
    T* tq = W;                  // [NQ][M]
    T* mp = W + NQ * M;         // [NPT][M]
    T* mm = mp + NPT * M;       // [NPT][M]
    nu = mm + NPT * M;          // [NPT][2]
    T* eq = nu + NPT * 2;       // [NQ][4]
    if (eq_out) *eq_out = eq;
    dUe = eq + NQ * 4;          // [NU]
    dUp = dUe + NU;             // [NUP]
    eps = dUp + NUP;            // [4]
    for (int t = lane; t < NQ + NPT; t += step) {
      if (t < NQ) {
        const int q = t;
        T sr[DIM][M];
#pragma unroll
        for (int r = 0; r < DIM; ++r)
#pragma unroll
          for (int a = 0; a < M; ++a) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < NB; ++i) v += D[(r * NQ + q) * NB + i] * R[i * M + a];
            sr[r][a] = v;
          }
        // t_q = sum_r Ahat_qr^T s_r with Ahat_qr = Ax cof[r] + Ay cof[2 + r]: the transposed
        // flux Jacobians at U_q (kept in Ah[q][0..3] by step 4) applied to
        // v_x = sum_r cof[r] s_r and v_y = sum_r cof[2 + r] s_r
        T vx[4], vy[4], Uq[4], tb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          vx[a] = cofv(q, 0) * sr[0][a] + cofv(q, 1) * sr[1][a];
          vy[a] = cofv(q, 2) * sr[0][a] + cofv(q, 3) * sr[1][a];
          Uq[a] = Ah[q * 4 + a];
        }
        euler_flux_vjp(Uq, g1, vx, vy, tb);
#pragma unroll
        for (int b = 0; b < 4; ++b) tq[q * M + b] = tb[b];
#pragma unroll
        for (int r = 0; r < DIM; ++r)
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            T v = T(0);
#pragma unroll
            for (int a = 0; a < M; ++a) v += sr[r][a] * fph[(q * DIM + d) * M + a];
            eq[q * 4 + r * 2 + d] = v;
          }
      } else {
        const int pt = t - NQ, kf = pt / NFQ, f = pt - kf * NFQ;
        T lam[4], Uin[4], Uout[4], Hv[4], up[4], um[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T v = T(0);
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            const int node = (kf == 0) ? Dd::face_node(0, j) : ((kf == 1) ? Dd::face_node(1, j) : Dd::face_node(2, j));
            v += Lt[f * NT + j] * R[node * M + a];
          }
          lam[a] = fw[f] * v;
          Uin[a] = Ui[pt * 4 + a];
          Uout[a] = Uo[pt * 4 + a];
        }
        const T n2[2] = {ntv(pt, kf, 0), ntv(pt, kf, 1)};
        euler_roe_vjp<T>(Uin, Uout, n2, g1, lam, Hv, up, um);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          mp[pt * 4 + b] = up[b];
          mm[pt * 4 + b] = um[b];
        }
        // lam^T Hn from [Hn n, Hn Jn] = [H, G(H) - Hp G(U+) - Hm G(U-)], G(V) = (0, -V_2, V_1, 0)
        const T lh = lam[0] * Hv[0] + lam[1] * Hv[1] + lam[2] * Hv[2] + lam[3] * Hv[3];
        const T lk = (-lam[1] * Hv[2] + lam[2] * Hv[1]) - (-up[1] * Uin[2] + up[2] * Uin[1]) -
                     (-um[1] * Uout[2] + um[2] * Uout[1]);
        const T inv = T(1) / (n2[0] * n2[0] + n2[1] * n2[1]);
        nu[pt * 2 + 0] = (lh * n2[0] - lk * n2[1]) * inv;
        nu[pt * 2 + 1] = (lh * n2[1] + lk * n2[0]) * inv;
      }
    }
    __syncwarp();
    for (int e = lane; e < NU + NUP + 4; e += step) {
      T v = T(0);
      if (e < NU) {
        const int j = e / M, b = e - j * M;
#pragma unroll
        for (int q = 0; q < NQ; ++q) v -= B[q * NB + j] * tq[q * M + b];
#pragma unroll
        for (int kf = 0; kf < NF; ++kf) {
          const int jj = face_pos(kf, j);
          if (jj < 0) continue;
          const bool outflow = bcs[kf] == 2;
#pragma unroll
          for (int f = 0; f < NFQ; ++f) {
            const int pt = kf * NFQ + f;
            v += Lt[f * NT + jj] * (mp[pt * M + b] + (outflow ? mm[pt * M + b] : T(0)));
          }
        }
        dUe[e] = v;
      } else if (e < NU + NUP) {
        const int i = e - NU, kj = i / M, b = i - kj * M, kf = kj / NT, jj = kj - kf * NT;
        if (bcs[kf] == 0) {
#pragma unroll
          for (int f = 0; f < NFQ; ++f) v += Lt[f * NT + jj] * mm[(kf * NFQ + f) * M + b];
        }
        dUp[i] = v;
      } else {
        const int rd = e - NU - NUP;
#pragma unroll
        for (int q = 0; q < NQ; ++q) v += eq[q * 4 + rd];
        eps[rd] = v;
      }
    }
    __syncwarp();
  }

  // Step 5: residual entries.
  __device__ bool residual(int lane, int step = 32) {
    bool bad = false;
    for (int ia = lane; ia < NU; ia += step) {
      const int i = ia / M, a = ia % M;
      T s = T(0);
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int r = 0; r < DIM; ++r) s -= D[(r * NQ + q) * NB + i] * Fh[(q * DIM + r) * M + a];
      if (PROB == PROB_BURGERS) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) s -= qw[q] * B[q * NB + i] * sq[q] * detJ;
      }
#pragma unroll
      for (int k = 0; k < NF; ++k)
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          if (Dd::face_node(k, j) != i) continue;
#pragma unroll
          for (int f = 0; f < NFQ; ++f) s += fw[f] * Lt[f * NT + j] * Hf[(k * NFQ + f) * M + a];
        }
      R[ia] = s;
      if (!isfinite(s)) bad = true;
    }
    return group_any(bad, step);
  }

  // Step 6a: derivative of R_e along a state direction (dUe: n_u values, dUp: n_u'
  // values, read through accessors), accumulated into dR.
  template <class FE, class FP>
  __device__ void jvp_state(FE dUe, FP dUp, const signed char* bcs, T dR[NU]) {
#pragma unroll
    for (int i = 0; i < NU; ++i) dR[i] = T(0);
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      T du[M];
#pragma unroll
      for (int b = 0; b < M; ++b) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < NB; ++j) s += B[q * NB + j] * dUe(j * M + b);
        du[b] = s;
      }
#pragma unroll
      for (int r = 0; r < DIM; ++r)
#pragma unroll
        for (int a = 0; a < M; ++a) {
          T dF = T(0);
#pragma unroll
          for (int b = 0; b < M; ++b) dF += Ah[q * AQ + (r * M + a) * M + b] * du[b];
#pragma unroll
          for (int i = 0; i < NB; ++i) dR[i * M + a] -= D[(r * NQ + q) * NB + i] * dF;
        }
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const signed char bt = bcs[k];
      // the face points stay a rolled loop: unrolled, the three faces' copies of
      // this body made the FP32 kernels stall on instruction fetch (0.290 ->
      // 0.264 ms at p = 2, 4.40 -> 3.78 ms at p = 3 rolled)
#pragma unroll 1
      for (int f = 0; f < NFQ; ++f) {
        T dui[M], duo[M];
#pragma unroll
        for (int b = 0; b < M; ++b) {
          T s = T(0), so = T(0);
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            s += Lt[f * NT + j] * dUe(Dd::face_node(k, j) * M + b);
            so += Lt[f * NT + j] * dUp((k * NT + j) * M + b);
          }
          dui[b] = s;
          duo[b] = (bt == 0) ? so : ((bt == 2) ? s : T(0));
        }
        const int pt = k * NFQ + f;
#pragma unroll
        for (int a = 0; a < M; ++a) {
          T dH = T(0);
#pragma unroll
          for (int b = 0; b < M; ++b) dH += Hp[(pt * M + a) * M + b] * dui[b] + Hm[(pt * M + a) * M + b] * duo[b];
#pragma unroll
          for (int j = 0; j < NT; ++j) dR[Dd::face_node(k, j) * M + a] += fw[f] * Lt[f * NT + j] * dH;
        }
      }
    }
  }

  // The FP32 Euler form of jvp_state (n_b even: p = 2, 3) on packed FP32 pairs: each
  // __ffma2_rn is two fused multiply-adds in one instruction, the operand pairs read
  // as 8-byte words. The interpolation and the flux-Jacobian products pair
  // consecutive table entries (nodes, state components) and add the two halves at
  // the end; the volume test pairs consecutive nodes i, 2h and 2h + 1, of dR. Same
  // arithmetic as jvp_state up to the order of the FP32 sums.
  template <class FE, class FP>
  __device__ void jvp_state_f2(FE dUe, FP dUp, const signed char* bcs, float dRo[NU]) {
    static_assert(M == 4 && NB % 2 == 0, "packed pairs need four variables and an even node count");
    constexpr int NB2 = NB / 2;
    auto ld2 = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
    float2 dR2[NB2][M];  // (dR[2h][a], dR[2h + 1][a])
#pragma unroll
    for (int h = 0; h < NB2; ++h)
#pragma unroll
      for (int a = 0; a < M; ++a) dR2[h][a] = make_float2(0.0f, 0.0f);
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      float du[M];
#pragma unroll
      for (int b = 0; b < M; ++b) {
        float2 s = __fmul2_rn(ld2(&B[q * NB]), make_float2(dUe(b), dUe(M + b)));
#pragma unroll
        for (int h = 1; h < NB2; ++h)
          s = __ffma2_rn(ld2(&B[q * NB + 2 * h]), make_float2(dUe(2 * h * M + b), dUe((2 * h + 1) * M + b)), s);
        du[b] = s.x + s.y;
      }
      const float2 du01 = make_float2(du[0], du[1]), du23 = make_float2(du[2], du[3]);
#pragma unroll
      for (int r = 0; r < DIM; ++r) {
        float dFn[M];  // minus the flux change: the volume term enters R_e with a minus sign
#pragma unroll
        for (int a = 0; a < M; ++a) {
          const float* ah = &Ah[q * AQ + (r * M + a) * M];
          const float2 t = __ffma2_rn(ld2(ah + 2), du23, __fmul2_rn(ld2(ah), du01));
          dFn[a] = -t.x - t.y;
        }
#pragma unroll
        for (int h = 0; h < NB2; ++h) {
          const float2 d2 = ld2(&D[(r * NQ + q) * NB + 2 * h]);
#pragma unroll
          for (int a = 0; a < M; ++a) dR2[h][a] = __ffma2_rn(d2, make_float2(dFn[a], dFn[a]), dR2[h][a]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const signed char bt = bcs[k];
      // rolled for the same instruction-fetch reason as in jvp_state
#pragma unroll 1
      for (int f = 0; f < NFQ; ++f) {
        float dui[M], duo[M];
#pragma unroll
        for (int b = 0; b < M; ++b) {
          float s = 0.0f, so = 0.0f;
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            s += Lt[f * NT + j] * dUe(Dd::face_node(k, j) * M + b);
            so += Lt[f * NT + j] * dUp((k * NT + j) * M + b);
          }
          dui[b] = s;
          duo[b] = (bt == 0) ? so : ((bt == 2) ? s : 0.0f);
        }
        const int pt = k * NFQ + f;
        const float2 ui01 = make_float2(dui[0], dui[1]), ui23 = make_float2(dui[2], dui[3]);
        const float2 uo01 = make_float2(duo[0], duo[1]), uo23 = make_float2(duo[2], duo[3]);
#pragma unroll
        for (int a = 0; a < M; ++a) {
          const float* hp = &Hp[(pt * M + a) * M];
          const float* hm = &Hm[(pt * M + a) * M];
          float2 t = __fmul2_rn(ld2(hp), ui01);
          t = __ffma2_rn(ld2(hp + 2), ui23, t);
          t = __ffma2_rn(ld2(hm), uo01, t);
          t = __ffma2_rn(ld2(hm + 2), uo23, t);
          const float dH = t.x + t.y;
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            const int node = Dd::face_node(k, j);
            const float v = fw[f] * Lt[f * NT + j] * dH;
            if (node & 1) dR2[node >> 1][a].y += v;
            else dR2[node >> 1][a].x += v;
          }
        }
      }
    }
#pragma unroll
    for (int h = 0; h < NB2; ++h)
#pragma unroll
      for (int a = 0; a < M; ++a) {
        dRo[(2 * h) * M + a] = dR2[h][a].x;
        dRo[(2 * h + 1) * M + a] = dR2[h][a].y;
      }
  }

  // FP32 Euler state columns (n_b even: p = 2) by rows of the element Jacobian.
  // Lane r owns row r = (i, a) of J = dR_e/dU_e with its n_u entries in registers,
  // paired over the nodes 2h, 2h + 1: the volume block
  //   J[(i,a)][(j,b)] = -sum_q B_q[j] sum_r D_r[q][i] Ahat_qr[a][b]
  // plus the interior trace's face blocks sum_f fw Lt[f][ii] Lt[f][jj] (dH/dU+,
  // plus dH/dU- on outflow faces where U- = U+)[a][b], then
  //   A[r][c] = sum_col J[r][col] Phi_e[col][c]
  // eight or four columns at a time on packed pairs. The neighbour traces of
  // interior faces are added by columns afterwards (jac_state_neighbours_f2). The
  // same sums as the Jacobian-vector products, taken in another order.
  __device__ void jac_state_rows_f2(int lane, const signed char* bcs, int ku, int k) {
    static_assert(M == 4 && NB % 2 == 0 && DIM == 2, "packed rows need four variables and an even node count");
    constexpr int NB2 = NB / 2;
    auto ld2 = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
    auto ld4 = [](const float* p) { return *reinterpret_cast<const float4*>(p); };
    const bool vec = (ku % 4 == 0) && (k % 4 == 0);  // 16-byte rows of Phi_e and A
    for (int row = lane; row < NU; row += 32) {
      const int i = row >> 2, a = row & 3;
      float2 J2[NB2][M];  // (J[row][(2h, b)], J[row][(2h + 1, b)])
#pragma unroll
      for (int h = 0; h < NB2; ++h)
#pragma unroll
        for (int b = 0; b < M; ++b) J2[h][b] = make_float2(0.0f, 0.0f);
#pragma unroll 1
      for (int q = 0; q < NQ; ++q) {
        // t[b] = -sum_r D_r[q][i] Ahat_qr[a][b] (the volume term enters R_e with a minus sign)
        const float d0 = -D[q * NB + i], d1 = -D[(NQ + q) * NB + i];
        const float4 a0 = ld4(&Ah[q * AQ + (0 * M + a) * M]);
        const float4 a1 = ld4(&Ah[q * AQ + (1 * M + a) * M]);
        const float2 dd0 = make_float2(d0, d0), dd1 = make_float2(d1, d1);
        const float2 t01 = __ffma2_rn(dd1, make_float2(a1.x, a1.y), __fmul2_rn(dd0, make_float2(a0.x, a0.y)));
        const float2 t23 = __ffma2_rn(dd1, make_float2(a1.z, a1.w), __fmul2_rn(dd0, make_float2(a0.z, a0.w)));
        const float2 tb[4] = {make_float2(t01.x, t01.x), make_float2(t01.y, t01.y), make_float2(t23.x, t23.x),
                              make_float2(t23.y, t23.y)};
#pragma unroll
        for (int h = 0; h < NB2; ++h) {
          const float2 b2 = ld2(&B[q * NB + 2 * h]);
#pragma unroll
          for (int b = 0; b < M; ++b) J2[h][b] = __ffma2_rn(b2, tb[b], J2[h][b]);
        }
      }
      // the interior trace's face blocks (both nodes on face kf)
#pragma unroll
      for (int kf = 0; kf < NF; ++kf) {
        const int ii = face_pos(kf, i);
        if (ii < 0) continue;
        const bool outflow = bcs[kf] == 2;
#pragma unroll 1
        for (int f = 0; f < NFQ; ++f) {
          const int o = ((kf * NFQ + f) * M + a) * M;
          float4 hv = ld4(&Hp[o]);
          if (outflow) {
            const float4 hm = ld4(&Hm[o]);
            hv.x += hm.x;
            hv.y += hm.y;
            hv.z += hm.z;
            hv.w += hm.w;
          }
          const float hb[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
          for (int jj = 0; jj < NT; ++jj) {
            const int node = Dd::face_node(kf, jj);
            const float cf = Cf[(f * NT + ii) * NT + jj];
#pragma unroll
            for (int b = 0; b < M; ++b) {
              if (node & 1) J2[node >> 1][b].y += cf * hb[b];
              else J2[node >> 1][b].x += cf * hb[b];
            }
          }
        }
      }
      // A[row][c] = J[row] . Phi_e[:, c]
      float* arow = &A[row * ka];
      int c0 = 0;
      if (vec) {
        for (; c0 + 8 <= ku; c0 += 8) {
          float2 s[4] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f),
                         make_float2(0.0f, 0.0f)};
#pragma unroll
          for (int h = 0; h < NB2; ++h)
#pragma unroll
            for (int b = 0; b < M; ++b)
#pragma unroll
              for (int o = 0; o < 2; ++o) {
                const float jv = o ? J2[h][b].y : J2[h][b].x;
                const float2 jj = make_float2(jv, jv);
                const float* pr = &Phie[((2 * h + o) * M + b) * ku + c0];
                const float4 p0 = ld4(pr), p1 = ld4(pr + 4);
                s[0] = __ffma2_rn(jj, make_float2(p0.x, p0.y), s[0]);
                s[1] = __ffma2_rn(jj, make_float2(p0.z, p0.w), s[1]);
                s[2] = __ffma2_rn(jj, make_float2(p1.x, p1.y), s[2]);
                s[3] = __ffma2_rn(jj, make_float2(p1.z, p1.w), s[3]);
              }
          *reinterpret_cast<float4*>(&arow[c0]) = make_float4(s[0].x, s[0].y, s[1].x, s[1].y);
          *reinterpret_cast<float4*>(&arow[c0 + 4]) = make_float4(s[2].x, s[2].y, s[3].x, s[3].y);
        }
        if (c0 + 4 <= ku) {
          float2 s[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll
          for (int h = 0; h < NB2; ++h)
#pragma unroll
            for (int b = 0; b < M; ++b)
#pragma unroll
              for (int o = 0; o < 2; ++o) {
                const float jv = o ? J2[h][b].y : J2[h][b].x;
                const float2 jj = make_float2(jv, jv);
                const float4 p0 = ld4(&Phie[((2 * h + o) * M + b) * ku + c0]);
                s[0] = __ffma2_rn(jj, make_float2(p0.x, p0.y), s[0]);
                s[1] = __ffma2_rn(jj, make_float2(p0.z, p0.w), s[1]);
              }
          *reinterpret_cast<float4*>(&arow[c0]) = make_float4(s[0].x, s[0].y, s[1].x, s[1].y);
          c0 += 4;
        }
      }
      for (int c = c0; c < ku; ++c) {
        float s = 0.0f;
#pragma unroll
        for (int h = 0; h < NB2; ++h)
#pragma unroll
          for (int b = 0; b < M; ++b) {
            s += J2[h][b].x * Phie[((2 * h) * M + b) * ku + c];
            s += J2[h][b].y * Phie[((2 * h + 1) * M + b) * ku + c];
          }
        arow[c] = s;
      }
    }
    __syncwarp();
    jac_state_neighbours_f2(lane, bcs, ku, k);
  }

  // The neighbour traces of the interior faces, one column of Phi per lane: at each
  // face point the neighbour's trace along the column, dU- = sum_j Lt[f][j]
  // Phi'[j][:, c], dH = dH/dU- dU-, lifted onto the face's nodes (fw Lt[f][j] dH) and
  // added to A. Boundary faces have none: their exterior state is the far field
  // (no dependence on U) or the interior trace (in the face blocks of J).
  __device__ void jac_state_neighbours_f2(int lane, const signed char* bcs, int ku, int k) {
    auto ld2 = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
    for (int c = lane; c < ku; c += 32) {
#pragma unroll
      for (int kf = 0; kf < NF; ++kf) {
        if (bcs[kf] != 0) continue;
        float up[NT][M];  // the neighbour's trace rows along this column
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          const long long off = poff[kf * NT + j];
#pragma unroll
          for (int b = 0; b < M; ++b) up[j][b] = PhiG[off + b * ku + c];
        }
        float add[NT][M];
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
          for (int a = 0; a < M; ++a) add[j][a] = 0.0f;
#pragma unroll 1
        for (int f = 0; f < NFQ; ++f) {
          float duo[M];
#pragma unroll
          for (int b = 0; b < M; ++b) {
            float s = 0.0f;
#pragma unroll
            for (int j = 0; j < NT; ++j) s += Lt[f * NT + j] * up[j][b];
            duo[b] = s;
          }
          const float2 u01 = make_float2(duo[0], duo[1]), u23 = make_float2(duo[2], duo[3]);
          const int pt = kf * NFQ + f;
          float dH[M];
#pragma unroll
          for (int a = 0; a < M; ++a) {
            const float* hm = &Hm[(pt * M + a) * M];
            const float2 t = __ffma2_rn(ld2(hm + 2), u23, __fmul2_rn(ld2(hm), u01));
            dH[a] = t.x + t.y;
          }
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            const float wl = fw[f] * Lt[f * NT + j];
#pragma unroll
            for (int a = 0; a < M; ++a) add[j][a] += wl * dH[a];
          }
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          const int node = Dd::face_node(kf, j);
#pragma unroll
          for (int a = 0; a < M; ++a) A[(node * M + a) * ka + c] += add[j][a];
        }
      }
    }
    __syncwarp();
  }

  // Curved geometry derivatives along a direction dx of the six nodes (12 values):
  // dJ at volume point q gives the cofactor change dcof (4), the tangent change at
  // face point pt the scaled-normal change dnt (2); both are linear in dx.
  __device__ __forceinline__ void dcof_curved(const double* dx, int stride, int q, T dcof[4]) const {
    const T* gd = &GdV[q * 12];
    T J0 = T(0), J1 = T(0), J2 = T(0), J3 = T(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const T x0 = (T)dx[(2 * j) * stride], x1 = (T)dx[(2 * j + 1) * stride];
      J0 += x0 * gd[2 * j];
      J1 += x0 * gd[2 * j + 1];
      J2 += x1 * gd[2 * j];
      J3 += x1 * gd[2 * j + 1];
    }
    dcof[0] = J3;
    dcof[1] = -J2;
    dcof[2] = -J1;
    dcof[3] = J0;
  }
  __device__ __forceinline__ void dnt_curved(const double* dx, int stride, int pt, T dn[2]) const {
    const T* tw = &GtF[pt * 6];
    T tx = T(0), ty = T(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      tx += (T)dx[(2 * j) * stride] * tw[j];
      ty += (T)dx[(2 * j + 1) * stride] * tw[j];
    }
    dn[0] = ty;
    dn[1] = -tx;
  }

  // Step 6b: derivative of R_e along a mesh direction dx (n_x values, FP64).
  __device__ void jvp_geom(const double* dx, const double* mu, T dR[NU]) {
#pragma unroll
    for (int i = 0; i < NU; ++i) dR[i] = T(0);
    if constexpr (Dd::CURVED) {
#pragma unroll 1
      for (int q = 0; q < NQ; ++q) {
        T dcof[4];
        dcof_curved(dx, 1, q, dcof);
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int a = 0; a < M; ++a) {
            T dF = fph[(q * 2 + 0) * M + a] * dcof[0 * 2 + r] + fph[(q * 2 + 1) * M + a] * dcof[1 * 2 + r];
#pragma unroll
            for (int i = 0; i < NB; ++i) dR[i * M + a] -= D[(r * NQ + q) * NB + i] * dF;
          }
      }
#pragma unroll
      for (int k = 0; k < NF; ++k)
#pragma unroll
        for (int f = 0; f < NFQ; ++f) {
          const int pt = k * NFQ + f;
          T dn[2];
          dnt_curved(dx, 1, pt, dn);
#pragma unroll
          for (int a = 0; a < M; ++a) {
            T dH = Hn[(pt * M + a) * 2 + 0] * dn[0] + Hn[(pt * M + a) * 2 + 1] * dn[1];
#pragma unroll
            for (int j = 0; j < NT; ++j) dR[Dd::face_node(k, j) * M + a] += fw[f] * Lt[f * NT + j] * dH;
          }
        }
    } else if (DIM == 2) {
      T dj00 = (T)(dx[2] - dx[0]), dj01 = (T)(dx[4] - dx[0]);
      T dj10 = (T)(dx[3] - dx[1]), dj11 = (T)(dx[5] - dx[1]);
      T dcof[4] = {dj11, -dj10, -dj01, dj00};
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int a = 0; a < M; ++a) {
            T dF = fph[(q * 2 + 0) * M + a] * dcof[0 * 2 + r] + fph[(q * 2 + 1) * M + a] * dcof[1 * 2 + r];
#pragma unroll
            for (int i = 0; i < NB; ++i) dR[i * M + a] -= D[(r * NQ + q) * NB + i] * dF;
          }
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int k1 = (k + 1) % 3;
        T dnx = (T)(dx[2 * k1 + 1] - dx[2 * k + 1]);
        T dny = (T)(-(dx[2 * k1] - dx[2 * k]));
#pragma unroll
        for (int f = 0; f < NFQ; ++f) {
          const int pt = k * NFQ + f;
#pragma unroll
          for (int a = 0; a < M; ++a) {
            T dH = Hn[(pt * M + a) * 2 + 0] * dnx + Hn[(pt * M + a) * 2 + 1] * dny;
#pragma unroll
            for (int j = 0; j < NT; ++j) dR[Dd::face_node(k, j) * M + a] += fw[f] * Lt[f * NT + j] * dH;
          }
        }
      }
    } else {
      // Burgers: only the source term -int v s(x) dX depends on the mesh
      T dx0 = (T)dx[0], ddet = (T)(dx[1] - dx[0]);
      T mu0 = (T)mu[0];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T dxq = dx0 + qxi[q] * ddet;
        T ds = qw[q] * (mu0 * sq[q] * dxq * detJ + sq[q] * ddet);
#pragma unroll
        for (int i = 0; i < NB; ++i) dR[i] -= B[q * NB + i] * ds;
      }
    }
  }

  // Position of element node i on face k (or -1).
  __device__ static int face_pos(int k, int i) {
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int node = (k == 0) ? Dd::face_node(0, j) : ((k == 1) ? Dd::face_node(1, j) : Dd::face_node(2, j));
      if (node == i) return j;
    }
    return -1;
  }

  // Step 6, state columns: A[row][c] = (dR_e/dU_e Phi_e + dR_e/dU_e' Phi_e')[row][c],
  // c < ku, with A stored row-major with stride k. The whole warp works on every
  // stage: per volume point it stages G = B_q Phi_e (M x ku) and F_r = Ahat_qr G
  // (DIM M x ku) in W, then every lane updates its own flattened (row, c) entries;
  // per face point it stages the trace directions dU+/dU- and dH = Hp dU+ + Hm dU-.
  __device__ void jac_state(int lane, const signed char* bcs, int ku, int k) {
    if constexpr (sizeof(T) == 4 && kStateRowsF32(M, NB)) {
      // FP32 Euler with p <= 2 (issue-bound): the rows of dR_e/dU_e in registers,
      // then their products with Phi_e, and the neighbour traces by columns
      jac_state_rows_f2(lane, bcs, ku, k);
      return;
    }
    if constexpr (sizeof(T) == 4) {
      // FP32 (issue-bound): one lane per column of Phi_e, the whole derivative of R_e
      // along it by Jacobian-vector products with no index arithmetic and no staging
      for (int c = lane; c < ku; c += 32) {
        T dR[NU];
        auto fe = [&](int i) { return Phie[i * ku + c]; };
        auto fp = [&](int i) {
          const int kj = i / M, b = i - kj * M;
          const long long off = poff[kj];
          return off >= 0 ? PhiG[off + b * ku + c] : T(0);
        };
        if constexpr (M == 4 && NB % 2 == 0) jvp_state_f2(fe, fp, bcs, dR);
        else jvp_state(fe, fp, bcs, dR);
#pragma unroll
        for (int i = 0; i < NU; ++i) A[i * ka + c] = dR[i];
      }
      __syncwarp();
      return;
    }
    if constexpr (kExplicitVolume(NU, sizeof(T))) {
      // volume part of dR_e/dU_e: Jv[(i,a)][(j,b)] = -sum_q B_q[j] T_q[(i,a)][b] with
      // T_q[(i,a)][b] = sum_r D_r[q][i] Ahat_qr[a][b], formed in passes of RP rows whose
      // entries are lane-owned registers, then A_vol = Jv Phi_e for those rows
      constexpr int NPASS = (NU * NU + kJvPass - 1) / kJvPass;
      static_assert(NU % NPASS == 0, "rows must split evenly into passes");
      constexpr int RP = NU / NPASS, NJ = (RP * NU + 31) / 32;
      T* Tq = W;            // [RP][M]
      T* Jp = W + RP * M;   // [RP][NU]
#pragma unroll 1
      for (int pass = 0; pass < NPASS; ++pass) {
        const int r0 = pass * RP;
        T jv[NJ];
#pragma unroll
        for (int t = 0; t < NJ; ++t) jv[t] = T(0);
        for (int q = 0; q < NQ; ++q) {
          __syncwarp();
          for (int e = lane; e < RP * M; e += 32) {
            const int rl = e / M, b = e - rl * M;
            const int row = r0 + rl, i = row / M, a = row - i * M;
            T s = T(0);
#pragma unroll
            for (int r = 0; r < DIM; ++r) s += D[(r * NQ + q) * NB + i] * Ah[q * AQ + (r * M + a) * M + b];
            Tq[e] = s;
          }
          __syncwarp();
#pragma unroll
          for (int t = 0; t < NJ; ++t) {
            const int e = lane + 32 * t;
            if (e < RP * NU) {
              const int rl = e / NU, col = e - rl * NU;
              const int j = col / M, b = col - j * M;
              jv[t] -= B[q * NB + j] * Tq[rl * M + b];
            }
          }
        }
        // the faces' blocks of dR_e/dU_e (both nodes on face kf): sum_f fw Lt[f][i] Lt[f][j]
        // times dH/dU+ (plus dH/dU- on outflow faces, where U- = U+), added before the
        // product with Phi_e; jac_state_faces then does the neighbour traces only
#pragma unroll
        for (int t = 0; t < NJ; ++t) {
          const int e = lane + 32 * t;
          if (e < RP * NU) {
            const int rl = e / NU, col = e - rl * NU;
            const int row = r0 + rl, i = row / M, a = row - i * M;
            const int j = col / M, b = col - j * M;
            T s = T(0);
#pragma unroll
            for (int kf = 0; kf < NF; ++kf) {
              const int ii = face_pos(kf, i), jj = face_pos(kf, j);
              if (ii < 0 || jj < 0) continue;
              const bool outflow = bcs[kf] == 2;
#pragma unroll
              for (int f = 0; f < NFQ; ++f) {
                const int o = ((kf * NFQ + f) * M + a) * M + b;
                const T h = outflow ? Hp[o] + Hm[o] : Hp[o];
                s += Cf[(f * NT + ii) * NT + jj] * h;
              }
            }
            jv[t] += s;
          }
        }
#pragma unroll
        for (int t = 0; t < NJ; ++t) {
          const int e = lane + 32 * t;
          if (e < RP * NU) Jp[e] = jv[t];
        }
        __syncwarp();
        for (int e = lane; e < RP * ku; e += 32) {
          const int rl = dku.div(e), c = e - rl * ku;
          const T* jr = &Jp[rl * NU];
          T s = T(0);
#pragma unroll
          for (int col = 0; col < NU; ++col) s += jr[col] * Phie[col * ku + c];
          A[(r0 + rl) * ka + c] = s;
        }
        __syncwarp();
      }
    } else {
      jac_state_volume_jvp(lane, ku, k);
    }
    jac_state_faces(lane, bcs, ku, k, kExplicitVolume(NU, sizeof(T)));
  }

  // Volume part of the state columns by Jacobian-vector products: per volume point,
  // G = B_q Phi_e (M x ku), F_r = Ahat_qr G (DIM M x ku), A -= D_r[q] F_r.
  __device__ void jac_state_volume_jvp(int lane, int ku, int k) {
    for (int e = lane; e < NU * ku; e += 32) {
      const int row = dku.div(e), c = e - row * ku;
      A[row * ka + c] = T(0);
    }
    T* G = W;
    T* F = W + M * ku;
    for (int q = 0; q < NQ; ++q) {
      __syncwarp();
      for (int e = lane; e < M * ku; e += 32) {
        const int b = dku.div(e), c = e - b * ku;
        T s = T(0);
#pragma unroll
        for (int j = 0; j < NB; ++j) s += B[q * NB + j] * Phie[(j * M + b) * ku + c];
        G[e] = s;
      }
      __syncwarp();
      for (int e = lane; e < DIM * M * ku; e += 32) {
        const int ra = dku.div(e), c = e - ra * ku;
        const T* ah = &Ah[q * AQ + ra * M];
        T s = T(0);
#pragma unroll
        for (int b = 0; b < M; ++b) s += ah[b] * G[b * ku + c];
        F[e] = s;
      }
      __syncwarp();
      for (int e = lane; e < NU * ku; e += 32) {
        const int row = dku.div(e), c = e - row * ku;
        const int i = row / M, a = row - i * M;
        T s = A[row * ka + c];
#pragma unroll
        for (int r = 0; r < DIM; ++r) s -= D[(r * NQ + q) * NB + i] * F[(r * M + a) * ku + c];
        A[row * ka + c] = s;
      }
    }
  }

  // Face part of the state columns: per face point, the trace directions dU+ (this
  // element's Phi rows) and dU- (the neighbour's trace rows), dH = Hp dU+ + Hm dU-,
  // lifted onto the face's nodes.
  // neighbour_only: the interior trace's blocks are already in the volume block
  // (explicit form), so only interior faces' neighbour traces remain: dH = Hm dU-.
  __device__ void jac_state_faces(int lane, const signed char* bcs, int ku, int k, bool neighbour_only = false) {
    T* dU = W;                // [2][M][ku]: interior, exterior
    T* dH = W + 2 * M * ku;   // [M][ku]
    const int s0 = neighbour_only ? 1 : 0;  // first side staged
    for (int pt = 0; pt < NF * NFQ; ++pt) {
      const int kf = pt / NFQ, f = pt - kf * NFQ;
      const signed char bt = bcs[kf];
      if (neighbour_only && bt != 0) continue;  // boundary faces: no neighbour trace
      __syncwarp();
      for (int e = lane + s0 * M * ku; e < 2 * M * ku; e += 32) {
        const int sb = dku.div(e), c = e - sb * ku;
        const int side = sb / M, b = sb - side * M;
        T s = T(0);
        if (side == 0 || bt == 2) {
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            const int node =
                (kf == 0) ? Dd::face_node(0, j) : ((kf == 1) ? Dd::face_node(1, j) : Dd::face_node(2, j));
            s += Lt[f * NT + j] * Phie[(node * M + b) * ku + c];
          }
        } else if (bt == 0) {
#pragma unroll
          for (int j = 0; j < NT; ++j) s += Lt[f * NT + j] * PhiG[poff[kf * NT + j] + b * ku + c];
        }
        dU[e] = s;
      }
      __syncwarp();
      for (int e = lane; e < M * ku; e += 32) {
        const int a = dku.div(e), c = e - a * ku;
        const T* hp = &Hp[(pt * M + a) * M];
        const T* hm = &Hm[(pt * M + a) * M];
        T s = T(0);
        if (neighbour_only) {
#pragma unroll
          for (int b = 0; b < M; ++b) s += hm[b] * dU[(M + b) * ku + c];
        } else {
#pragma unroll
          for (int b = 0; b < M; ++b) s += hp[b] * dU[b * ku + c] + hm[b] * dU[(M + b) * ku + c];
        }
        dH[e] = fw[f] * s;
      }
      __syncwarp();
      for (int e = lane; e < NT * M * ku; e += 32) {
        const int ja = dku.div(e), c = e - ja * ku;
        const int j = ja / M, a = ja - j * M;
        const int node = (kf == 0) ? Dd::face_node(0, j) : ((kf == 1) ? Dd::face_node(1, j) : Dd::face_node(2, j));
        A[(node * M + a) * ka + c] += Lt[f * NT + j] * dH[a * ku + c];
      }
    }
    __syncwarp();
  }

  // Step 6, mesh columns: A[row][ku + c] = (dR_e/dx_e Psi_e)[row][c], c < kx.
  // Volume: the flux enters through the cofactor matrix, linear in x_e, so the
  // direction dx = Psi_e[:, c] gives dF_r = sum_d f_d dcof[d][r]; the quadrature
  // sum is taken once per element, E[i][a][r][d] = sum_q D_r[q][i] f_d(U_q)_a
  // (staged in W), and each column is then sum_{r,d} dcof[c][d][r] E[i][a][r][d].
  // Faces: dH = Hn dn with the scaled-normal change dn; Burgers: the source only.
  // Mesh columns of A_e on curved elements: the cofactor and the normals vary by
  // point, so the quadrature sum cannot be factored out of the columns as for
  // straight sides. Per (volume point, column) the flux change dF_r = sum_d f_d
  // dcof[d][r], per (face point, column) the flux change dH = Hn dnt are staged in
  // W; each entry (row, column) is then -sum_q sum_r D_r[q][i] dF + the lifted dH.
  __device__ void jac_geom_curved(int lane, int ku, int kx, int k, bool dist) {
    T* dF = W;                     // [NQ][kx][M][2]
    T* dHf = W + NQ * kx * M * 2;  // [NF NFQ][kx][M]
    for (int t = lane; t < NQ * kx; t += 32) {
      const int q = dkx.div(t), c = t - q * kx;
      T dcof[4];
      dcof_curved(&Psie[c], kx, q, dcof);
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int r = 0; r < 2; ++r)
          dF[(t * M + a) * 2 + r] = fph[(q * 2 + 0) * M + a] * dcof[0 * 2 + r] + fph[(q * 2 + 1) * M + a] * dcof[1 * 2 + r];
    }
    for (int t = lane; t < NF * NFQ * kx; t += 32) {
      const int pt = dkx.div(t), c = t - pt * kx;
      T dn[2];
      dnt_curved(&Psie[c], kx, pt, dn);
#pragma unroll
      for (int a = 0; a < M; ++a) dHf[t * M + a] = Hn[(pt * M + a) * 2 + 0] * dn[0] + Hn[(pt * M + a) * 2 + 1] * dn[1];
    }
    __syncwarp();
    for (int e = lane; e < NU * kx; e += 32) {
      const int row = dkx.div(e), c = e - row * kx;
      const int i = row / M, a = row - i * M;
      T s = T(0);
#pragma unroll 4
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r) s -= D[(r * NQ + q) * NB + i] * dF[((q * kx + c) * M + a) * 2 + r];
#pragma unroll
      for (int kf = 0; kf < NF; ++kf) {
        const int j = face_pos(kf, i);
        if (j < 0) continue;
#pragma unroll
        for (int f = 0; f < NFQ; ++f) s += fw[f] * Lt[f * NT + j] * dHf[(((kf * NFQ + f) * kx) + c) * M + a];
      }
      A[row * ka + ku + c] = s;
    }
    if (dist) {
      for (int c = lane; c < kx; c += 32) {
        double s = 0.0;
#pragma unroll
        for (int r = 0; r < NXE; ++r) s += dN[r] * Psie[r * kx + c];
        dNt[c] = (T)s;
      }
    }
    __syncwarp();
  }

  // Distortion of a curved element (Eqs. dist_elem0-1): eta_e = sum_q w_q det JX_q
  // (|G_q|_F^2 / max(g_q, eps))^2 with G_q = Jx_q JX_q^{-1} (d = 2), and its
  // derivative through dJx_q / dx_js = delta_rs dN_j/dxi; written by one lane into
  // dN[0..NXE-1] and dN[NXE] = kappa (eta(x_e) - eta(X_e)). Xe: reference nodes.
  __device__ void distortion_curved(const double* Xe, double kappa, double eps) {
    double eta = 0.0, eta0 = 0.0, de[NXE];
#pragma unroll
    for (int r = 0; r < NXE; ++r) de[r] = 0.0;
    for (int q = 0; q < NQ; ++q) {
      const T* gd = &GdV[q * 12];
      double A4[4] = {0.0, 0.0, 0.0, 0.0}, J4[4] = {0.0, 0.0, 0.0, 0.0};  // [r * 2 + c]
      for (int j = 0; j < 6; ++j)
        for (int r = 0; r < 2; ++r)
          for (int c = 0; c < 2; ++c) {
            A4[r * 2 + c] += Xe[2 * j + r] * (double)gd[2 * j + c];
            J4[r * 2 + c] += xe[2 * j + r] * (double)gd[2 * j + c];
          }
      const double dA = A4[0] * A4[3] - A4[1] * A4[2];
      const double Ai[4] = {A4[3] / dA, -A4[1] / dA, -A4[2] / dA, A4[0] / dA};
      const double w = (double)qw[q] * dA;
      // value at the reference nodes (G = I) and at x_e
      for (int pass = 0; pass < 2; ++pass) {
        const double* Jx = pass == 0 ? A4 : J4;
        double G[4];
        for (int r = 0; r < 2; ++r)
          for (int c = 0; c < 2; ++c) G[r * 2 + c] = Jx[r * 2] * Ai[c] + Jx[r * 2 + 1] * Ai[2 + c];
        const double n2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2] + G[3] * G[3];
        const double g = G[0] * G[3] - G[1] * G[2];
        const double den = g >= eps ? g : eps;
        const double ratio = n2 / den;
        if (pass == 0) {
          eta0 += w * ratio * ratio;
          continue;
        }
        eta += w * ratio * ratio;
        // d ratio / d Jx[r][k]: |G|^2 through G = Jx Ai, g = det Jx / det JX (the g-branch only)
        const double cofJ[4] = {Jx[3], -Jx[2], -Jx[1], Jx[0]};  // d det Jx / d Jx[r][k]
        for (int r = 0; r < 2; ++r)
          for (int k2 = 0; k2 < 2; ++k2) {
            const double dn2 = 2.0 * (G[r * 2] * Ai[k2 * 2] + G[r * 2 + 1] * Ai[k2 * 2 + 1]);
            const double dg = g >= eps ? cofJ[r * 2 + k2] / dA : 0.0;
            const double dratio = dn2 / den - n2 / (den * den) * dg;
            const double dval = w * 2.0 * ratio * dratio;
            for (int j = 0; j < 6; ++j) de[2 * j + r] += dval * (double)gd[2 * j + k2];
          }
      }
    }
#pragma unroll
    for (int r = 0; r < NXE; ++r) dN[r] = kappa * de[r];
    dN[NXE] = kappa * (eta - eta0);
  }

  __device__ void distortion_any(const double* Xe, double kappa, double eps) {
    if constexpr (Dd::CURVED) distortion_curved(Xe, kappa, eps);
    else distortion(Xe, kappa, eps);
  }

  __device__ void jac_geom(int lane, const double* mu, int ku, int kx, int k, bool dist) {
    if (kx == 0) return;
    if constexpr (Dd::CURVED) {
      jac_geom_curved(lane, ku, kx, k, dist);
      return;
    }
    T* E = W;                  // [NB][M][DIM][DIM]
    T* dcof = W + NB * M * 4;  // [kx][4]
    T* K = dcof + 4 * kx;      // [NF][NT][M][2]: sum_f fw[f] Lt[f][j] Hn[kf, f][a][d]
    T* dnt = K + NF * NT * M * 2;  // [NF][kx][2]: change of face kf's scaled normal along column c
    if (DIM == 2) {
      // the mesh-direction differences, once per column (FP64 differences of the
      // vertex rows of Psi, then one conversion each)
      for (int c = lane; c < kx; c += 32) {
        if constexpr (sizeof(T) == 4) {
          if (g32) {
            // the column's edge differences from the FP32 edge table: (dj00, dj10, dj01, dj11)
            const float4 d = reinterpret_cast<const float4*>(Psie)[1 + c];
            dcof[c * 4 + 0] = d.w;
            dcof[c * 4 + 1] = -d.y;
            dcof[c * 4 + 2] = -d.z;
            dcof[c * 4 + 3] = d.x;
            dnt[(0 * kx + c) * 2 + 0] = d.y;
            dnt[(0 * kx + c) * 2 + 1] = -d.x;
            dnt[(1 * kx + c) * 2 + 0] = d.w - d.y;
            dnt[(1 * kx + c) * 2 + 1] = -(d.z - d.x);
            dnt[(2 * kx + c) * 2 + 0] = -d.w;
            dnt[(2 * kx + c) * 2 + 1] = d.z;
            continue;
          }
        }
        const double* d = &Psie[c];  // column c, stride kx
        const T dj00 = (T)(d[2 * kx] - d[0]), dj01 = (T)(d[4 * kx] - d[0]);
        const T dj10 = (T)(d[3 * kx] - d[1 * kx]), dj11 = (T)(d[5 * kx] - d[1 * kx]);
        dcof[c * 4 + 0] = dj11;
        dcof[c * 4 + 1] = -dj10;
        dcof[c * 4 + 2] = -dj01;
        dcof[c * 4 + 3] = dj00;
#pragma unroll
        for (int kf = 0; kf < NF; ++kf) {
          const int k1 = (kf + 1) % 3;
          dnt[(kf * kx + c) * 2 + 0] = (T)(d[(2 * k1 + 1) * kx] - d[(2 * kf + 1) * kx]);
          dnt[(kf * kx + c) * 2 + 1] = (T)(-(d[(2 * k1) * kx] - d[(2 * kf) * kx]));
        }
      }
      for (int e = lane; e < NB * M * 4; e += 32) {
        const int ia = e >> 2, rd = e & 3, r = rd >> 1, d = rd & 1;
        const int i = ia / M, a = ia - i * M;
        T s = T(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) s += D[(r * NQ + q) * NB + i] * fph[(q * 2 + d) * M + a];
        E[e] = s;
      }
      for (int e = lane; e < NF * NT * M * 2; e += 32) {
        const int kja = e >> 1, d = e & 1;
        const int kf = kja / (NT * M), ja = kja - kf * NT * M;
        const int j = ja / M, a = ja - j * M;
        T s = T(0);
#pragma unroll
        for (int f = 0; f < NFQ; ++f) s += fw[f] * Lt[f * NT + j] * Hn[((kf * NFQ + f) * M + a) * 2 + d];
        K[e] = s;
      }
      __syncwarp();
      for (int e = lane; e < NU * kx; e += 32) {
        const int row = dkx.div(e), c = e - row * kx;
        const int i = row / M, a = row - i * M;
        const T* er = &E[row * 4];
        const T* dc = &dcof[c * 4];
        // dcof[c][d*2 + r] pairs with E[i][a][r][d]
        T s = -(er[0] * dc[0] + er[1] * dc[2] + er[2] * dc[1] + er[3] * dc[3]);
        // faces through the nodes of this row
#pragma unroll
        for (int kf = 0; kf < NF; ++kf) {
          const int j = face_pos(kf, i);
          if (j < 0) continue;
          const T* dn = &dnt[(kf * kx + c) * 2];
          const T* kk = &K[((kf * NT + j) * M + a) * 2];
          s += kk[0] * dn[0] + kk[1] * dn[1];
        }
        A[row * ka + ku + c] = s;
      }
    } else {
      const T mu0 = (T)mu[0];
      for (int e = lane; e < NU * kx; e += 32) {
        const int i = dkx.div(e), c = e - i * kx;
        const T dx0 = (T)Psie[0 * kx + c], ddet = (T)(Psie[1 * kx + c] - Psie[0 * kx + c]);
        T s = T(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const T dxq = dx0 + qxi[q] * ddet;
          s -= B[q * NB + i] * qw[q] * (mu0 * sq[q] * dxq * detJ + sq[q] * ddet);
        }
        A[i * ka + ku + c] = s;
      }
    }
    if (dist) {
      for (int c = lane; c < kx; c += 32) {
        double s = 0.0;
#pragma unroll
        for (int r = 0; r < NXE; ++r) s += dN[r] * Psie[r * kx + c];
        dNt[c] = (T)s;
      }
    }
    __syncwarp();
  }

  // Distortion N_e (Eq. dist_elem0-1) for straight-sided simplices and dN/dx_e,
  // written by lane 0 into dN[0..NXE-1], dN[NXE] = N_e. Xe: reference vertices.
  __device__ void distortion(const double* Xe, double kappa, double eps) {
    if (DIM == 1) {
      // eta = |Omega_0e| (G^2 / max(g, eps)^2)^2 with G = g = (x1 - x0)/(X1 - X0)
      double h0 = Xe[1] - Xe[0];
      double G = (xe[1] - xe[0]) / h0;
      double den = G >= eps ? G : eps;
      double r = G * G / (den * den);
      double eta = h0 * r * r;
      double dr_dG = (G >= eps) ? 0.0 : 2.0 * G / (den * den);
      double deta = h0 * 2.0 * r * dr_dG / h0;  // d/dx1 (and minus for x0)
      dN[0] = -kappa * deta;
      dN[1] = kappa * deta;
      dN[NXE] = kappa * (eta - h0);
      return;
    }
    // G = Jx JX^{-1}; eta = |Omega_0e| (|G|_F^2 / max(g, eps))^2
    double a00 = Xe[2] - Xe[0], a01 = Xe[4] - Xe[0], a10 = Xe[3] - Xe[1], a11 = Xe[5] - Xe[1];
    double dA = a00 * a11 - a01 * a10;
    double i00 = a11 / dA, i01 = -a01 / dA, i10 = -a10 / dA, i11 = a00 / dA;
    double j00 = xe[2] - xe[0], j01 = xe[4] - xe[0], j10 = xe[3] - xe[1], j11 = xe[5] - xe[1];
    double G00 = j00 * i00 + j01 * i10, G01 = j00 * i01 + j01 * i11;
    double G10 = j10 * i00 + j11 * i10, G11 = j10 * i01 + j11 * i11;
    double nrm = G00 * G00 + G01 * G01 + G10 * G10 + G11 * G11;
    double g = G00 * G11 - G01 * G10;
    double area = 0.5 * dA;
    double den = g >= eps ? g : eps;
    double ratio = nrm / den;
    double eta = area * ratio * ratio;
    double eta0 = area * 4.0;  // G = I: |I|_F^2 / 1 = 2
    // d eta / d G = 2 area ratio (2 G / den - [g >= eps] nrm / den^2 cof(G))
    double c = 2.0 * area * ratio;
    double gb = (g >= eps) ? nrm / (den * den) : 0.0;
    double dG00 = c * (2.0 * G00 / den - gb * G11), dG01 = c * (2.0 * G01 / den + gb * G10);
    double dG10 = c * (2.0 * G10 / den + gb * G01), dG11 = c * (2.0 * G11 / den - gb * G00);
    // dG = dJx JX^{-1}: d eta / d Jx = (d eta / d G) JX^{-T}
    double dJ00 = dG00 * i00 + dG01 * i01, dJ01 = dG00 * i10 + dG01 * i11;
    double dJ10 = dG10 * i00 + dG11 * i01, dJ11 = dG10 * i10 + dG11 * i11;
    // Jx columns: vertex 1 - vertex 0, vertex 2 - vertex 0
    dN[0] = -kappa * (dJ00 + dJ01);
    dN[1] = -kappa * (dJ10 + dJ11);
    dN[2] = kappa * dJ00;
    dN[3] = kappa * dJ10;
    dN[4] = kappa * dJ01;
    dN[5] = kappa * dJ11;
    dN[NXE] = kappa * (eta - eta0);
  }
};

// Stage the shared reference tables (converted to T) and the evaluation point.
template <class T, int PROB, int P>
__device__ inline void stage_cta(const AsmArgs<T>& a, unsigned char* smem, const double* w, const double* tau,
                                 T*& tab, T*& wT, double*& tauD, float** tauF = nullptr) {
  using TB = Tabs<T, PROB, P>;
  using Dd = Disc<PROB, P>;
  tab = (T*)smem;
  const size_t o_w = align16(TB::total * sizeof(T)) + align16(TB::nC * sizeof(T));
  wT = (T*)(smem + o_w);
  tauD = (double*)(smem + o_w + align16((size_t)(a.ku > 0 ? a.ku : 1) * sizeof(T)));
  for (int i = threadIdx.x; i < TB::total; i += blockDim.x) tab[i] = (T)a.tables[i];
  // fw[f] Lt[f][i] Lt[f][j] from the FP64 host tables (packed D | B | Lt | fw | ...)
  T* cf = (T*)(smem + TB::cf_offset());
  for (int i = threadIdx.x; i < TB::nC; i += blockDim.x) {
    const int f = i / (Dd::NTRACE * Dd::NTRACE), ij = i - f * Dd::NTRACE * Dd::NTRACE;
    const int ii = ij / Dd::NTRACE, jj = ij - ii * Dd::NTRACE;
    const double* Lt = a.tables + TB::nD + TB::nB;
    const double w = a.tables[TB::nD + TB::nB + TB::nL + f];
    cf[i] = (T)(w * Lt[f * Dd::NTRACE + ii] * Lt[f * Dd::NTRACE + jj]);
  }
  for (int i = threadIdx.x; i < a.ku; i += blockDim.x) wT[i] = (T)w[i];
  for (int i = threadIdx.x; i < a.kx; i += blockDim.x) tauD[i] = tau[i];
  float* tf = (float*)((unsigned char*)tauD + align16((size_t)(a.kx > 0 ? a.kx : 1) * 8));
  for (int i = threadIdx.x; i < a.kx; i += blockDim.x) tf[i] = (float)tau[i];
  if (tauF) *tauF = tf;
}

template <class T, int PROB, int P, bool JAC>
__device__ inline void bind_tables(ElemCore<T, PROB, P, JAC>& C, T* tab) {
  using TB = Tabs<T, PROB, P>;
  C.D = tab;
  C.B = C.D + TB::nD;
  C.Lt = C.B + TB::nB;
  C.fw = C.Lt + TB::nL;
  C.qw = C.fw + TB::nfw;
  C.qxi = C.qw + TB::nqw;
  C.GdV = C.qxi + TB::nqx;
  C.GtF = C.GdV + TB::nGv;
  C.Cf = (const T*)((const unsigned char*)tab + TB::cf_offset());
}

// Steps 1-5 for element e at the state (wT, tauD) and parameters mu: gather,
// reconstruction, geometry, pointwise fluxes (and their derivatives when JAC)
// and R_e in C.R. bcs receives the element's face types. Returns true if the
// element is non-physical or R_e is not finite.
template <class T, int PROB, int P, bool JAC>
__device__ __forceinline__ bool element_front(ElemCore<T, PROB, P, JAC>& C, const AsmArgs<T>& a, int e,
                                              const T* wT, const double* tauD, const double* mu, int lane,
                                              signed char* bcs, bool face_jac = true, bool vol_jac = true,
                                              int step = 32, const float* tauF = nullptr) {
  using Dd = Disc<PROB, P>;
  constexpr int M = Dd::M, DIM = Dd::DIM, NU = Dd::NU, NUP = Dd::NUP, NXE = Dd::NXE, NF = Dd::NFACE,
                NT = Dd::NTRACE, NV = Dd::NV;
  const int ku = a.ku, kx = a.kx;
  const bool need_hn = JAC && (kx > 0 || a.need_hn) && face_jac;
    const int* vv = &a.ev[(long)e * NV];
    // FP32 straight-sided elements without the distortion term take their geometry
    // from the FP32 edge table (no FP64 arithmetic in the element pass)
    bool g32 = false;
    if constexpr (sizeof(T) == 4 && !Dd::CURVED && DIM == 2)
      g32 = tauF != nullptr && a.geo32 != nullptr && a.kappa == 0.0;
    C.g32 = g32;
    // 1. gather: Phi_e and Psi_e (or the element's edge-table rows) by asynchronous
    // copies (all in flight at once), overlapped with the neighbour offsets
    warp_copy_async(C.Phie, a.Phi + (size_t)e * NU * ku, NU * ku, lane, step);
    if (g32) {
      const float4* src = a.geo32 + (size_t)e * (1 + kx);
      for (int i = lane; i < 1 + kx; i += step) cp_async16(reinterpret_cast<float4*>(C.Psie) + i, src + i);
    } else {
      for (int i = lane; i < NXE * kx; i += step) {
        const int r = C.dkx.div(i), c = i - r * kx;
        const int v = r / DIM, d = r - v * DIM;
        cp_async8(&C.Psie[i], &a.Psi[((size_t)vv[v] * DIM + d) * kx + c]);
      }
    }
    for (int t = lane; t < NF * NT; t += step) {
      const int kf = t / NT, j = t - kf * NT;
      const int e2 = a.nbr[(long)e * NF + kf];
      const int k2 = a.nbr_face[(long)e * NF + kf];
      long long off = -1;
      if (e2 >= 0) {
        // neighbour trace node at position j along this face = its node NT-1-j on face k2
        const int jj = NT - 1 - j;
        const int node = (k2 == 0) ? Dd::face_node(0, jj) : ((k2 == 1) ? Dd::face_node(1, jj) : Dd::face_node(2, jj));
        off = ((long long)e2 * NU + node * M) * ku;
      }
      C.poff[t] = off;
    }
    C.PhiG = a.Phi;
    cp_async_wait_all();
    __syncwarp();
    // 2. reconstruction
    for (int i = lane; i < NU + NUP; i += step) {
      T s = T(0);
      if (i < NU) {
        const T* row = &C.Phie[i * ku];
        for (int c = 0; c < ku; ++c) s += row[c] * wT[c];
        C.Ue[i] = s;
      } else {
        const int r = i - NU, kj = r / M, b = r - kj * M;
        const long long off = C.poff[kj];
        if (off >= 0) {
          const T* row = C.PhiG + off + b * ku;
          for (int c = 0; c < ku; ++c) s += row[c] * wT[c];
        }
        C.Up[r] = s;
      }
    }
    for (int t = g32 ? NXE : lane; t < NXE; t += step) {
      const int v = t / DIM, d = t - v * DIM;
      double s = a.X[(size_t)vv[v] * DIM + d];
      for (int c = 0; c < kx; ++c) s += C.Psie[t * kx + c] * tauD[c];
      C.xe[t] = s;
    }
    __syncwarp();
    // 3. geometry
    bool bad;
    if constexpr (Dd::CURVED) {
      bad = !C.geometry_curved(lane, step);
      __syncwarp();
    } else if constexpr (sizeof(T) == 4 && DIM == 2) {
      bad = g32 ? !C.geometry32(tauF, kx) : !C.geometry();
    } else {
      bad = !C.geometry();
    }
#pragma unroll
    for (int kf = 0; kf < NF; ++kf) bcs[kf] = a.bc[(long)e * NF + kf];
    // 4. pointwise, 5. residual
    bad |= C.pointwise(lane, bcs, mu, a.gamma, need_hn, face_jac, vol_jac, step);
    __syncwarp();
    bad |= C.residual(lane, step);
    return bad;
}

// One element of the pass: steps 1-7 for element e with weight rho at the state
// (wT, tauD) and parameters mu; accumulates into the warp's C.acc. TC: H on the
// tensor cores (FP32 only; a separate instantiation, so the FP32 FMA kernel does
// not carry the tensor-core code's registers).
template <class T, int PROB, int P, bool JAC, bool TC = false>
__device__ __forceinline__ void element_pass(ElemCore<T, PROB, P, JAC>& C, const AsmArgs<T>& a, int e, double rho,
                                             const T* wT, const double* tauD, const double* mu,
                                             const unsigned char* pairs, int lane, const float* tauF = nullptr,
                                             long item = -1) {
  using Dd = Disc<PROB, P>;
  constexpr int DIM = Dd::DIM, NU = Dd::NU, NXE = Dd::NXE, NF = Dd::NFACE, NV = Dd::NV;
  const int ku = a.ku, kx = a.kx, k = ku + kx;
    const int* vv = &a.ev[(long)e * NV];
    signed char bcs[NF];
    bool bad = element_front<T, PROB, P, JAC>(C, a, e, wT, tauD, mu, lane, bcs, true, true, 32, tauF);
    // distortion
    const bool dist = a.kappa != 0.0;
    if (dist && lane == 0) {
      double Xe[NXE];
      for (int r = 0; r < NXE; ++r) Xe[r] = a.X[(size_t)vv[r / DIM] * DIM + (r % DIM)];
      C.distortion_any(Xe, a.kappa, a.eps);
    }
    __syncwarp();
    const T Ne = dist ? (T)C.dN[NXE] : T(0);
    if (JAC) {
      // 6. columns of A_e (state, then mesh), all lanes on every stage
      C.jac_state(lane, bcs, ku, k);
      C.jac_geom(lane, mu, ku, kx, k, dist);
      // 7. weighted contraction over the upper triangle: lane-owned pairs (r <= b),
      // or tensor-core tiles (FP32 contexts that ask for them)
      const T rT = (T)rho;
      bool simt_h = true;
      if constexpr (std::is_same<T, float>::value && TC) {
        {
          __syncwarp();
          if (a.contraction == 3 && NU % 2 == 0 && a.at_out != nullptr && item >= 0) {
            // the rows of sqrt(rho_e) A_e, transposed, to the stack the tensor-core
            // product reads after the pass (rho >= 0): word (m at_ld + item n_u) / 2 + j
            // holds (row 2j, row 2j + 1) of column m
            constexpr int NP = NU / 2;
            const float sr = sqrtf(rT);
            uint32_t* col0 = a.at_out + ((size_t)item * NU) / 2;
            for (int idx = lane; idx < k * NP; idx += 32) {
              const int m = idx / NP, j = idx - m * NP;
              col0[((size_t)m * a.at_ld) / 2 + j] =
                  pack_bf16x2(sr * C.A[(2 * j) * C.ka + m], sr * C.A[(2 * j + 1) * C.ka + m]);
            }
          } else if (a.contraction == 3) {
            // staged operands when T fits in the (no longer needed) Phi_e buffer
            if ((size_t)syrk_bf16_rs(NU) * k <= (size_t)NU * ku * sizeof(float))
              syrk_upper_bf16_staged<NU>(C.A, k, C.ka, reinterpret_cast<unsigned char*>(C.Phie), C.acc, rT, lane);
            else
              syrk_upper_bf16<NU>(C.A, k, C.ka, C.acc, rT, lane);
          }
          else if (a.contraction == 2) syrk_upper_tf32<NU, true>(C.A, k, C.ka, C.acc, rT, lane);
          else syrk_upper_tf32<NU, false>(C.A, k, C.ka, C.acc, rT, lane);
          if (dist) {
            // distortion block of the mesh columns, Eq. levmarq-elem
            const int np = kx * (kx + 1) / 2;
            for (int pidx = lane; pidx < np; pidx += 32) {
              int r = 0, rem = pidx;
              while (rem >= kx - r) {
                rem -= kx - r;
                ++r;
              }
              const int b = r + rem;
              C.acc[acc_h(ku + r, ku + b, k)] += rT * (C.dNt[r] * C.dNt[b]);
            }
          }
          simt_h = false;
        }
      }
      if constexpr (std::is_same<T, float>::value) {
        if (simt_h && k % 4 == 0) {
          // FP32 (issue-bound): each lane forms a 4 x 4 block of H's upper block
          // triangle with float4 loads of A's rows, 16 FMA per 2 shared loads
          __syncwarp();
          const int nb = k / 4, nblk = nb * (nb + 1) / 2;
          for (int blk = lane; blk < nblk; blk += 32) {
            int R = 0, rem = blk;
            while (rem >= nb - R) {
              rem -= nb - R;
              ++R;
            }
            const int Bc = R + rem;
            // the block on packed pairs: h2[x][p] = (h[x][2p], h[x][2p + 1])
            float2 h2[4][2];
#pragma unroll
            for (int x = 0; x < 4; ++x) h2[x][0] = h2[x][1] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < NU; ++i) {
              const float4 ar = *reinterpret_cast<const float4*>(&C.A[i * C.ka + 4 * R]);
              const float4 bc = *reinterpret_cast<const float4*>(&C.A[i * C.ka + 4 * Bc]);
              const float av[4] = {ar.x, ar.y, ar.z, ar.w};
              const float2 b01 = make_float2(bc.x, bc.y), b23 = make_float2(bc.z, bc.w);
#pragma unroll
              for (int x = 0; x < 4; ++x) {
                const float2 a2 = make_float2(av[x], av[x]);
                h2[x][0] = __ffma2_rn(a2, b01, h2[x][0]);
                h2[x][1] = __ffma2_rn(a2, b23, h2[x][1]);
              }
            }
            float h[4][4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
              h[x][0] = h2[x][0].x;
              h[x][1] = h2[x][0].y;
              h[x][2] = h2[x][1].x;
              h[x][3] = h2[x][1].y;
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int y = 0; y < 4; ++y) {
                const int r = 4 * R + x, b = 4 * Bc + y;
                if (r > b) continue;
                float v = h[x][y];
                if (dist && r >= ku) v += C.dNt[r - ku] * C.dNt[b - ku];
                C.acc[acc_h(r, b, k)] += rT * v;
              }
          }
          simt_h = false;
        }
      }
      const int npairs = simt_h ? k * (k + 1) / 2 : 0;
      for (int pidx = lane; pidx < npairs; pidx += 32) {
        const int r = pairs[2 * pidx], b = pairs[2 * pidx + 1];
        T s = T(0);
#pragma unroll
        for (int i = 0; i < NU; ++i) s += C.A[i * C.ka + r] * C.A[i * C.ka + b];
        if (dist && r >= ku) s += C.dNt[r - ku] * C.dNt[b - ku];
        C.acc[pidx] += rT * s;  // pairs run over the upper triangle in accumulator order
      }
      for (int r = lane; r < k; r += 32) {
        T s = T(0);
#pragma unroll
        for (int i = 0; i < NU; ++i) s += C.A[i * C.ka + r] * C.R[i];
        if (dist && r >= ku) s += C.dNt[r - ku] * Ne;
        C.acc[acc_tail(k) + r] += rT * s;
      }
    }
    if (lane == 0) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < NU; ++i) s += C.R[i] * C.R[i];
      C.acc[acc_tail(k) + k] += T(0.5) * (T)rho * (s + Ne * Ne);
      if (bad) C.acc[acc_tail(k) + k + 1] += T(1);
    }
    __syncwarp();
}

// One element of the gradient pass (FP64 residual, gradient and objective for LM
// iterations whose Gauss-Newton matrix comes from an FP32 assembly): R_e, then
// g += rho [Phi_e^T dUe + Phi_e'^T dUp ; Psi_e^T (dR_e/dx_e^T R_e + dN_e^T N_e)] with
// (dUe, dUp) the adjoint of the state Jacobians applied to R_e (no Jacobian
// columns are formed for the state), J += rho (|R_e|^2 + N_e^2) / 2.
template <class T, int PROB, int P>
// step 16 (Euler): the calling half-warp evaluates this element (lane = 0..15 in it)
// while the other half evaluates another; count = false: an idle half's stand-in
// element (rho = 0), whose non-physical flag is not counted.
__device__ __forceinline__ void element_grad_pass(ElemCore<T, PROB, P, true>& C, const AsmArgs<T>& a, int e,
                                                  double rho, const T* wT, const double* tauD, const double* mu,
                                                  int lane, int step = 32, bool count = true) {
  using Dd = Disc<PROB, P>;
  constexpr int DIM = Dd::DIM, M = Dd::M, NU = Dd::NU, NUP = Dd::NUP, NXE = Dd::NXE, NF = Dd::NFACE,
                NFQ = Dd::NFQ, NV = Dd::NV, NQ = Dd::NQ;
  constexpr bool kVJP = Dd::EULER;  // Euler: reverse-mode face adjoint, no face Jacobians
  const int ku = a.ku, kx = a.kx, k = ku + kx;
  const int* vv = &a.ev[(long)e * NV];
  signed char bcs[NF];
  const bool bad = element_front<T, PROB, P, true>(C, a, e, wT, tauD, mu, lane, bcs, !kVJP, !kVJP, step);
  const bool dist = a.kappa != 0.0;
  if (dist && lane == 0) {
    double Xe[NXE];
    for (int r = 0; r < NXE; ++r) Xe[r] = a.X[(size_t)vv[r / DIM] * DIM + (r % DIM)];
    C.distortion_any(Xe, a.kappa, a.eps);
  }
  __syncwarp();
  const T Ne = dist ? (T)C.dN[NXE] : T(0);
  const T rT = (T)rho;
  T *dUe, *dUp, *eps = nullptr, *nu = nullptr, *eq = nullptr;
  if constexpr (kVJP) C.adj_state_vjp(lane, bcs, a.gamma, dUe, dUp, eps, nu, step, &eq);
  else C.adj_state(lane, bcs, dUe, dUp);
  T* g = C.gacc;
  for (int c = lane; c < ku; c += step) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < NU; ++i) s += C.Phie[i * ku + c] * dUe[i];
#pragma unroll
    for (int i = 0; i < NUP; ++i) {
      const long long off = C.poff[i / M];
      if (off >= 0) s += C.PhiG[off + (i % M) * ku + c] * dUp[i];
    }
    g[c] += rT * s;
  }
  if (kx > 0) {
    if constexpr (kVJP) {
      // R_e^T dR_e/dx_e Psi_e[:, c]: the volume term through the cofactor change of the
      // direction, the face term through the scaled-normal change, plus distortion
      for (int c = lane; c < kx; c += step) {
        const double* d = &C.Psie[c];  // column c, stride kx
        T s = T(0);
        if constexpr (Dd::CURVED) {
          // per point: eq[q][r][d] = (D_r[q]^T R) . f_d(U_q) against the cofactor change,
          // nu[pt] against the scaled-normal change
#pragma unroll 1
          for (int q = 0; q < NQ; ++q) {
            T dcof[4];
            C.dcof_curved(d, kx, q, dcof);
            s -= eq[q * 4 + 0] * dcof[0] + eq[q * 4 + 1] * dcof[2] + eq[q * 4 + 2] * dcof[1] + eq[q * 4 + 3] * dcof[3];
          }
#pragma unroll
          for (int pt = 0; pt < NF * NFQ; ++pt) {
            T dn[2];
            C.dnt_curved(d, kx, pt, dn);
            s += nu[pt * 2 + 0] * dn[0] + nu[pt * 2 + 1] * dn[1];
          }
        } else {
          const T dj00 = (T)(d[2 * kx] - d[0]), dj01 = (T)(d[4 * kx] - d[0]);
          const T dj10 = (T)(d[3 * kx] - d[1 * kx]), dj11 = (T)(d[5 * kx] - d[1 * kx]);
          // dcof[d*2 + r] = (dj11, -dj10, -dj01, dj00) pairs with eps[r*2 + d]
          s = -(eps[0] * dj11 + eps[1] * (-dj01) + eps[2] * (-dj10) + eps[3] * dj00);
#pragma unroll
          for (int kf = 0; kf < NF; ++kf) {
            const int k1 = (kf + 1) % 3;
            const T dnx = (T)(d[(2 * k1 + 1) * kx] - d[(2 * kf + 1) * kx]);
            const T dny = (T)(-(d[(2 * k1) * kx] - d[(2 * kf) * kx]));
#pragma unroll
            for (int f = 0; f < NFQ; ++f) {
              const int pt = kf * NFQ + f;
              s += nu[pt * 2 + 0] * dnx + nu[pt * 2 + 1] * dny;
            }
          }
        }
        if (dist) {
          double dn = 0.0;
#pragma unroll
          for (int r = 0; r < NXE; ++r) dn += C.dN[r] * d[r * kx];
          s += (T)dn * Ne;
        }
        g[ku + c] += rT * s;
      }
    } else {
      __syncwarp();
      C.jac_geom(lane, mu, ku, kx, k, dist);  // mesh columns of A_e (overwrites the adjoint staging)
      for (int c = lane; c < kx; c += 32) {
        T s = T(0);
#pragma unroll
        for (int i = 0; i < NU; ++i) s += C.A[i * C.ka + ku + c] * C.R[i];
        if (dist) s += C.dNt[c] * Ne;
        g[ku + c] += rT * s;
      }
    }
  }
  if (lane == 0) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < NU; ++i) s += C.R[i] * C.R[i];
    g[k] += T(0.5) * rT * (s + Ne * Ne);
    if (bad && count) g[k + 1] += T(1);
  }
  __syncwarp();
}

// Upper-triangle (row <= col) pairs of the k x k Gauss-Newton matrix, row-major order.
__device__ inline void build_pairs(unsigned char* pairs, int k) {
  int n = 0;
  for (int r = 0; r < k; ++r)
    for (int b = r; b < k; ++b) {
      pairs[2 * n] = (unsigned char)r;
      pairs[2 * n + 1] = (unsigned char)b;
      ++n;
    }
}

// Accumulator entry i of the full [H | g | J | count] vector (H mirrored from its upper triangle).
__device__ inline int acc_source(int i, int k) {
  if (i < k * k) {
    int r = i / k, b = i - r * k;
    if (r > b) {
      const int t = r;
      r = b;
      b = t;
    }
    return acc_h(r, b, k);
  }
  return acc_tail(k) + (i - k * k);
}

// The fused assembly kernel (JAC = true) and the objective-only kernel (JAC = false)
// for one query: a grid-stride loop of warps over the items; one FP64 partial per CTA.
// The FP32 Jacobian form is capped at 168 registers (3 CTAs of 128 threads, 6 of
// the 64-thread CTAs it runs with); its small spill costs less than lost warps.
// Register cap of the FP32 Jacobian assembly (blocks of 128 threads per SM): 128
// registers where the element's state fits in them without spilling and its
// shared memory lets 16 warps reside (straight-sided p <= 2); 168 elsewhere
// (curved elements spill at 128; at p = 3 shared memory holds 6 warps anyway).
constexpr int kFp32JacMinBlocks(int prob, int p) { return (prob == PROB_EULER_Q2 || p > 2) ? 3 : 4; }

template <class T, int PROB, int P, bool JAC, bool TC = false, bool GRAD = false>
__global__ void __launch_bounds__(128, (sizeof(T) == 4 && JAC) ? kFp32JacMinBlocks(PROB, P) : 0)
    assemble_kernel(AsmArgs<T> a) {
  using Core = ElemCore<T, PROB, P, JAC>;
  extern __shared__ __align__(16) unsigned char smem[];
  if (a.skip != nullptr && *(volatile const int*)a.skip) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ku = a.ku, kx = a.kx, k = ku + kx;
  T *tab, *wT;
  double* tauD;
  float* tauF;
  stage_cta<T, PROB, P>(a, smem, a.w, a.tau, tab, wT, tauD, &tauF);
  using Lay = WarpLayout<T, PROB, P, JAC, GRAD, !GRAD>;
  constexpr int PW = Lay::PER_WARP;  // 2: two elements per warp, one per half-warp
  const int half = PW == 2 ? (lane >> 4) : 0, sub = PW == 2 ? (lane & 15) : lane, step = 32 / PW;
  const size_t cb = cta_bytes<T, PROB, P>(ku, kx);
  const size_t eb = Lay(ku, kx).bytes;  // one element's region; a warp holds PW of them
  Core C;
  C.template carve<GRAD, !GRAD>(smem + cb + (warp * PW + half) * eb, ku, kx);
  bind_tables(C, tab);
  const int nacc = k * k + k + 2;  // entries of a partial row (full H)
  const int nzero = Lay::SLIM ? k + 2 : acc_count(k);
  for (int i = sub; i < nzero; i += step) C.acc[i] = T(0);
  unsigned char* pairs = smem + cb + nw * PW * eb;
  if (needs_pair_table<T>(JAC, GRAD, true, k) && threadIdx.x == 0) build_pairs(pairs, k);
  __syncthreads();
  if constexpr (PW == 2) {
    // both halves take the same number of trips; a half without an element of its
    // own re-evaluates its partner's with rho = 0
    for (long base = ((long)blockIdx.x * nw + warp) * 2; base < a.n_items; base += (long)gridDim.x * nw * 2) {
      const long it = base + half;
      const bool real = it < a.n_items;
      const long ir = real ? it : base;
      const int e = a.elems ? a.elems[ir] : (int)ir;
      const double rho = real ? (a.rho ? a.rho[ir] : 1.0) : 0.0;
      element_grad_pass<T, PROB, P>(C, a, e, rho, wT, tauD, a.mu, sub, 16, real);
    }
  } else {
    for (long it = (long)blockIdx.x * nw + warp; it < a.n_items; it += (long)gridDim.x * nw) {
      const int e = a.elems ? a.elems[it] : (int)it;
      const double rho = a.rho ? a.rho[it] : 1.0;
      if constexpr (GRAD && JAC) element_grad_pass<T, PROB, P>(C, a, e, rho, wT, tauD, a.mu, lane);
      else element_pass<T, PROB, P, JAC, TC>(C, a, e, rho, wT, tauD, a.mu, pairs, lane, tauF, it);
    }
  }
  __syncthreads();
  // CTA partial: sum the accumulators of the CTA's element regions in order, in FP64
  // (gradient pass: rows of [g | J | count] only). FP32 accumulators are added in
  // FP32 and converted once: the FP64 unit takes a whole warp instruction per
  // conversion or add, and all CTAs reach this step at once at the end of the launch.
  Lay L(ku, kx);
  const int nrow = GRAD ? k + 2 : nacc;
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) {
    const int src = GRAD ? Lay::gacc_offset(k) + i : acc_source(i, k);
    double s = 0.0;
    if constexpr (sizeof(T) == 4) {
      T f = T(0);
      for (int w = 0; w < nw * PW; ++w) f += ((const T*)(smem + cb + w * eb + L.oacc))[src];
      s = (double)f;
    } else {
      for (int w = 0; w < nw * PW; ++w) s += (double)((const T*)(smem + cb + w * eb + L.oacc))[src];
    }
    a.partial[(size_t)blockIdx.x * nrow + i] = s;
  }
}

// Many queries at once (the batched hyperreduced path): every query has its own
// element list, weights, evaluation point and parameters. The items of query q
// are split into chunks of at most a few dozen elements; one warp evaluates one
// chunk and writes one FP64 partial row for it. Chunks of finished queries are
// skipped.
struct BatchArgs {
  const int* chunk_start;  // n_chunks + 1 offsets into the item arrays (elems, rho)
  const int* chunk_query;  // query of each chunk
  int n_chunks;
  const double* w;         // evaluation point of query q at w + q * wstride (tau follows at + ku)
  long wstride;
  const double* mu;        // parameters of query q at mu + q * mustride
  int mustride;
  const int* done;         // finished flag of query q at done + q * donestride (may be null)
  long donestride;
};

template <class T, int PROB, int P, bool JAC, bool TC = false, bool GRAD = false>
__global__ void __launch_bounds__(128, (sizeof(T) == 4 && JAC && PROB != PROB_EULER_Q2) ? kFp32JacMinBlocks(PROB, P) : 0)
    assemble_batched_kernel(AsmArgs<T> a, BatchArgs b) {
  using Core = ElemCore<T, PROB, P, JAC>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ku = a.ku, kx = a.kx, k = ku + kx;
  T *tab, *wT_unused;
  double* tau_unused;
  stage_cta<T, PROB, P>(a, smem, a.w, a.tau, tab, wT_unused, tau_unused);
  using Lay = WarpLayout<T, PROB, P, JAC, GRAD, !GRAD>;
  constexpr int PW = Lay::PER_WARP;  // 2: two elements per warp, one per half-warp
  const int half = PW == 2 ? (lane >> 4) : 0, sub = PW == 2 ? (lane & 15) : lane, step = 32 / PW;
  const size_t cb = cta_bytes<T, PROB, P>(ku, kx);
  const size_t eb = Lay(ku, kx).bytes;
  Lay L(ku, kx);
  unsigned char* wbase = smem + cb + (warp * PW + half) * eb;
  Core C;
  C.template carve<GRAD, !GRAD>(wbase, ku, kx);
  bind_tables(C, tab);
  T* wq = (T*)(wbase + L.owq);
  double* tq = (double*)(wbase + L.otq);
  float* tqf = (float*)(wbase + L.otqf);
  const int nacc = k * k + k + 2;
  const int nzero = Lay::SLIM ? k + 2 : acc_count(k);
  unsigned char* pairs = smem + cb + nw * PW * eb;
  if (needs_pair_table<T>(JAC, GRAD, true, k) && threadIdx.x == 0) build_pairs(pairs, k);
  __syncthreads();
  for (int ch = blockIdx.x * nw + warp; ch < b.n_chunks; ch += gridDim.x * nw) {
    const int q = b.chunk_query[ch];
    if (b.done != nullptr && *(volatile const int*)(b.done + (long)q * b.donestride)) continue;
    const double* wsrc = b.w + (long)q * b.wstride;
    for (int i = sub; i < ku; i += step) wq[i] = (T)wsrc[i];
    for (int i = sub; i < kx; i += step) {
      tq[i] = wsrc[ku + i];
      tqf[i] = (float)wsrc[ku + i];
    }
    for (int i = sub; i < nzero; i += step) C.acc[i] = T(0);
    __syncwarp();
    const double* muq = b.mu + (long)q * b.mustride;
    if constexpr (PW == 2) {
      // the chunk's items in pairs, one per half-warp; an odd last item leaves the
      // second half re-evaluating it with rho = 0
      const int i0 = b.chunk_start[ch], i1 = b.chunk_start[ch + 1];
#pragma unroll 1
      for (int it = i0; it < i1; it += 2) {
        const int my = it + half;
        const bool real = my < i1;
        const int ir = real ? my : it;
        element_grad_pass<T, PROB, P>(C, a, a.elems[ir], real ? a.rho[ir] : 0.0, wq, tq, muq, sub, 16, real);
      }
    } else {
#pragma unroll 1
      for (int it = b.chunk_start[ch]; it < b.chunk_start[ch + 1]; ++it) {
        if constexpr (GRAD && JAC) element_grad_pass<T, PROB, P>(C, a, a.elems[it], a.rho[it], wq, tq, muq, lane);
        else element_pass<T, PROB, P, JAC, TC>(C, a, a.elems[it], a.rho[it], wq, tq, muq, pairs, lane, tqf);
      }
    }
    __syncwarp();
    if (GRAD) {
      // both halves' accumulators (one region when PW = 1)
      const unsigned char* r0 = smem + cb + warp * PW * eb;
      for (int i = lane; i < k + 2; i += 32) {
        double v = 0.0;
        for (int h = 0; h < PW; ++h) v += (double)((const T*)(r0 + h * eb + L.oacc))[Lay::gacc_offset(k) + i];
        a.partial[(size_t)ch * (k + 2) + i] = v;
      }
    } else {
      for (int i = lane; i < nacc; i += 32) a.partial[(size_t)ch * nacc + i] = (double)C.acc[acc_source(i, k)];
    }
    __syncwarp();
  }
}

// HDM residual norms at many points (the greedy-search indicator, Eq. greedy0):
// rho = 1 on every element, no Jacobians. Work item t = (query q, element chunk c)
// of `chunk` consecutive elements: one warp evaluates R_e on the chunk at query
// q's point (w | tau at wpts + q wstride, parameters at mu + q mustride) and
// writes sum_e |R_e|^2 in FP64 to out[t] (+inf if an element is non-physical).
template <class T, int PROB, int P>
__global__ void __launch_bounds__(128) residual_norms_kernel(AsmArgs<T> a, const double* wpts, long wstride,
                                                             const double* mu, int mustride, int B, int nchunk,
                                                             int chunk, double* out) {
  using Dd = Disc<PROB, P>;
  using Core = ElemCore<T, PROB, P, false>;
  constexpr int NU = Dd::NU, NF = Dd::NFACE;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ku = a.ku, kx = a.kx;
  T *tab, *wT_unused;
  double* tau_unused;
  stage_cta<T, PROB, P>(a, smem, a.w, a.tau, tab, wT_unused, tau_unused);
  const size_t cb = cta_bytes<T, PROB, P>(ku, kx);
  const size_t wb = WarpLayout<T, PROB, P, false>(ku, kx).bytes;
  WarpLayout<T, PROB, P, false> L(ku, kx);
  unsigned char* wbase = smem + cb + warp * wb;
  Core C;
  C.carve(wbase, ku, kx);
  bind_tables(C, tab);
  T* wq = (T*)(wbase + L.owq);
  double* tq = (double*)(wbase + L.otq);
  __syncthreads();
  const long total = (long)B * nchunk;
  for (long t = (long)blockIdx.x * nw + warp; t < total; t += (long)gridDim.x * nw) {
    const int q = (int)(t / nchunk), c = (int)(t - (long)q * nchunk);
    const double* wsrc = wpts + (long)q * wstride;
    for (int i = lane; i < ku; i += 32) wq[i] = (T)wsrc[i];
    for (int i = lane; i < kx; i += 32) tq[i] = wsrc[ku + i];
    __syncwarp();
    const double* muq = mu + (long)q * mustride;
    const long e0 = (long)c * chunk, e1 = (e0 + chunk < a.n_items) ? e0 + chunk : a.n_items;
    double s = 0.0;
    bool bad = false;
    for (long e = e0; e < e1; ++e) {
      signed char bcs[NF];
      bad |= element_front<T, PROB, P, false>(C, a, (int)e, wq, tq, muq, lane, bcs);
      double r2 = 0.0;
      for (int i = lane; i < NU; i += 32) r2 += (double)C.R[i] * (double)C.R[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
      s += r2;
      __syncwarp();
    }
    if (lane == 0) out[t] = bad ? (double)INFINITY : s;
    __syncwarp();
  }
}

// Per-element reduced-residual contributions (the columns of the EQP linear
// program, Eq. eqp-con): for each listed element e, out[e][0..k) = [S^(e); T^(e)]
// with S~ = sum_e rho_e S^(e), T~ = sum_e rho_e T^(e) (Eq. ift-eqp-res0): the
// element's A_e^T R_e plus, in the mesh rows, Psi_e^T dN_e^T N_e. One warp per
// element; out[e][k] = (|R_e|^2 + N_e^2) / 2, the element's share of J~.
template <class T, int PROB, int P>
__global__ void __launch_bounds__(128) element_gradients_kernel(AsmArgs<T> a, double* out) {
  using Dd = Disc<PROB, P>;
  using Core = ElemCore<T, PROB, P, true>;
  constexpr int DIM = Dd::DIM, NU = Dd::NU, NXE = Dd::NXE, NF = Dd::NFACE, NV = Dd::NV;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ku = a.ku, kx = a.kx, k = ku + kx;
  T *tab, *wT;
  double* tauD;
  stage_cta<T, PROB, P>(a, smem, a.w, a.tau, tab, wT, tauD);
  const size_t cb = cta_bytes<T, PROB, P>(ku, kx);
  const size_t wb = WarpLayout<T, PROB, P, true>(ku, kx).bytes;
  Core C;
  C.carve(smem + cb + warp * wb, ku, kx);
  bind_tables(C, tab);
  __syncthreads();
  const bool dist = a.kappa != 0.0;
  for (long it = (long)blockIdx.x * nw + warp; it < a.n_items; it += (long)gridDim.x * nw) {
    const int e = a.elems ? a.elems[it] : (int)it;
    const int* vv = &a.ev[(long)e * NV];
    signed char bcs[NF];
    const bool bad = element_front<T, PROB, P, true>(C, a, e, wT, tauD, a.mu, lane, bcs);
    if (dist && lane == 0) {
      double Xe[NXE];
      for (int r = 0; r < NXE; ++r) Xe[r] = a.X[(size_t)vv[r / DIM] * DIM + (r % DIM)];
      C.distortion_any(Xe, a.kappa, a.eps);
    }
    __syncwarp();
    const T Ne = dist ? (T)C.dN[NXE] : T(0);
    C.jac_state(lane, bcs, ku, k);
    C.jac_geom(lane, a.mu, ku, kx, k, dist);
    double* row = out + (size_t)it * (k + 1);
    for (int r = lane; r < k; r += 32) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < NU; ++i) s += C.A[i * C.ka + r] * C.R[i];
      if (dist && r >= ku) s += C.dNt[r - ku] * Ne;
      row[r] = bad ? (double)NAN : (double)s;
    }
    if (lane == 0) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < NU; ++i) s += C.R[i] * C.R[i];
      row[k] = bad ? (double)INFINITY : 0.5 * (double)(s + Ne * Ne);
    }
    __syncwarp();
  }
}

// norms[q] = sqrt(sum_c part[q * nchunk + c]), summed in chunk order.
__global__ void residual_norms_finish_kernel(const double* part, int B, int nchunk, double* norms);

// Sum of the per-CTA partials: out[i] = sum_c partial[c][i], in a fixed order
// (eight contiguous runs of CTAs, then the eight run sums in order).
__global__ void reduce_partials_kernel(const double* partial, int nparts, int nacc, double* out);

// Per-element inspection: R_e and [dR_e/dU_e | dR_e/dU_e' | dR_e/dx_e], N_e, dN_e
// at a full state (U, x). One warp per listed element; the Jacobian columns are
// the same Jacobian-vector products as in the fused kernel, taken along unit vectors.
template <class T, int PROB, int P>
__global__ void __launch_bounds__(128) inspect_kernel(AsmArgs<T> a, const double* U, const double* x, double* Rout,
                                                      double* Jout, double* Nout, double* dNout) {
  using Dd = Disc<PROB, P>;
  using Core = ElemCore<T, PROB, P, true>;
  constexpr int M = Dd::M, DIM = Dd::DIM, NU = Dd::NU, NUP = Dd::NUP, NXE = Dd::NXE, NF = Dd::NFACE,
                NT = Dd::NTRACE, NV = Dd::NV;
  constexpr int ND = NU + NUP + NXE;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T *tab, *wT;
  double* tauD;
  // ku = ND (state columns), kx = 0: only the layout of the warp buffers is used
  stage_cta<T, PROB, P>(a, smem, a.w, a.tau, tab, wT, tauD);
  const size_t cb = cta_bytes<T, PROB, P>(a.ku, a.kx);
  const size_t wb = WarpLayout<T, PROB, P, true>(a.ku, a.kx).bytes;
  Core C;
  C.carve(smem + cb + warp * wb, a.ku, a.kx);
  bind_tables(C, tab);
  __syncthreads();
  for (long it = (long)blockIdx.x * nw + warp; it < a.n_items; it += (long)gridDim.x * nw) {
    const int e = a.elems[it];
    const int* vv = &a.ev[(long)e * NV];
    for (int i = lane; i < NU; i += 32) C.Ue[i] = (T)U[(size_t)e * NU + i];
    for (int i = lane; i < NUP; i += 32) {
      const int kf = i / (NT * M), rem = i - kf * NT * M, j = rem / M, b = rem - j * M;
      const int e2 = a.nbr[(long)e * NF + kf], k2 = a.nbr_face[(long)e * NF + kf];
      T v = T(0);
      if (e2 >= 0) {
        const int jj = NT - 1 - j;
        const int node = (k2 == 0) ? Dd::face_node(0, jj) : ((k2 == 1) ? Dd::face_node(1, jj) : Dd::face_node(2, jj));
        v = (T)U[(size_t)e2 * NU + node * M + b];
      }
      C.Up[i] = v;
    }
    if (lane < NXE) C.xe[lane] = x[(size_t)vv[lane / DIM] * DIM + (lane % DIM)];
    __syncwarp();
    if constexpr (Dd::CURVED) {
      C.geometry_curved(lane, 32);
      __syncwarp();
    } else {
      C.geometry();
    }
    signed char bcs[NF];
#pragma unroll
    for (int kf = 0; kf < NF; ++kf) bcs[kf] = a.bc[(long)e * NF + kf];
    C.pointwise(lane, bcs, a.mu, a.gamma, true);
    __syncwarp();
    C.residual(lane);
    if (lane == 0) {
      double Xe[NXE];
      for (int r = 0; r < NXE; ++r) Xe[r] = a.X[(size_t)vv[r / DIM] * DIM + (r % DIM)];
      C.distortion_any(Xe, a.kappa, a.eps);
    }
    __syncwarp();
    for (int c = lane; c < ND; c += 32) {
      T dR[NU];
      if (c < NU + NUP) {
        auto fe = [&](int i) { return (c < NU && i == c) ? T(1) : T(0); };
        auto fp = [&](int i) { return (c >= NU && i == c - NU) ? T(1) : T(0); };
        C.jvp_state(fe, fp, bcs, dR);
      } else {
        double dx[NXE];
#pragma unroll
        for (int r = 0; r < NXE; ++r) dx[r] = (r == c - NU - NUP) ? 1.0 : 0.0;
        C.jvp_geom(dx, a.mu, dR);
      }
#pragma unroll
      for (int i = 0; i < NU; ++i) Jout[((size_t)it * NU + i) * ND + c] = (double)dR[i];
    }
    for (int i = lane; i < NU; i += 32) Rout[(size_t)it * NU + i] = (double)C.R[i];
    if (lane < NXE) dNout[(size_t)it * NXE + lane] = C.dN[lane];
    if (lane == 0) Nout[it] = C.dN[NXE];
    __syncwarp();
  }
}

// Snapshot alignment (Eq. align0): the full-space objective (1/2)|F|^2 with
// F = [R(Phi w, x; mu); N(x)] over the state coefficients w and every mesh node x.
// The element pass runs at (w, x) with x in place of the reference nodes (no mesh
// basis), and per element, one warp:
//   MODE 0: F_e = (R_e, N_e) into F (R rows e n_u.., N at n_elems n_u + e), and the
//           number of non-physical elements added to outX[0];
//   MODE 1: J v for v = (dU = Phi dw, dx): dF_e = dR_e/dU_e dU_e + dR_e/dU_e' dU_e'
//           + dR_e/dx_e dx_e, dN_e . dx_e (one lane per product);
//   MODE 2: J^T v: (dR_e/dU_e)^T v_e added to gU's rows of e, (dR_e/dU_e')^T v_e to
//           the neighbours' trace rows, (dR_e/dx_e)^T v_e + dN_e v_N,e to gx's nodes
//           (atomic adds: neighbouring elements share rows and nodes).
// Xref: the reference nodes of the distortion N_e = kappa (eta(x_e) - eta(X_e)).
template <class T, int PROB, int P, int MODE>
__global__ void __launch_bounds__(128) align_kernel(AsmArgs<T> a, const double* Xref, const double* vU,
                                                    const double* vx, const double* vN, double* outU,
                                                    double* outX) {
  using Dd = Disc<PROB, P>;
  // the residual (mode 0) needs no Jacobian data: the objective-only layout and front
  constexpr bool JK = MODE != 0;
  using Core = ElemCore<T, PROB, P, JK>;
  constexpr int M = Dd::M, DIM = Dd::DIM, NU = Dd::NU, NUP = Dd::NUP, NXE = Dd::NXE, NF = Dd::NFACE,
                NV = Dd::NV;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ku = a.ku;
  T *tab, *wT;
  double* tauD;
  stage_cta<T, PROB, P>(a, smem, a.w, a.tau, tab, wT, tauD);
  const size_t cb = cta_bytes<T, PROB, P>(a.ku, a.kx);
  const size_t wb = WarpLayout<T, PROB, P, JK>(a.ku, a.kx).bytes;
  Core C;
  C.carve(smem + cb + warp * wb, a.ku, a.kx);
  bind_tables(C, tab);
  __syncthreads();
  const long Nu = (long)a.n_items * NU;
  for (long e = (long)blockIdx.x * nw + warp; e < a.n_items; e += (long)gridDim.x * nw) {
    const int* vv = &a.ev[e * NV];
    signed char bcs[NF];
    const bool bad = element_front<T, PROB, P, JK>(C, a, (int)e, wT, tauD, a.mu, lane, bcs);
    if (lane == 0) {
      double Xe[NXE];
      for (int r = 0; r < NXE; ++r) Xe[r] = Xref[(size_t)vv[r / DIM] * DIM + (r % DIM)];
      C.distortion_any(Xe, a.kappa, a.eps);  // dN[0..NXE-1], N_e = dN[NXE] (kappa = 0: zero)
    }
    __syncwarp();
    if constexpr (MODE == 0) {
      for (int i = lane; i < NU; i += 32) outU[e * NU + i] = (double)C.R[i];
      if (lane == 0) {
        outU[Nu + e] = C.dN[NXE];
        if (bad && outX) atomicAdd(outX, 1.0);
      }
    } else if constexpr (MODE == 1) {
      // lane 0: the state product, lane 1: the mesh product; summed through W
      T* part = C.W;
      if (lane < 2) {
        T dR[NU];
        if (lane == 0) {
          auto fe = [&](int i) { return (T)vU[e * NU + i]; };
          auto fp = [&](int i) {
            const int kj = i / M, b = i - kj * M;
            const long long off = C.poff[kj];
            return off >= 0 ? (T)vU[off / ku + b] : T(0);
          };
          C.jvp_state(fe, fp, bcs, dR);
        } else {
          double dx[NXE];
          for (int r = 0; r < NXE; ++r) dx[r] = vx[(size_t)vv[r / DIM] * DIM + (r % DIM)];
          C.jvp_geom(dx, a.mu, dR);
        }
#pragma unroll
        for (int i = 0; i < NU; ++i) part[lane * NU + i] = dR[i];
      }
      __syncwarp();
      for (int i = lane; i < NU; i += 32) outU[e * NU + i] = (double)(part[i] + part[NU + i]);
      if (lane == 0) {
        double s = 0.0;
        for (int r = 0; r < NXE; ++r) s += C.dN[r] * vx[(size_t)vv[r / DIM] * DIM + (r % DIM)];
        outU[Nu + e] = s;
      }
    } else {
      // the transposed element Jacobian applied to v_e (v_e replaces R_e)
      for (int i = lane; i < NU; i += 32) C.R[i] = (T)vU[e * NU + i];
      __syncwarp();
      // mesh coordinates first (jvp_geom per unit direction; it reads pointwise data only)
      for (int r = lane; r < NXE; r += 32) {
        double dx[NXE];
        for (int t = 0; t < NXE; ++t) dx[t] = (t == r) ? 1.0 : 0.0;
        T dR[NU];
        C.jvp_geom(dx, a.mu, dR);
        double s = C.dN[r] * vN[e];
#pragma unroll
        for (int i = 0; i < NU; ++i) s += (double)dR[i] * (double)C.R[i];
        atomicAdd(&outX[(size_t)vv[r / DIM] * DIM + (r % DIM)], s);
      }
      __syncwarp();
      T *dUe, *dUp;
      C.adj_state(lane, bcs, dUe, dUp);
      for (int i = lane; i < NU; i += 32) atomicAdd(&outU[e * NU + i], (double)dUe[i]);
      for (int i = lane; i < NUP; i += 32) {
        const int kj = i / M, b = i - kj * M;
        const long long off = C.poff[kj];
        if (off >= 0) atomicAdd(&outU[off / ku + b], (double)dUp[i]);
      }
    }
    __syncwarp();
  }
}

// Snapshot alignment with stored element systems: per element, one warp forms
//   A_e = [dR_e/dU_e Phi_e + dR_e/dU_e' Phi_e' | dR_e/dx_e]   (n_u x k, k = k_u + n_xe),
// the fused assembly's columns with the unit directions of the element's node
// coordinates in place of Psi_e (an identity Psi_e in shared memory), at (w, x) with
// x in place of the reference nodes. The element's share of the Gauss-Newton
// system of (1/2)|F|^2, F = [R; N], is M_e = A_e^T A_e + [0 0; 0 dN_e^T dN_e] and
// g_e = A_e^T R_e + [0; dN_e^T N_e]. The state coefficients w are shared by every
// element, so the w-w blocks enter the products only through their sum
//   H_ww = sum_e (M_e)_ww   (the reduced Gauss-Newton matrix of the state block),
// accumulated per warp and written per CTA (packed upper triangle, acc_h order)
// into hpart[block]; per element the kernel stores
//   (M_e)_wx (k_u x n_xe, row-major) then (M_e)_xx (n_xe x n_xe) into Mout[e]
//   (k_u n_xe + n_xe^2 doubles), g_e into gout[e] (k),
// R_e and N_e into F (as align_kernel mode 0) and the non-physical count into nbad[0].
template <class T, int PROB, int P>
__global__ void __launch_bounds__(128) align_jac_kernel(AsmArgs<T> a, const double* Xref, double* Mout,
                                                        double* gout, double* F, double* nbad, double* hpart) {
  using Dd = Disc<PROB, P>;
  using Core = ElemCore<T, PROB, P, true>;
  using Lay = WarpLayout<T, PROB, P, true>;
  constexpr int DIM = Dd::DIM, NU = Dd::NU, NXE = Dd::NXE, NF = Dd::NFACE, NV = Dd::NV;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ku = a.ku, k = ku + NXE, nh = ku * (ku + 1) / 2, S = ku * NXE + NXE * NXE;
  T *tab, *wT;
  double* tauD;
  stage_cta<T, PROB, P>(a, smem, a.w, a.tau, tab, wT, tauD);
  const size_t cb = cta_bytes<T, PROB, P>(ku, a.kx);
  const Lay L(ku, NXE);
  Core C;
  C.carve(smem + cb + warp * L.bytes, ku, NXE);
  bind_tables(C, tab);
  for (int i = lane; i < NXE * NXE; i += 32) C.Psie[i] = (i / NXE == i % NXE) ? 1.0 : 0.0;
  T* hacc = C.acc;  // this warp's H_ww (nh <= acc_count(k) entries)
  for (int i = lane; i < nh; i += 32) hacc[i] = T(0);
  __syncthreads();
  const long Nu = (long)a.n_items * NU;
  for (long e = (long)blockIdx.x * nw + warp; e < a.n_items; e += (long)gridDim.x * nw) {
    const int* vv = &a.ev[e * NV];
    signed char bcs[NF];
    const bool bad = element_front<T, PROB, P, true>(C, a, (int)e, wT, tauD, a.mu, lane, bcs);
    if (lane == 0) {
      double Xe[NXE];
      for (int r = 0; r < NXE; ++r) Xe[r] = Xref[(size_t)vv[r / DIM] * DIM + (r % DIM)];
      C.distortion_any(Xe, a.kappa, a.eps);
    }
    C.jac_state(lane, bcs, ku, k);
    C.jac_geom(lane, a.mu, ku, NXE, k, false);
    __syncwarp();
    const double Ne = C.dN[NXE];
    double* Me = Mout + (size_t)e * S;
    auto dot = [&](int j, int c) {
      double m = 0.0;
#pragma unroll 8
      for (int i = 0; i < NU; ++i) m += (double)C.A[i * C.ka + j] * (double)C.A[i * C.ka + c];
      return m;
    };
    for (int c = lane; c < k; c += 32) {
      const double dnc = c >= ku ? C.dN[c - ku] : 0.0;
      double gc = dnc * Ne;
      for (int i = 0; i < NU; ++i) gc += (double)C.A[i * C.ka + c] * (double)C.R[i];
      gout[(size_t)e * k + c] = gc;
      if (c < ku) {
        // column c of H_ww (rows j <= c), the row c of (M_e)_wx
        for (int j = 0; j <= c; ++j) hacc[acc_h(j, c, ku)] += (T)dot(j, c);
#pragma unroll
        for (int r = 0; r < NXE; ++r) Me[c * NXE + r] = dot(c, ku + r);
      } else {
        const int r = c - ku;
#pragma unroll
        for (int q = 0; q < NXE; ++q) Me[ku * NXE + q * NXE + r] = dot(ku + q, c) + C.dN[q] * C.dN[r];
      }
    }
    for (int i = lane; i < NU; i += 32) F[e * NU + i] = (double)C.R[i];
    if (lane == 0) {
      F[Nu + e] = Ne;
      if (bad) atomicAdd(nbad, 1.0);
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    double sacc = 0.0;
    for (int wi = 0; wi < nw; ++wi) sacc += (double)((const T*)(smem + cb + wi * L.bytes + L.oacc))[i];
    hpart[(size_t)blockIdx.x * nh + i] = sacc;
  }
}

// Elements per warp group of align_apply_kernel mode 0, and its shared memory in
// doubles: one staging buffer holds the group's (M_e)_wx rows at the odd stride
// nxp = n_xe | 1, its (M_e)_xx, mesh directions and free indices; a warp has two.
__host__ __device__ inline int align_group(int nxe) { return 32 / nxe; }
__host__ __device__ inline int align_apply_buf(int nxe, int ku) {
  const int E = align_group(nxe), nxp = nxe | 1;
  return E * ku * nxp + E * nxe * nxe + E * nxe + (E * nxe + 1) / 2;
}
__host__ __device__ inline int align_apply_warp_doubles(int nxe, int ku) { return 2 * align_apply_buf(nxe, ku); }

// Products with the stored element systems of align_jac_kernel over the unknowns
// (w, free x), J^T J = [H_ww, sum_e (M_e)_wx; sum_e (M_e)_xw, sum_e (M_e)_xx] (the mesh
// blocks at the element's coordinates) and J^T F = sum_e g_e. This kernel forms
// every part but the H_ww terms:
//   MODE 0: for v = (dw, dx), the mesh part given per element in xdir (n_xe values
//           per element, zero on fixed coordinates):
//             w rows  sum_e (M_e)_wx dx_e,
//             mesh rows of element e  (M_e)_xw dw + (M_e)_xx dx_e;
//   MODE 1: y = g_e (w rows and mesh rows);
//   MODE 2: the mesh rows of diag(J^T J): diag((M_e)_xx).
// efree[e][r]: the free index of element e's coordinate r (-1: fixed; its rows are
// dropped); a free coordinate's row goes to its own slot yslot[e][r] (no atomics:
// the free rows are summed from the slots in a fixed order afterwards). MODE 0 takes the elements in groups of E = 32 / n_xe consecutive
// elements per warp (groups strided over the grid), staged in shared memory by
// cp.async, double-buffered: lane (s, r) forms mesh row r of the group's element s
// (k_u + n_xe FMAs), lane c accumulates w row c over the group (E n_xe FMAs), so all
// lanes work on both parts. MODES 1-2: one warp per element, reading their values
// directly. The w rows are summed per CTA into part[block][0..ku) (summed over
// blocks in block order afterwards). k_u <= 96.
template <int NXE, int MODE>
__global__ void __launch_bounds__(256) align_apply_kernel(const double* __restrict__ M,
                                                          const double* __restrict__ g,
                                                          const int* __restrict__ efree,
                                                          const double* __restrict__ xdir, long n_elems, int ku,
                                                          const double* __restrict__ dw, double* part, double* yslot) {
  constexpr int E = 32 / NXE, NXP = NXE | 1;
  extern __shared__ __align__(16) double dsm[];
  __shared__ double sw[96];
  __shared__ double red[8][96];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int k = ku + NXE, S = ku * NXE + NXE * NXE;
  double accw[3] = {0.0, 0.0, 0.0};
  if constexpr (MODE == 0) {
    for (int i = threadIdx.x; i < ku; i += blockDim.x) sw[i] = dw[i];
    __syncthreads();
    const int bufd = align_apply_buf(NXE, ku);
    double* base = dsm + (size_t)warp * align_apply_warp_doubles(NXE, ku);
    // buffer layout: Mwx [E][ku][NXP] | Mxx [E][NXE][NXE] | xd [E][NXE] | free indices [E][NXE]
    auto stage = [&](long e0, int cnt, double* b) {
      const double* src = M + (size_t)e0 * S;
      for (int t = lane; t < cnt * S; t += 32) {
        const int sl = t / S, o = t - sl * S;
        if (o < ku * NXE) {
          const int c = o / NXE, r = o - c * NXE;
          cp_async8(&b[(sl * ku + c) * NXP + r], &src[t]);
        } else {
          cp_async8(&b[E * ku * NXP + sl * NXE * NXE + (o - ku * NXE)], &src[t]);
        }
      }
      double* xd = b + E * ku * NXP + E * NXE * NXE;
      if (lane < cnt * NXE) cp_async8(&xd[lane], &xdir[e0 * NXE + lane]);
      int* fi = (int*)(xd + E * NXE);
      if (lane < cnt * NXE) cp_async4(&fi[lane], &efree[e0 * NXE + lane]);
    };
    const long ngroups = (n_elems + E - 1) / E, stride = (long)gridDim.x * nw;
    long gi = (long)blockIdx.x * nw + warp;
    int cur = 0;
    auto count = [&](long gg) { return (int)min((long)E, n_elems - gg * E); };
    if (gi < ngroups) stage(gi * E, count(gi), base);
    cp_async_commit();
    for (; gi < ngroups; gi += stride) {
      const long gn = gi + stride;
      if (gn < ngroups) stage(gn * E, count(gn), base + (cur ^ 1) * bufd);
      cp_async_commit();
      cp_async_wait_prev();
      __syncwarp();
      const int cnt = count(gi);
      const double* Mwx = base + cur * bufd;
      const double* Mxx = Mwx + E * ku * NXP;
      const double* xd = Mxx + E * NXE * NXE;
      const int* fi = (const int*)(xd + E * NXE);
      // mesh rows: lane (sl, r)
      if (lane < cnt * NXE && fi[lane] >= 0) {
        const int sl = lane / NXE, r = lane - sl * NXE;
        const double* mw = Mwx + sl * ku * NXP + r;
        double y = 0.0;
#pragma unroll 4
        for (int c = 0; c < ku; ++c) y += mw[c * NXP] * sw[c];
        const double* mx = Mxx + sl * NXE * NXE + r;
#pragma unroll
        for (int q = 0; q < NXE; ++q) y += mx[q * NXE] * xd[sl * NXE + q];
        yslot[gi * E * NXE + lane] = y;
      }
      // w rows: lane c over the group's elements
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const int c = ch * 32 + lane;
        if (c < ku) {
          double y = 0.0;
          for (int sl = 0; sl < cnt; ++sl) {
            const double* mw = Mwx + (sl * ku + c) * NXP;
#pragma unroll
            for (int r = 0; r < NXE; ++r) y += mw[r] * xd[sl * NXE + r];
          }
          accw[ch] += y;
        }
      }
      __syncwarp();
      cur ^= 1;
    }
    cp_async_wait_all();
  } else {
    for (long e = (long)blockIdx.x * nw + warp; e < n_elems; e += (long)gridDim.x * nw) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const int c = ch * 32 + lane;
        if (c < k) {
          const int r = c - ku;
          if (r >= 0) {
            const int q = efree[e * NXE + r];
            if (q >= 0)
              yslot[e * NXE + r] = (MODE == 1) ? g[(size_t)e * k + c] : M[(size_t)e * S + ku * NXE + r * NXE + r];
          } else if (MODE == 1) {
            accw[ch] += g[(size_t)e * k + c];
          }
        }
      }
    }
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) red[warp][ch * 32 + lane] = accw[ch];
  __syncthreads();
  for (int c = threadIdx.x; c < ku; c += blockDim.x) {
    double sacc = 0.0;
    for (int wi = 0; wi < nw; ++wi) sacc += red[wi][c];
    part[(size_t)blockIdx.x * ku + c] = sacc;
  }
}

}  // namespace ift
