// FP64 CPU oracle for the EQP-IFT hot path (arXiv 2305.15661).
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow restatement of what the
// paper defines, written to be checked by eye against the equations. Only the
// tests, the smoke check and the CPU-baseline leg of the benchmark may load it.
// It shares no code, header, table or helper with the CUDA library.
//
// What it computes, in the paper's notation:
//   * the transformed conservation law on the reference domain (Sec. 2.2,
//     Eq. p2r-flux): F = g f(U) G^{-T}, S = g s, G = dx/dX, g = det G;
//   * a nodal DG residual of that law, element by element (Sec. 2.3,
//     Eq. hdm_elem): R = sum_e P_e R_e(U_e, U_e', x_e, mu);
//   * the element Jacobians dR_e/dU_e, dR_e/dU_e', dR_e/dx_e by forward-mode
//     dual numbers, one seed direction per evaluation (App. A, Eq. hdm_elem_jac1);
//   * the mesh-distortion residual N_e = kappa (eta_e(x_e) - eta_e(X_e))
//     (Eqs. dist_elem0, dist_elem1);
//   * the weighted reduced residuals S~, T~ (Eq. ift-eqp-res0 with the elemental
//     forms of Eq. ift-res-elem2), the Gauss-Newton blocks of Eq. levmarq-elem and
//     the objective J~ of Eq. ift-opt-eqp2;
//   * the Levenberg-Marquardt iteration of Sec. 3.2.3 (Eqs. levmarq-step, lmstep)
//     with the initialization and stopping test of Remark rem:solver.
//
// The paper leaves the DG weak form, the numerical flux, boundary states, nodes,
// quadrature, the damping rule and the line-search constants open. Each reading
// used here is stated at its point of use below: the weak form above
// element_residual, the Roe flux with Harten's entropy fix above euler_roe and
// burgers_roe, the boundary states in element_residual's face loop, nodes and
// quadrature with the reference element, and the LM constants above lm_phase.
//
// Parity status: every function below is pinned by a CPU test (closed forms,
// conservation, free-stream preservation, equivalence with a physical-space DG
// routine, p-convergence, finite differences, the global-assembly route of App. A).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual number: value and one directional derivative.
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double a) : v(a), d(0.0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) {
  double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }

inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
inline double dsqrt(double a) { return std::sqrt(a); }
inline Dual dsqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline double dexp(double a) { return std::exp(a); }
inline Dual dexp(Dual a) {
  double e = std::exp(a.v);
  return Dual(e, e * a.d);
}
// |a| with d|a|/da = sign(a) and sign(0) = 0.
inline double dabs(double a) { return std::fabs(a); }
inline Dual dabs(Dual a) {
  double s = (a.v > 0.0) ? 1.0 : ((a.v < 0.0) ? -1.0 : 0.0);
  return Dual(std::fabs(a.v), s * a.d);
}
// max(a, eps) with the derivative taken from the a-branch when a >= eps.
inline double dmaxe(double a, double eps) { return a >= eps ? a : eps; }
inline Dual dmaxe(Dual a, double eps) { return a.v >= eps ? a : Dual(eps, 0.0); }

// ---------------------------------------------------------------------------
// Operation counting (work accounting only; never used for results). Cnt is a
// forward-mode dual number that counts the floating-point operations it performs:
// prim counts the value's operations, tan the derivative's. A derivative that is
// structurally zero (it does not depend on the seeded inputs) is tracked by the
// flag z and costs nothing, so the tangent count is what a forward-mode sweep
// along one direction needs. Each +, -, *, / counts one operation (a fused
// multiply-add two), sqrt and exp one each; sign changes, |.|, max and
// comparisons count none.
// ---------------------------------------------------------------------------
struct CntTally {
  long long prim = 0, tan = 0;
};
thread_local CntTally g_cnt;

struct Cnt {
  double v, d;
  bool z;
  Cnt() : v(0.0), d(0.0), z(true) {}
  Cnt(double a) : v(a), d(0.0), z(true) {}
  Cnt(double a, double b, bool zero) : v(a), d(b), z(zero) {}
};
inline Cnt operator+(Cnt a, Cnt b) {
  g_cnt.prim += 1;
  if (!a.z && !b.z) g_cnt.tan += 1;
  return Cnt(a.v + b.v, a.d + b.d, a.z && b.z);
}
inline Cnt operator-(Cnt a, Cnt b) {
  g_cnt.prim += 1;
  if (!a.z && !b.z) g_cnt.tan += 1;
  return Cnt(a.v - b.v, a.d - b.d, a.z && b.z);
}
inline Cnt operator-(Cnt a) { return Cnt(-a.v, -a.d, a.z); }
inline Cnt operator*(Cnt a, Cnt b) {
  g_cnt.prim += 1;
  g_cnt.tan += (!a.z && !b.z) ? 3 : ((!a.z || !b.z) ? 1 : 0);
  return Cnt(a.v * b.v, a.d * b.v + a.v * b.d, a.z && b.z);
}
inline Cnt operator/(Cnt a, Cnt b) {
  g_cnt.prim += 1;
  double q = a.v / b.v;
  g_cnt.tan += (!a.z && !b.z) ? 3 : (!a.z ? 1 : (!b.z ? 2 : 0));
  return Cnt(q, (a.d - q * b.d) / b.v, a.z && b.z);
}
inline Cnt operator+(Cnt a, double b) { g_cnt.prim += 1; return Cnt(a.v + b, a.d, a.z); }
inline Cnt operator+(double a, Cnt b) { g_cnt.prim += 1; return Cnt(a + b.v, b.d, b.z); }
inline Cnt operator-(Cnt a, double b) { g_cnt.prim += 1; return Cnt(a.v - b, a.d, a.z); }
inline Cnt operator-(double a, Cnt b) { g_cnt.prim += 1; return Cnt(a - b.v, -b.d, b.z); }
inline Cnt operator*(Cnt a, double b) {
  g_cnt.prim += 1;
  if (!a.z) g_cnt.tan += 1;
  return Cnt(a.v * b, a.d * b, a.z);
}
inline Cnt operator*(double a, Cnt b) { return b * a; }
inline Cnt operator/(Cnt a, double b) {
  g_cnt.prim += 1;
  if (!a.z) g_cnt.tan += 1;
  return Cnt(a.v / b, a.d / b, a.z);
}
inline Cnt operator/(double a, Cnt b) {
  g_cnt.prim += 1;
  double q = a / b.v;
  if (!b.z) g_cnt.tan += 2;
  return Cnt(q, -q * b.d / b.v, b.z);
}
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { a = a * b; return a; }
inline double val(Cnt a) { return a.v; }
inline Cnt dsqrt(Cnt a) {
  g_cnt.prim += 1;
  double s = std::sqrt(a.v);
  if (!a.z) g_cnt.tan += 2;
  return Cnt(s, a.d / (2.0 * s), a.z);
}
inline Cnt dexp(Cnt a) {
  g_cnt.prim += 1;
  double e = std::exp(a.v);
  if (!a.z) g_cnt.tan += 1;
  return Cnt(e, e * a.d, a.z);
}
inline Cnt dabs(Cnt a) {
  double s = (a.v > 0.0) ? 1.0 : ((a.v < 0.0) ? -1.0 : 0.0);
  return Cnt(std::fabs(a.v), s * a.d, a.z);
}
inline Cnt dmaxe(Cnt a, double eps) { return a.v >= eps ? a : Cnt(eps); }

// Harten's entropy fix of a wave speed: |lam| when |lam| >= delta, else
// (lam^2 + delta^2) / (2 delta), which joins |lam| with a continuous slope.
template <class T>
T harten_abs(const T& lam, const T& delta) {
  T a = dabs(lam);
  if (val(a) >= val(delta)) return a;
  return (lam * lam + delta * delta) / (2.0 * delta);
}

// ---------------------------------------------------------------------------
// Reference element: nodes, Lagrange basis (by Vandermonde inversion in the
// monomial basis), Gauss-Legendre and collapsed (Duffy) quadrature.
// ---------------------------------------------------------------------------

// Gauss-Legendre rule on [-1, 1] with n points, by Newton's method on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p1 = z; p0 = 1.0; }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;  // ascending order
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Dense solve by Gauss-Jordan elimination with partial pivoting; A is n x n
// row-major, B is n x nrhs row-major; on return B holds A^{-1} B.
bool gauss_jordan(int n, std::vector<double> A, std::vector<double>& B, int nrhs) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[piv * n + j]);
      for (int j = 0; j < nrhs; ++j) std::swap(B[c * nrhs + j], B[piv * nrhs + j]);
    }
    double d = A[c * n + c];
    for (int j = 0; j < n; ++j) A[c * n + j] /= d;
    for (int j = 0; j < nrhs; ++j) B[c * nrhs + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
      for (int j = 0; j < nrhs; ++j) B[r * nrhs + j] -= f * B[c * nrhs + j];
    }
  }
  return true;
}

struct RefElem {
  int dim = 1, p = 1, nb = 0, nmono = 0;
  int nface = 0, ntrace = 0;     // faces per element, trace nodes per face
  std::vector<double> nodes;     // nb x dim (master coordinates)
  std::vector<int> mono;         // nmono x dim exponents
  std::vector<double> coef;      // nmono x nb: phi_i = sum_j coef[j*nb+i] * mono_j
  std::vector<double> vq, vw;    // volume rule: nq x dim points, nq weights (master measure)
  std::vector<double> ft, fw;    // face rule: parameter t in [0,1], weights summing to 1
  std::vector<std::vector<int>> face_nodes;  // per face, trace nodes in the face's direction
  std::vector<double> mvert;     // master vertices (dim+1) x dim
  // basis tables at the quadrature points, filled once by tabulate():
  std::vector<double> tv_phi, tv_dphi;   // nq x nb, nq x nb x dim
  std::vector<double> tf_phi;            // nface x nfq x nb at xi(t) on face k
  std::vector<double> tf_phi_rev;        // nface x nfq x nb at xi(1 - t) on face k (neighbour side)
  std::vector<double> tf_xi;             // nface x nfq x dim face points xi(t)

  int nq() const { return (int)vw.size(); }
  int nfq() const { return (int)fw.size(); }

  double mono_val(int j, const double* xi) const {
    double r = 1.0;
    for (int d = 0; d < dim; ++d) r *= std::pow(xi[d], mono[j * dim + d]);
    return r;
  }
  double mono_grad(int j, const double* xi, int dd) const {
    double r = 1.0;
    for (int d = 0; d < dim; ++d) {
      int e = mono[j * dim + d];
      if (d == dd) {
        if (e == 0) return 0.0;
        r *= e * std::pow(xi[d], e - 1);
      } else {
        r *= std::pow(xi[d], e);
      }
    }
    return r;
  }
  double phi(int i, const double* xi) const {
    double s = 0.0;
    for (int j = 0; j < nmono; ++j) s += coef[j * nb + i] * mono_val(j, xi);
    return s;
  }
  double dphi(int i, const double* xi, int d) const {
    double s = 0.0;
    for (int j = 0; j < nmono; ++j) s += coef[j * nb + i] * mono_grad(j, xi, d);
    return s;
  }
};

// Face point xi(t) of face k: in 1-D the end point of the face, in 2-D
// V_k + t (V_{k+1} - V_k) on the master triangle.
void face_point(const RefElem& re, int k, double t, double* xi) {
  if (re.dim == 1) {
    xi[0] = (k == 0) ? 0.0 : 1.0;
  } else {
    int k1 = (k + 1) % 3;
    for (int d = 0; d < 2; ++d) xi[d] = re.mvert[2 * k + d] + t * (re.mvert[2 * k1 + d] - re.mvert[2 * k + d]);
  }
}

void tabulate(RefElem& re) {
  const int nb = re.nb, dim = re.dim, nq = re.nq(), nfq = re.nfq();
  re.tv_phi.assign(nq * nb, 0.0);
  re.tv_dphi.assign(nq * nb * dim, 0.0);
  for (int q = 0; q < nq; ++q)
    for (int i = 0; i < nb; ++i) {
      re.tv_phi[q * nb + i] = re.phi(i, &re.vq[q * dim]);
      for (int d = 0; d < dim; ++d) re.tv_dphi[(q * nb + i) * dim + d] = re.dphi(i, &re.vq[q * dim], d);
    }
  re.tf_phi.assign(re.nface * nfq * nb, 0.0);
  re.tf_phi_rev.assign(re.nface * nfq * nb, 0.0);
  re.tf_xi.assign(re.nface * nfq * dim, 0.0);
  for (int k = 0; k < re.nface; ++k)
    for (int f = 0; f < nfq; ++f) {
      double xi[2], xr[2];
      face_point(re, k, re.ft[f], xi);
      face_point(re, k, 1.0 - re.ft[f], xr);
      for (int d = 0; d < dim; ++d) re.tf_xi[(k * nfq + f) * dim + d] = xi[d];
      for (int i = 0; i < nb; ++i) {
        re.tf_phi[(k * nfq + f) * nb + i] = re.phi(i, xi);
        re.tf_phi_rev[(k * nfq + f) * nb + i] = re.phi(i, xr);
      }
    }
}

bool build_ref(int dim, int p, RefElem& re) {
  re.dim = dim;
  re.p = p;
  re.nodes.clear();
  re.mono.clear();
  if (dim == 1) {
    if (p < 0 || p > 8) return false;
    re.nb = p + 1;
    if (p == 0) {
      re.nodes.push_back(0.5);
    } else {
      for (int j = 0; j <= p; ++j) re.nodes.push_back((double)j / p);
    }
    for (int j = 0; j <= p; ++j) re.mono.push_back(j);
    re.nface = 2;
    re.ntrace = 1;
    re.face_nodes = {{0}, {p == 0 ? 0 : p}};
    re.mvert = {0.0, 1.0};
  } else if (dim == 2) {
    if (p < 1 || p > 6) return false;
    re.nb = (p + 1) * (p + 2) / 2;
    re.mvert = {0.0, 0.0, 1.0, 0.0, 0.0, 1.0};
    // vertices
    for (int k = 0; k < 3; ++k) {
      re.nodes.push_back(re.mvert[2 * k]);
      re.nodes.push_back(re.mvert[2 * k + 1]);
    }
    // edge-interior nodes, edge k from vertex k to vertex k+1
    std::vector<std::vector<int>> edge_int(3);
    for (int k = 0; k < 3; ++k) {
      int k1 = (k + 1) % 3;
      for (int t = 1; t < p; ++t) {
        double s = (double)t / p;
        edge_int[k].push_back((int)re.nodes.size() / 2);
        re.nodes.push_back(re.mvert[2 * k] + s * (re.mvert[2 * k1] - re.mvert[2 * k]));
        re.nodes.push_back(re.mvert[2 * k + 1] + s * (re.mvert[2 * k1 + 1] - re.mvert[2 * k + 1]));
      }
    }
    // interior nodes (i/p, j/p), i, j >= 1, i + j <= p - 1, ordered by j then i
    for (int j = 1; j < p; ++j)
      for (int i = 1; i + j < p; ++i) {
        re.nodes.push_back((double)i / p);
        re.nodes.push_back((double)j / p);
      }
    for (int a = 0; a <= p; ++a)
      for (int b = 0; a + b <= p; ++b) {
        re.mono.push_back(a);
        re.mono.push_back(b);
      }
    re.nface = 3;
    re.ntrace = p + 1;
    re.face_nodes.assign(3, {});
    for (int k = 0; k < 3; ++k) {
      re.face_nodes[k].push_back(k);
      for (int n : edge_int[k]) re.face_nodes[k].push_back(n);
      re.face_nodes[k].push_back((k + 1) % 3);
    }
  } else {
    return false;
  }
  re.nmono = (int)re.mono.size() / dim;
  if (re.nmono != re.nb) return false;
  // Vandermonde V[i][j] = mono_j(node_i); coefficients C = V^{-1}.
  std::vector<double> V(re.nb * re.nb), C(re.nb * re.nb, 0.0);
  for (int i = 0; i < re.nb; ++i)
    for (int j = 0; j < re.nb; ++j) V[i * re.nb + j] = re.mono_val(j, &re.nodes[i * dim]);
  for (int i = 0; i < re.nb; ++i) C[i * re.nb + i] = 1.0;
  if (!gauss_jordan(re.nb, V, C, re.nb)) return false;
  re.coef = C;  // row j of V^{-1} is the mono_j coefficient of every phi_i
  // quadrature: n1d = p + 2 Gauss-Legendre points
  int n1d = p + 2;
  std::vector<double> gx, gw;
  gauss_legendre(n1d, gx, gw);
  re.vq.clear();
  re.vw.clear();
  if (dim == 1) {
    for (int i = 0; i < n1d; ++i) {
      re.vq.push_back(0.5 * (1.0 + gx[i]));
      re.vw.push_back(0.5 * gw[i]);
    }
    re.ft = {0.0};
    re.fw = {1.0};
  } else {
    // collapsed (Duffy) rule: r = (1+a)(1-b)/4, s = (1+b)/2, weight w_a w_b (1-b)/8
    for (int ib = 0; ib < n1d; ++ib)
      for (int ia = 0; ia < n1d; ++ia) {
        double a = gx[ia], b = gx[ib];
        re.vq.push_back(0.25 * (1.0 + a) * (1.0 - b));
        re.vq.push_back(0.5 * (1.0 + b));
        re.vw.push_back(gw[ia] * gw[ib] * (1.0 - b) / 8.0);
      }
    re.ft.clear();
    re.fw.clear();
    for (int i = 0; i < n1d; ++i) {
      re.ft.push_back(0.5 * (1.0 + gx[i]));
      re.fw.push_back(0.5 * gw[i]);
    }
  }
  tabulate(re);
  return true;
}

// ---------------------------------------------------------------------------
// Physics: Burgers (m = 1, d = 1) and compressible Euler (m = 4, d = 2).
// ---------------------------------------------------------------------------
enum { PROB_BURGERS1D = 1, PROB_EULER2D = 2 };
enum { BC_DEFAULT = 0, BC_SHEAR_TEST = 2 };

struct Oracle {
  int problem = 0, dim = 1, m = 1, p = 1;
  int q = 1;                        // geometry degree: 1 straight-sided, 2 curved (2-D)
  RefElem re;
  RefElem geo;                      // q = 2: the six-node quadratic map (vertices, edge midpoints)
  long n_verts = 0, n_elems = 0;
  std::vector<double> X;            // n_verts x dim, reference mesh nodes (all geometry nodes)
  std::vector<int> ev;              // n_elems x nv(): element geometry nodes
  std::vector<int> nbr;             // n_elems x nface: neighbour element or -1
  std::vector<int> nbr_face;        // n_elems x nface: neighbour's local face
  double gamma = 1.4, kappa = 0.0, eps = 1e-8;
  int bc_mode = BC_DEFAULT;
  int nu() const { return re.nb * m; }
  int nup() const { return re.nface * re.ntrace * m; }
  int nv() const { return q == 1 ? dim + 1 : 6; }  // geometry nodes per element
  int nxe() const { return nv() * dim; }
  long Nu() const { return n_elems * (long)nu(); }
  long Nx() const { return n_verts * (long)dim; }
};

// Physical flux f(U) (m x d, row-major [a][r]) and pressure.
template <class T>
void euler_flux(const Oracle& O, const T* U, T* f, T& P) {
  T rho = U[0], u = U[1] / rho, v = U[2] / rho, E = U[3];
  P = (O.gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  f[0] = U[1];
  f[1] = U[2];
  f[2] = U[1] * u + P;
  f[3] = U[1] * v;
  f[4] = U[2] * u;
  f[5] = U[2] * v + P;
  f[6] = u * (E + P);
  f[7] = v * (E + P);
}

// Far-field state U_inf(mu): rho = 1, P = 1, c = sqrt(gamma),
// v = M c (cos a, sin a), mu = (M, a) (Sec. 4.2 free-stream definition).
void euler_freestream(double gamma, const double* mu, double* U) {
  double c = std::sqrt(gamma);
  double M = mu[0], a = mu[1];
  double vx = M * c * std::cos(a), vy = M * c * std::sin(a);
  U[0] = 1.0;
  U[1] = vx;
  U[2] = vy;
  U[3] = 1.0 / (gamma - 1.0) + 0.5 * (vx * vx + vy * vy);
}


inline double dsin(double a) { return std::sin(a); }
inline double dcos(double a) { return std::cos(a); }
inline Dual dsin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
inline Dual dcos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
inline Cnt dsin(Cnt a) {
  g_cnt.prim += 1;
  if (!a.z) g_cnt.tan += 2;
  return Cnt(std::sin(a.v), std::cos(a.v) * a.d, a.z);
}
inline Cnt dcos(Cnt a) {
  g_cnt.prim += 1;
  if (!a.z) g_cnt.tan += 2;
  return Cnt(std::cos(a.v), -std::sin(a.v) * a.d, a.z);
}

// Exact steady parallel shear flow, used only as the boundary state of the
// p-convergence test. With the flow direction d = (cos th, sin th), th = 0.4, and
// the cross-stream coordinate s = -sin(th) x + cos(th) y:
//   rho = 1 + 0.2 sin(2 pi s), velocity = (1.5 + 0.25 cos(2 pi s)) d, P = 1.
// It solves the steady Euler equations: the state is constant along d, the
// velocity is along d, and the pressure is uniform.
template <class T>
void euler_shear_state(double gamma, const T& x, const T& y, T* U) {
  const double tp = 2.0 * 3.14159265358979323846, th = 0.4;
  T s = -std::sin(th) * x + std::cos(th) * y;
  T rho = 1.0 + 0.2 * dsin(tp * s);
  T q = 1.5 + 0.25 * dcos(tp * s);
  U[0] = rho;
  U[1] = rho * q * std::cos(th);
  U[2] = rho * q * std::sin(th);
  U[3] = 1.0 / (gamma - 1.0) + 0.5 * rho * q * q;
}

// Roe flux for the Euler equations with an unnormalised normal nt (|nt| = L):
// H = L [ (F(U+) + F(U-)).n / 2 - |A_roe(n)| (U- - U+) / 2 ], n = nt / L,
// U+ the interior and U- the exterior state.
// |A_roe| dU is written as the sum over the four Roe waves (acoustic waves
// v_n -+ c and the entropy/shear waves at v_n) of |lambda_k| alpha_k r_k, with
// Harten's entropy fix on every |lambda_k| (delta = 0.1 c of the Roe state), so
// that the residual is continuously differentiable where a wave speed vanishes.
template <class T>
void euler_roe(double gamma, const T* Up, const T* Um, const T* nt, T* H) {
  T L = dsqrt(nt[0] * nt[0] + nt[1] * nt[1]);
  T nx = nt[0] / L, ny = nt[1] / L;
  T fp[8], fm[8], Pp, Pm;
  {
    T rho = Up[0], u = Up[1] / rho, v = Up[2] / rho, E = Up[3];
    Pp = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    fp[0] = Up[1]; fp[1] = Up[2];
    fp[2] = Up[1] * u + Pp; fp[3] = Up[1] * v;
    fp[4] = Up[2] * u; fp[5] = Up[2] * v + Pp;
    fp[6] = u * (E + Pp); fp[7] = v * (E + Pp);
  }
  {
    T rho = Um[0], u = Um[1] / rho, v = Um[2] / rho, E = Um[3];
    Pm = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    fm[0] = Um[1]; fm[1] = Um[2];
    fm[2] = Um[1] * u + Pm; fm[3] = Um[1] * v;
    fm[4] = Um[2] * u; fm[5] = Um[2] * v + Pm;
    fm[6] = u * (E + Pm); fm[7] = v * (E + Pm);
  }
  T rL = Up[0], uL = Up[1] / rL, vL = Up[2] / rL, HL = (Up[3] + Pp) / rL;
  T rR = Um[0], uR = Um[1] / rR, vR = Um[2] / rR, HR = (Um[3] + Pm) / rR;
  T sL = dsqrt(rL), sR = dsqrt(rR);
  T ut = (sL * uL + sR * uR) / (sL + sR);
  T vt = (sL * vL + sR * vR) / (sL + sR);
  T Ht = (sL * HL + sR * HR) / (sL + sR);
  T rt = sL * sR;
  T q2 = ut * ut + vt * vt;
  T c2 = (gamma - 1.0) * (Ht - 0.5 * q2);
  T ct = dsqrt(c2);
  T vnt = ut * nx + vt * ny;
  T dr = rR - rL, dP = Pm - Pp, du = uR - uL, dv = vR - vL;
  T dvn = du * nx + dv * ny;
  T a1 = (dP - rt * ct * dvn) / (2.0 * c2);
  T a4 = (dP + rt * ct * dvn) / (2.0 * c2);
  T a2 = dr - dP / c2;
  T del = 0.1 * ct;
  T l1 = harten_abs(vnt - ct, del), l2 = harten_abs(vnt, del), l4 = harten_abs(vnt + ct, del);
  T D[4];
  D[0] = l1 * a1 + l4 * a4 + l2 * a2;
  D[1] = l1 * a1 * (ut - ct * nx) + l4 * a4 * (ut + ct * nx) + l2 * (a2 * ut + rt * (du - dvn * nx));
  D[2] = l1 * a1 * (vt - ct * ny) + l4 * a4 * (vt + ct * ny) + l2 * (a2 * vt + rt * (dv - dvn * ny));
  D[3] = l1 * a1 * (Ht - ct * vnt) + l4 * a4 * (Ht + ct * vnt) +
         l2 * (a2 * (0.5 * q2) + rt * (ut * du + vt * dv - vnt * dvn));
  for (int a = 0; a < 4; ++a) {
    T Fp = fp[2 * a] * nx + fp[2 * a + 1] * ny;
    T Fm = fm[2 * a] * nx + fm[2 * a + 1] * ny;
    H[a] = L * (0.5 * (Fp + Fm) - 0.5 * D[a]);
  }
}

// Roe flux for Burgers, f(u) = u^2/2, with (scalar) normal n:
// H = (f(u+) + f(u-)) n / 2 - |a n| (u- - u+) / 2, a = (u+ + u-) / 2, with
// Harten's entropy fix on |a n| (delta = 0.05 (|u+| + |u-|) |n|).
template <class T>
T burgers_roe(const T& up, const T& um, const T& n) {
  T a = 0.5 * (up + um);
  T del = 0.05 * (dabs(up) + dabs(um)) * dabs(n);
  T aa = (val(del) > 0.0) ? harten_abs(a * n, del) : dabs(a * n);
  return 0.5 * (0.5 * up * up + 0.5 * um * um) * n - 0.5 * aa * (um - up);
}

// Burgers source s(x; mu) = 0.5 exp(mu x).
template <class T>
T burgers_source(const T& x, double mu) { return 0.5 * dexp(mu * x); }

// ---------------------------------------------------------------------------
// Element geometry of the reference-domain formulation.
// JX = dX/dxi (reference mesh element), Jx = dx/dxi (physical element),
// G = dx/dX = Jx JX^{-1}, g = det G (Eq. p2r-stvc). Row-major 2x2 [r][c].
// ---------------------------------------------------------------------------
template <class T>
struct Geom {
  int dim;
  double JX[4], JXinv[4], detJX;
  T Jx[4];
  T G[4], Ginv[4], g;
  double X0[2];
  T x0[2];
};

template <class T>
void element_geometry(const Oracle& O, long e, const T* xe, Geom<T>& gm) {
  int dim = O.dim;
  gm.dim = dim;
  const int* vv = &O.ev[e * (dim + 1)];
  if (dim == 1) {
    gm.X0[0] = O.X[vv[0]];
    gm.x0[0] = xe[0];
    gm.JX[0] = O.X[vv[1]] - O.X[vv[0]];
    gm.detJX = gm.JX[0];
    gm.JXinv[0] = 1.0 / gm.JX[0];
    gm.Jx[0] = xe[1] - xe[0];
    gm.G[0] = gm.Jx[0] * gm.JXinv[0];
    gm.g = gm.G[0];
    gm.Ginv[0] = 1.0 / gm.G[0];
  } else {
    for (int r = 0; r < 2; ++r) {
      gm.X0[r] = O.X[vv[0] * 2 + r];
      gm.x0[r] = xe[r];
      for (int c = 0; c < 2; ++c) {
        gm.JX[r * 2 + c] = O.X[vv[c + 1] * 2 + r] - O.X[vv[0] * 2 + r];
        gm.Jx[r * 2 + c] = xe[(c + 1) * 2 + r] - xe[r];
      }
    }
    gm.detJX = gm.JX[0] * gm.JX[3] - gm.JX[1] * gm.JX[2];
    gm.JXinv[0] = gm.JX[3] / gm.detJX;
    gm.JXinv[1] = -gm.JX[1] / gm.detJX;
    gm.JXinv[2] = -gm.JX[2] / gm.detJX;
    gm.JXinv[3] = gm.JX[0] / gm.detJX;
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 2; ++c) {
        T s = 0.0;
        for (int k = 0; k < 2; ++k) s += gm.Jx[r * 2 + k] * gm.JXinv[k * 2 + c];
        gm.G[r * 2 + c] = s;
      }
    gm.g = gm.G[0] * gm.G[3] - gm.G[1] * gm.G[2];
    gm.Ginv[0] = gm.G[3] / gm.g;
    gm.Ginv[1] = -gm.G[1] / gm.g;
    gm.Ginv[2] = -gm.G[2] / gm.g;
    gm.Ginv[3] = gm.G[0] / gm.g;
  }
}

// Physical point x(xi) = x0 + Jx xi of the affine element map.
template <class T>
void phys_point(const Geom<T>& gm, const double* xi, T* x) {
  if (gm.dim == 1) {
    x[0] = gm.x0[0] + gm.Jx[0] * xi[0];
  } else {
    for (int r = 0; r < 2; ++r) x[r] = gm.x0[r] + gm.Jx[r * 2] * xi[0] + gm.Jx[r * 2 + 1] * xi[1];
  }
}

// Curved (q = 2, 2-D) element geometry at the master point xi. The element map is
// the six-node quadratic Lagrange map x(xi) = sum_j N_j(xi) x_j over the vertices
// and edge midpoints, and likewise X(xi) for the reference mesh, so
// JX = dX/dxi and Jx = dx/dxi vary over the element; G = Jx JX^{-1}, g = det G.
template <class T>
void point_geometry(const Oracle& O, long e, const T* xe, const double* xi, Geom<T>& gm) {
  gm.dim = 2;
  const int* vv = &O.ev[e * 6];
  double dN[6][2];
  for (int j = 0; j < 6; ++j)
    for (int c = 0; c < 2; ++c) dN[j][c] = O.geo.dphi(j, xi, c);
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      double sX = 0.0;
      T sx = 0.0;
      for (int j = 0; j < 6; ++j) {
        sX += O.X[vv[j] * 2 + r] * dN[j][c];
        sx += xe[j * 2 + r] * dN[j][c];
      }
      gm.JX[r * 2 + c] = sX;
      gm.Jx[r * 2 + c] = sx;
    }
  gm.detJX = gm.JX[0] * gm.JX[3] - gm.JX[1] * gm.JX[2];
  gm.JXinv[0] = gm.JX[3] / gm.detJX;
  gm.JXinv[1] = -gm.JX[1] / gm.detJX;
  gm.JXinv[2] = -gm.JX[2] / gm.detJX;
  gm.JXinv[3] = gm.JX[0] / gm.detJX;
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      T s = 0.0;
      for (int k = 0; k < 2; ++k) s += gm.Jx[r * 2 + k] * gm.JXinv[k * 2 + c];
      gm.G[r * 2 + c] = s;
    }
  gm.g = gm.G[0] * gm.G[3] - gm.G[1] * gm.G[2];
  gm.Ginv[0] = gm.G[3] / gm.g;
  gm.Ginv[1] = -gm.G[1] / gm.g;
  gm.Ginv[2] = -gm.G[2] / gm.g;
  gm.Ginv[3] = gm.G[0] / gm.g;
}

// Physical point x(xi) = sum_j N_j(xi) x_j of the curved element map.
template <class T>
void phys_point_q2(const Oracle& O, const T* xe, const double* xi, T* x) {
  for (int r = 0; r < 2; ++r) {
    T s = 0.0;
    for (int j = 0; j < 6; ++j) s += O.geo.phi(j, xi) * xe[j * 2 + r];
    x[r] = s;
  }
}

inline bool bad(double a) { return !std::isfinite(a); }

// Element residual R_e(U_e, U_e', x_e; mu) of the transformed law (Eq. p2r-flux)
// in the DG weak form (the paper says only "nodal DG"; this reading is a steady
// residual without a mass matrix, the flux tested against the gradients of the
// basis functions and the Roe flux on the faces):
//   R_e[i] = - int_{Omega_0e} F(U) . grad_0 v_i dX
//            + int_{dOmega_0e} v_i H(U+, U-; g G^{-T} N) dS_0
//            - int_{Omega_0e} v_i S dX.
// Ue: nb x m; Up: nface x ntrace x m (neighbour trace nodes in the order of
// this element's face direction); xe: (dim+1) x dim vertex coordinates.
template <class T>
void element_residual(const Oracle& O, long e, const T* Ue, const T* Up, const T* xe,
                      const double* mu, T* Re, bool* nonphys) {
  const RefElem& re = O.re;
  const int dim = O.dim, m = O.m, nb = re.nb;
  for (int i = 0; i < nb * m; ++i) Re[i] = T(0.0);
  Geom<T> gm;
  if (O.q == 1) {
    element_geometry(O, e, xe, gm);
    if (!(val(gm.g) > 0.0)) *nonphys = true;
  }
  // volume integral
  for (int q = 0; q < re.nq(); ++q) {
    const double* xi = &re.vq[q * dim];
    const double* phi = &re.tv_phi[q * nb];
    const double* dphi = &re.tv_dphi[q * nb * dim];
    if (O.q == 2) {  // curved: the geometry of this point
      point_geometry(O, e, xe, xi, gm);
      if (!(val(gm.g) > 0.0) || !(gm.detJX > 0.0)) *nonphys = true;
    }
    double dX = gm.detJX * re.vw[q];
    T U[4];
    for (int a = 0; a < m; ++a) {
      T s = 0.0;
      for (int j = 0; j < nb; ++j) s += phi[j] * Ue[j * m + a];
      U[a] = s;
    }
    if (O.problem == PROB_BURGERS1D) {
      T f = 0.5 * U[0] * U[0];
      T F = gm.g * f * gm.Ginv[0];  // g f G^{-T}
      T xq[2];
      phys_point(gm, xi, xq);
      T S = gm.g * burgers_source(xq[0], mu[0]);
      for (int i = 0; i < nb; ++i) {
        double gv = dphi[i] * gm.JXinv[0];  // grad_0 v_i
        Re[i] -= F * gv * dX;
        Re[i] -= phi[i] * S * dX;
      }
    } else {
      T f[8], P;
      euler_flux(O, U, f, P);
      if (!(val(U[0]) > 0.0) || !(val(P) > 0.0)) *nonphys = true;
      // F[a][r] = g sum_s f[a][s] (G^{-T})[s][r],  (G^{-T})[s][r] = Ginv[r][s]
      T F[8];
      for (int a = 0; a < 4; ++a)
        for (int r = 0; r < 2; ++r) {
          T s = 0.0;
          for (int k = 0; k < 2; ++k) s += f[a * 2 + k] * gm.Ginv[r * 2 + k];
          F[a * 2 + r] = gm.g * s;
        }
      for (int i = 0; i < nb; ++i) {
        double gv[2];
        for (int r = 0; r < 2; ++r)
          gv[r] = dphi[i * 2] * gm.JXinv[0 * 2 + r] + dphi[i * 2 + 1] * gm.JXinv[1 * 2 + r];
        for (int a = 0; a < 4; ++a) Re[i * 4 + a] -= (F[a * 2] * gv[0] + F[a * 2 + 1] * gv[1]) * dX;
      }
    }
  }
  // face integrals
  for (int k = 0; k < re.nface; ++k) {
    long e2 = O.nbr[e * re.nface + k];
    int k2 = O.nbr_face[e * re.nface + k];
    for (int fq = 0; fq < re.nfq(); ++fq) {
      const double* xi = &re.tf_xi[(k * re.nfq() + fq) * dim];
      const double* phi = &re.tf_phi[(k * re.nfq() + fq) * nb];
      // the neighbour runs the shared edge the other way: its point is xi(1 - t) on its face k2
      const double* phi2 = (e2 >= 0) ? &re.tf_phi_rev[(k2 * re.nfq() + fq) * nb] : nullptr;
      double N[2], dS0;
      if (dim == 1) {
        N[0] = (k == 0) ? -1.0 : 1.0;
        dS0 = re.fw[fq];
      } else if (O.q == 2) {
        // curved: the reference tangent dX/dt = JX (V_{k+1} - V_k) at this face point
        point_geometry(O, e, xe, xi, gm);
        if (!(val(gm.g) > 0.0) || !(gm.detJX > 0.0)) *nonphys = true;
        int k1 = (k + 1) % 3;
        double dv[2] = {re.mvert[2 * k1] - re.mvert[2 * k], re.mvert[2 * k1 + 1] - re.mvert[2 * k + 1]};
        double E[2] = {gm.JX[0] * dv[0] + gm.JX[1] * dv[1], gm.JX[2] * dv[0] + gm.JX[3] * dv[1]};
        double Ln = std::sqrt(E[0] * E[0] + E[1] * E[1]);
        N[0] = E[1] / Ln;
        N[1] = -E[0] / Ln;
        dS0 = Ln * re.fw[fq];
      } else {
        int k1 = (k + 1) % 3;
        const int* vv = &O.ev[e * 3];
        double E[2] = {O.X[vv[k1] * 2] - O.X[vv[k] * 2], O.X[vv[k1] * 2 + 1] - O.X[vv[k] * 2 + 1]};
        double Ln = std::sqrt(E[0] * E[0] + E[1] * E[1]);
        N[0] = E[1] / Ln;
        N[1] = -E[0] / Ln;
        dS0 = Ln * re.fw[fq];
      }
      // scaled normal g G^{-T} N (Nanson)
      T nt[2];
      for (int r = 0; r < dim; ++r) {
        T s = 0.0;
        for (int k3 = 0; k3 < dim; ++k3) s += gm.Ginv[k3 * dim + r] * N[k3];
        nt[r] = gm.g * s;
      }
      T Uin[4], Uout[4];
      for (int a = 0; a < m; ++a) {
        T s = 0.0;
        for (int j = 0; j < nb; ++j) s += phi[j] * Ue[j * m + a];
        Uin[a] = s;
      }
      if (e2 >= 0) {
        int nt_ = re.ntrace;
        for (int a = 0; a < m; ++a) {
          T s = 0.0;
          for (int j = 0; j < nt_; ++j) {
            int node2 = re.face_nodes[k2][nt_ - 1 - j];
            s += phi2[node2] * Up[(k * nt_ + j) * m + a];
          }
          Uout[a] = s;
        }
      } else if (O.problem == PROB_BURGERS1D) {
        // inflow u = 1 where the outward normal points to -x, outflow u- = u+ elsewhere
        Uout[0] = (N[0] < 0.0) ? T(1.0) : Uin[0];
      } else if (O.bc_mode == BC_SHEAR_TEST) {
        T xp[2] = {T(0.0), T(0.0)};
        if (O.q == 2) phys_point_q2(O, xe, xi, xp);
        else phys_point(gm, xi, xp);
        euler_shear_state(O.gamma, xp[0], xp[1], Uout);
      } else {
        double Uf[4];
        euler_freestream(O.gamma, mu, Uf);
        for (int a = 0; a < 4; ++a) Uout[a] = T(Uf[a]);
      }
      T H[4];
      if (O.problem == PROB_BURGERS1D) {
        H[0] = burgers_roe(Uin[0], Uout[0], nt[0]);
      } else {
        T f1[8], P1, f2[8], P2;
        euler_flux(O, Uin, f1, P1);
        euler_flux(O, Uout, f2, P2);
        if (!(val(Uin[0]) > 0.0) || !(val(P1) > 0.0) || !(val(Uout[0]) > 0.0) || !(val(P2) > 0.0))
          *nonphys = true;
        euler_roe(O.gamma, Uin, Uout, nt, H);
      }
      for (int i = 0; i < nb; ++i)
        for (int a = 0; a < m; ++a) Re[i * m + a] += phi[i] * H[a] * dS0;
    }
  }
  for (int i = 0; i < nb * m; ++i)
    if (bad(val(Re[i]))) *nonphys = true;
}

// Physical-space DG residual of Eq. claw-phys on the straight-sided element with
// vertices xe, written directly with physical gradients, normals and lengths.
// Used only to check that the reference-domain form above reproduces it.
void element_residual_physical(const Oracle& O, long e, const double* Ue, const double* Up,
                               const double* xe, const double* mu, double* Re) {
  const RefElem& re = O.re;
  const int dim = O.dim, m = O.m, nb = re.nb;
  for (int i = 0; i < nb * m; ++i) Re[i] = 0.0;
  double J[4] = {0, 0, 0, 0}, Jinv[4] = {0, 0, 0, 0}, detJ;
  if (dim == 1) {
    J[0] = xe[1] - xe[0];
    detJ = J[0];
    Jinv[0] = 1.0 / J[0];
  } else {
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 2; ++c) J[r * 2 + c] = xe[(c + 1) * 2 + r] - xe[r];
    detJ = J[0] * J[3] - J[1] * J[2];
    Jinv[0] = J[3] / detJ; Jinv[1] = -J[1] / detJ; Jinv[2] = -J[2] / detJ; Jinv[3] = J[0] / detJ;
  }
  for (int q = 0; q < re.nq(); ++q) {
    const double* xi = &re.vq[q * dim];
    double w = std::fabs(detJ) * re.vw[q];
    double U[4] = {0, 0, 0, 0};
    for (int a = 0; a < m; ++a)
      for (int j = 0; j < nb; ++j) U[a] += re.phi(j, xi) * Ue[j * m + a];
    if (dim == 1) {
      double xq = xe[0] + J[0] * xi[0];
      double f = 0.5 * U[0] * U[0], s = 0.5 * std::exp(mu[0] * xq);
      for (int i = 0; i < nb; ++i) Re[i] -= (f * re.dphi(i, xi, 0) * Jinv[0] + re.phi(i, xi) * s) * w;
    } else {
      double f[8], P;
      euler_flux(O, U, f, P);
      for (int i = 0; i < nb; ++i) {
        double gx = re.dphi(i, xi, 0) * Jinv[0] + re.dphi(i, xi, 1) * Jinv[2];
        double gy = re.dphi(i, xi, 0) * Jinv[1] + re.dphi(i, xi, 1) * Jinv[3];
        for (int a = 0; a < 4; ++a) Re[i * 4 + a] -= (f[a * 2] * gx + f[a * 2 + 1] * gy) * w;
      }
    }
  }
  for (int k = 0; k < re.nface; ++k) {
    long e2 = O.nbr[e * re.nface + k];
    int k2 = O.nbr_face[e * re.nface + k];
    for (int fq = 0; fq < re.nfq(); ++fq) {
      double t = re.ft[fq], xi[2], xi2[2] = {0, 0}, n[2], ds;
      if (dim == 1) {
        xi[0] = (k == 0) ? 0.0 : 1.0;
        n[0] = (k == 0) ? -1.0 : 1.0;
        ds = re.fw[fq];
        if (e2 >= 0) xi2[0] = (k2 == 0) ? 0.0 : 1.0;
      } else {
        int k1 = (k + 1) % 3;
        for (int d = 0; d < 2; ++d) xi[d] = re.mvert[2 * k + d] + t * (re.mvert[2 * k1 + d] - re.mvert[2 * k + d]);
        double ed[2] = {xe[k1 * 2] - xe[k * 2], xe[k1 * 2 + 1] - xe[k * 2 + 1]};
        double L = std::sqrt(ed[0] * ed[0] + ed[1] * ed[1]);
        n[0] = ed[1] / L;
        n[1] = -ed[0] / L;
        ds = L * re.fw[fq];
        if (e2 >= 0) {
          int k21 = (k2 + 1) % 3;
          for (int d = 0; d < 2; ++d) xi2[d] = re.mvert[2 * k2 + d] + (1.0 - t) * (re.mvert[2 * k21 + d] - re.mvert[2 * k2 + d]);
        }
      }
      double Uin[4] = {0, 0, 0, 0}, Uout[4] = {0, 0, 0, 0};
      for (int a = 0; a < m; ++a)
        for (int j = 0; j < nb; ++j) Uin[a] += re.phi(j, xi) * Ue[j * m + a];
      if (e2 >= 0) {
        for (int a = 0; a < m; ++a)
          for (int j = 0; j < re.ntrace; ++j)
            Uout[a] += re.phi(re.face_nodes[k2][re.ntrace - 1 - j], xi2) * Up[(k * re.ntrace + j) * m + a];
      } else if (dim == 1) {
        Uout[0] = (n[0] < 0.0) ? 1.0 : Uin[0];
      } else if (O.bc_mode == BC_SHEAR_TEST) {
        double xq = xe[0] + J[0] * xi[0] + J[1] * xi[1];
        double yq = xe[1] + J[2] * xi[0] + J[3] * xi[1];
        euler_shear_state(O.gamma, xq, yq, Uout);
      } else {
        euler_freestream(O.gamma, mu, Uout);
      }
      double H[4];
      if (dim == 1) {
        H[0] = burgers_roe(Uin[0], Uout[0], n[0]);
      } else {
        euler_roe(O.gamma, Uin, Uout, n, H);
      }
      for (int i = 0; i < nb; ++i)
        for (int a = 0; a < m; ++a) Re[i * m + a] += re.phi(i, xi) * H[a] * ds;
    }
  }
}

// Elemental distortion eta_e(x_e) = int_{Omega_0e} (|G|_F^2 / max(g, eps)^{2/d})^2 dX
// (Eq. dist_elem1), integrated with the element's volume rule.
template <class T>
T distortion_eta(const Oracle& O, long e, const T* xe) {
  Geom<T> gm;
  if (O.q == 2) {  // curved: G varies, one geometry per volume point
    T eta = 0.0;
    for (int q = 0; q < O.re.nq(); ++q) {
      point_geometry(O, e, xe, &O.re.vq[q * 2], gm);
      T nrm2 = 0.0;
      for (int i = 0; i < 4; ++i) nrm2 += gm.G[i] * gm.G[i];
      T ratio = nrm2 / dmaxe(gm.g, O.eps);  // max(g, eps)^{2/d}, d = 2
      eta += ratio * ratio * (gm.detJX * O.re.vw[q]);
    }
    return eta;
  }
  element_geometry(O, e, xe, gm);
  T nrm2 = 0.0;
  for (int i = 0; i < O.dim * O.dim; ++i) nrm2 += gm.G[i] * gm.G[i];
  T den = dmaxe(gm.g, O.eps);
  T denp = (O.dim == 1) ? den * den : den;  // max(g, eps)^{2/d}
  T ratio = nrm2 / denp;
  T eta = 0.0;
  for (int q = 0; q < O.re.nq(); ++q) eta += ratio * ratio * (gm.detJX * O.re.vw[q]);
  return eta;
}

// N_e(x_e) = kappa (eta_e(x_e) - eta_e(X_e)) (Eq. dist_elem0).
template <class T>
T distortion_N(const Oracle& O, long e, const T* xe) {
  int nx = O.nxe();
  std::vector<T> Xe(nx);
  const int* vv = &O.ev[e * O.nv()];
  for (int v = 0; v < O.nv(); ++v)
    for (int c = 0; c < O.dim; ++c) Xe[v * O.dim + c] = T(O.X[vv[v] * O.dim + c]);
  return O.kappa * (distortion_eta(O, e, xe) - distortion_eta(O, e, Xe.data()));
}

// Element residual and its Jacobians by forward-mode duals: one seeded
// evaluation per input direction (U_e, then U_e', then x_e).
void element_eval(const Oracle& O, long e, const double* Ue, const double* Up, const double* xe,
                  const double* mu, double* Re, double* JU, double* JUp, double* Jx,
                  double* Ne, double* dNe, bool* nonphys) {
  const int nu = O.nu(), nup = O.nup(), nx = O.nxe();
  bool np = false;
  element_residual<double>(O, e, Ue, Up, xe, mu, Re, &np);
  if (Ne) *Ne = distortion_N<double>(O, e, xe);
  if (JU || JUp || Jx || dNe) {
    std::vector<Dual> dU(nu), dUp(nup), dx(nx), dR(nu);
    for (int i = 0; i < nu; ++i) dU[i] = Dual(Ue[i]);
    for (int i = 0; i < nup; ++i) dUp[i] = Dual(Up[i]);
    for (int i = 0; i < nx; ++i) dx[i] = Dual(xe[i]);
    bool np2 = false;
    if (JU)
      for (int j = 0; j < nu; ++j) {
        dU[j].d = 1.0;
        element_residual<Dual>(O, e, dU.data(), dUp.data(), dx.data(), mu, dR.data(), &np2);
        for (int i = 0; i < nu; ++i) JU[i * nu + j] = dR[i].d;
        dU[j].d = 0.0;
      }
    if (JUp)
      for (int j = 0; j < nup; ++j) {
        dUp[j].d = 1.0;
        element_residual<Dual>(O, e, dU.data(), dUp.data(), dx.data(), mu, dR.data(), &np2);
        for (int i = 0; i < nu; ++i) JUp[i * nup + j] = dR[i].d;
        dUp[j].d = 0.0;
      }
    for (int j = 0; j < nx; ++j) {
      dx[j].d = 1.0;
      if (Jx) {
        element_residual<Dual>(O, e, dU.data(), dUp.data(), dx.data(), mu, dR.data(), &np2);
        for (int i = 0; i < nu; ++i) Jx[i * nx + j] = dR[i].d;
      }
      if (dNe) dNe[j] = distortion_N<Dual>(O, e, dx.data()).d;
      dx[j].d = 0.0;
    }
  }
  if (nonphys) *nonphys = np;
}

// Gather U_e = P_e^T U, U_e' = (P_e')^T U and x_e = Q_e^T x.
void gather(const Oracle& O, const double* U, const double* x, long e, double* Ue, double* Up, double* xe) {
  const RefElem& re = O.re;
  const int nu = O.nu(), m = O.m, nt = re.ntrace;
  if (Ue)
    for (int i = 0; i < nu; ++i) Ue[i] = U[e * nu + i];
  if (Up) {
    for (int k = 0; k < re.nface; ++k) {
      long e2 = O.nbr[e * re.nface + k];
      int k2 = O.nbr_face[e * re.nface + k];
      for (int j = 0; j < nt; ++j)
        for (int a = 0; a < m; ++a) {
          double v = 0.0;
          if (e2 >= 0) v = U[e2 * nu + re.face_nodes[k2][nt - 1 - j] * m + a];
          Up[(k * nt + j) * m + a] = v;
        }
    }
  }
  if (xe) {
    const int* vv = &O.ev[e * O.nv()];
    for (int v = 0; v < O.nv(); ++v)
      for (int c = 0; c < O.dim; ++c) xe[v * O.dim + c] = x[vv[v] * O.dim + c];
  }
}

// Same gather applied to the rows of a basis: rows of Phi for U_e and U_e'
// (zero rows on boundary faces) and rows of Psi for x_e.
void gather_rows(const Oracle& O, int ku, const double* Phi, int kx, const double* Psi, long e,
                 double* Phie, double* Phip, double* Psie) {
  const RefElem& re = O.re;
  const int nu = O.nu(), m = O.m, nt = re.ntrace;
  for (int i = 0; i < nu; ++i)
    for (int c = 0; c < ku; ++c) Phie[i * ku + c] = Phi[(e * nu + i) * (long)ku + c];
  for (int k = 0; k < re.nface; ++k) {
    long e2 = O.nbr[e * re.nface + k];
    int k2 = O.nbr_face[e * re.nface + k];
    for (int j = 0; j < nt; ++j)
      for (int a = 0; a < m; ++a) {
        int row = (k * nt + j) * m + a;
        for (int c = 0; c < ku; ++c) {
          double v = 0.0;
          if (e2 >= 0) v = Phi[(e2 * nu + re.face_nodes[k2][nt - 1 - j] * m + a) * (long)ku + c];
          Phip[row * ku + c] = v;
        }
      }
  }
  const int* vv = &O.ev[e * O.nv()];
  for (int v = 0; v < O.nv(); ++v)
    for (int c = 0; c < O.dim; ++c)
      for (int j = 0; j < kx; ++j) Psie[(v * O.dim + c) * kx + j] = Psi[(vv[v] * (long)O.dim + c) * kx + j];
}

// Per-element weighted contributions of Eqs. ift-eqp-res0, levmarq-elem, ift-opt-eqp2.
struct Contrib {
  std::vector<double> S, T, H;  // ku, kx, k x k
  double J = 0.0;
  bool nonphys = false;
};

void element_reduced(const Oracle& O, int ku, const double* Phi, int kx, const double* Psi, long e,
                     double rho, const double* w, const double* tau, const double* mu, bool with_jac,
                     Contrib& C) {
  const int nu = O.nu(), nup = O.nup(), nx = O.nxe(), k = ku + kx;
  std::vector<double> Phie(nu * ku), Phip(nup * ku), Psie(nx * (kx > 0 ? kx : 1));
  gather_rows(O, ku, Phi, kx, Psi, e, Phie.data(), Phip.data(), Psie.data());
  // U^_e = Phi_e w, U^_e' = Phi_e' w, x^_e = X_e + Psi_e tau
  std::vector<double> Ue(nu, 0.0), Up(nup, 0.0), xe(nx, 0.0);
  for (int i = 0; i < nu; ++i)
    for (int c = 0; c < ku; ++c) Ue[i] += Phie[i * ku + c] * w[c];
  for (int i = 0; i < nup; ++i)
    for (int c = 0; c < ku; ++c) Up[i] += Phip[i * ku + c] * w[c];
  const int* vv = &O.ev[e * O.nv()];
  for (int v = 0; v < O.nv(); ++v)
    for (int c = 0; c < O.dim; ++c) {
      int r = v * O.dim + c;
      double s = O.X[vv[v] * O.dim + c];
      for (int j = 0; j < kx; ++j) s += Psie[r * kx + j] * tau[j];
      xe[r] = s;
    }
  std::vector<double> Re(nu), JU, JUp, Jx, dN(nx, 0.0);
  double Ne = 0.0;
  bool np = false;
  if (with_jac) {
    JU.assign(nu * nu, 0.0);
    JUp.assign(nu * nup, 0.0);
    Jx.assign(nu * nx, 0.0);
    element_eval(O, e, Ue.data(), Up.data(), xe.data(), mu, Re.data(), JU.data(), JUp.data(), Jx.data(),
                 &Ne, dN.data(), &np);
  } else {
    element_eval(O, e, Ue.data(), Up.data(), xe.data(), mu, Re.data(), nullptr, nullptr, nullptr, &Ne,
                 nullptr, &np);
  }
  C.nonphys = np;
  double rr = 0.0;
  for (int i = 0; i < nu; ++i) rr += Re[i] * Re[i];
  C.J = 0.5 * rho * (rr + Ne * Ne);
  if (!with_jac) return;
  // A_w = dR_e/dU_e Phi_e + dR_e/dU_e' Phi_e'  (nu x ku), A_t = dR_e/dx_e Psi_e  (nu x kx)
  std::vector<double> A(nu * k, 0.0), dNt(kx, 0.0);
  for (int i = 0; i < nu; ++i) {
    for (int c = 0; c < ku; ++c) {
      double s = 0.0;
      for (int j = 0; j < nu; ++j) s += JU[i * nu + j] * Phie[j * ku + c];
      for (int j = 0; j < nup; ++j) s += JUp[i * nup + j] * Phip[j * ku + c];
      A[i * k + c] = s;
    }
    for (int c = 0; c < kx; ++c) {
      double s = 0.0;
      for (int j = 0; j < nx; ++j) s += Jx[i * nx + j] * Psie[j * kx + c];
      A[i * k + ku + c] = s;
    }
  }
  for (int c = 0; c < kx; ++c)
    for (int j = 0; j < nx; ++j) dNt[c] += dN[j] * Psie[j * kx + c];
  C.S.assign(ku, 0.0);
  C.T.assign(kx, 0.0);
  C.H.assign(k * k, 0.0);
  for (int c = 0; c < ku; ++c) {
    double s = 0.0;
    for (int i = 0; i < nu; ++i) s += A[i * k + c] * Re[i];
    C.S[c] = rho * s;
  }
  for (int c = 0; c < kx; ++c) {
    double s = 0.0;
    for (int i = 0; i < nu; ++i) s += A[i * k + ku + c] * Re[i];
    C.T[c] = rho * (s + dNt[c] * Ne);
  }
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) {
      double s = 0.0;
      for (int i = 0; i < nu; ++i) s += A[i * k + a] * A[i * k + b];
      if (a >= ku && b >= ku) s += dNt[a - ku] * dNt[b - ku];
      C.H[a * k + b] = rho * s;
    }
}

// Weighted sums over a list of (element, weight) pairs, in list order.
// nnz < 0 means every element with weight 1 (the unweighted ROM, Remark rom-eqp-ones).
int reduced_assemble(const Oracle& O, int ku, const double* Phi, int kx, const double* Psi, long nnz,
                     const int* elems, const double* rho, const double* w, const double* tau,
                     const double* mu, bool with_jac, double* S, double* T, double* H, double* J,
                     int nthreads) {
  const int k = ku + kx;
  long n = (nnz < 0) ? O.n_elems : nnz;
  if (with_jac) {
    for (int c = 0; c < ku; ++c) S[c] = 0.0;
    for (int c = 0; c < kx; ++c) T[c] = 0.0;
    for (int c = 0; c < k * k; ++c) H[c] = 0.0;
  }
  double Jsum = 0.0;
  int n_nonphys = 0;
  const long chunk = 2048;
  std::vector<Contrib> buf(chunk);
  for (long s0 = 0; s0 < n; s0 += chunk) {
    long s1 = (s0 + chunk < n) ? s0 + chunk : n;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (long s = s0; s < s1; ++s) {
      long e = (nnz < 0) ? s : elems[s];
      double r = (nnz < 0) ? 1.0 : rho[s];
      element_reduced(O, ku, Phi, kx, Psi, e, r, w, tau, mu, with_jac, buf[s - s0]);
    }
    for (long s = s0; s < s1; ++s) {
      const Contrib& C = buf[s - s0];
      if (C.nonphys) ++n_nonphys;
      Jsum += C.J;
      if (with_jac) {
        for (int c = 0; c < ku; ++c) S[c] += C.S[c];
        for (int c = 0; c < kx; ++c) T[c] += C.T[c];
        for (int c = 0; c < k * k; ++c) H[c] += C.H[c];
      }
    }
  }
  *J = Jsum;
  return n_nonphys;
}

// Cholesky factorisation A = L L^T in place (lower triangle); false if not SPD.
bool cholesky(int n, std::vector<double>& A) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return false;
    double d = std::sqrt(s);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / d;
    }
  }
  return true;
}

void chol_solve(int n, const std::vector<double>& L, std::vector<double>& b) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * b[k];
    b[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * b[k];
    b[i] = s / L[i * n + i];
  }
}

}  // namespace

namespace {

// Levenberg-Marquardt constants (readings of Sec. 3.2.3, which leaves them open):
// lambda_0 = 1e-4; after a full step lambda <- max(lambda/10, 1e-12), after a
// backtracked step lambda <- min(10 lambda, 1e8); damping on the tau block only
// (Eq. levmarq-step); Armijo backtracking with c1 = 1e-4 and at most 30 halvings;
// a non-physical or non-finite trial counts as J = +inf. The sufficient-decrease
// test carries an allowance of 16 machine epsilons of |J| for rounding in J, so
// that steps whose predicted decrease is below the resolution of J are taken.
const double LM_ROUND_ALLOW = 16.0 * 2.220446049250313e-16;
const double LM_LAMBDA0 = 1e-4, LM_LAMBDA_MIN = 1e-12, LM_LAMBDA_MAX = 1e8;
const double LM_C1 = 1e-4;
const int LM_MAX_HALVINGS = 30;
const int LM_MAX_SHIFTS = 10;

enum { ST_CONVERGED = 0, ST_MAXITER = 1, ST_LINESEARCH = 2, ST_NONPHYS_START = -5 };

struct Problem {
  const Oracle* O;
  int ku, kx;
  const double *Phi, *Psi;
  long nnz;
  const int* elems;
  const double* rho;
  const double* mu;
  int nthreads;
};

struct PhaseStats {
  int iters = 0, trials = 0, shifts = 0, status = 0;
  double g0 = 0.0;
};

// One LM run. full = false optimises w alone with tau frozen (the initialisation
// of Remark rem:solver); full = true optimises (w, tau) jointly.
// trace (may be null) receives one row per accepted step:
// [phase (0 init, 1 joint), lambda used in the step, step length alpha, w (ku), tau (kx)].
void lm_phase(const Problem& P, bool full, double* w, double* tau, double tol, int max_iters,
              PhaseStats& st, std::vector<double>& hist, double* Jout, double* S, double* T,
              std::vector<double>* trace) {
  const int ku = P.ku, kx = P.kx, k = ku + kx;
  const int ka = full ? k : ku;
  std::vector<double> H(k * k);
  double J = 0.0;
  int np = reduced_assemble(*P.O, ku, P.Phi, kx, P.Psi, P.nnz, P.elems, P.rho, w, tau, P.mu, true, S, T,
                            H.data(), &J, P.nthreads);
  hist.push_back(J);
  if (np > 0 || !std::isfinite(J)) {
    st.status = ST_NONPHYS_START;
    *Jout = J;
    return;
  }
  double lam = LM_LAMBDA0;
  auto gnorm = [&]() {
    double s = 0.0;
    for (int c = 0; c < ku; ++c) s += S[c] * S[c];
    if (full)
      for (int c = 0; c < kx; ++c) s += T[c] * T[c];
    return std::sqrt(s);
  };
  st.g0 = gnorm();
  const double thresh = tol * (st.g0 > 1.0 ? st.g0 : 1.0);
  std::vector<double> wt(ku), tt(kx > 0 ? kx : 1);
  for (int it = 0;; ++it) {
    if (gnorm() <= thresh) {
      st.status = ST_CONVERGED;
      break;
    }
    if (it >= max_iters) {
      st.status = ST_MAXITER;
      break;
    }
    // (H + diag(0, lambda I)) dz = -[S; T]   (Eq. lmstep with the damping of Eq. levmarq-step)
    std::vector<double> M(ka * ka), Lf;
    for (int a = 0; a < ka; ++a)
      for (int b = 0; b < ka; ++b) M[a * ka + b] = H[a * k + b];
    if (full)
      for (int a = ku; a < k; ++a) M[a * ka + a] += lam;
    Lf = M;
    if (!cholesky(ka, Lf)) {
      double tr = 0.0;
      for (int a = 0; a < ka; ++a) tr += M[a * ka + a];
      double sh = 1e-14 * tr / ka;
      bool ok = false;
      for (int r = 0; r < LM_MAX_SHIFTS && !ok; ++r, sh *= 10.0) {
        Lf = M;
        for (int a = 0; a < ka; ++a) Lf[a * ka + a] += sh;
        ok = cholesky(ka, Lf);
        ++st.shifts;
      }
      if (!ok) {
        st.status = ST_LINESEARCH;
        break;
      }
    }
    std::vector<double> dz(ka);
    for (int c = 0; c < ku; ++c) dz[c] = -S[c];
    if (full)
      for (int c = 0; c < kx; ++c) dz[ku + c] = -T[c];
    chol_solve(ka, Lf, dz);
    double slope = 0.0;
    for (int c = 0; c < ku; ++c) slope += S[c] * dz[c];
    if (full)
      for (int c = 0; c < kx; ++c) slope += T[c] * dz[ku + c];
    double alpha = 1.0;
    int h = 0;
    bool accepted = false;
    for (h = 0; h <= LM_MAX_HALVINGS; ++h) {
      for (int c = 0; c < ku; ++c) wt[c] = w[c] + alpha * dz[c];
      for (int c = 0; c < kx; ++c) tt[c] = full ? tau[c] + alpha * dz[ku + c] : tau[c];
      double Jt = 0.0;
      int npt = reduced_assemble(*P.O, ku, P.Phi, kx, P.Psi, P.nnz, P.elems, P.rho, wt.data(), tt.data(),
                                 P.mu, false, nullptr, nullptr, nullptr, &Jt, P.nthreads);
      ++st.trials;
      if (npt == 0 && std::isfinite(Jt) && Jt <= J + LM_C1 * alpha * slope + LM_ROUND_ALLOW * std::fabs(J)) {
        accepted = true;
        break;
      }
      alpha *= 0.5;
    }
    if (!accepted) {
      st.status = ST_LINESEARCH;
      break;
    }
    const double lam_used = lam;
    lam = (h == 0) ? std::max(lam / 10.0, LM_LAMBDA_MIN) : std::min(lam * 10.0, LM_LAMBDA_MAX);
    for (int c = 0; c < ku; ++c) w[c] = wt[c];
    for (int c = 0; c < kx; ++c) tau[c] = tt[c];
    if (trace) {
      trace->push_back(full ? 1.0 : 0.0);
      trace->push_back(lam_used);
      trace->push_back(alpha);
      for (int c = 0; c < ku; ++c) trace->push_back(w[c]);
      for (int c = 0; c < kx; ++c) trace->push_back(tau[c]);
    }
    ++st.iters;
    reduced_assemble(*P.O, ku, P.Phi, kx, P.Psi, P.nnz, P.elems, P.rho, w, tau, P.mu, true, S, T, H.data(), &J,
                     P.nthreads);
    hist.push_back(J);
  }
  *Jout = J;
}

bool build_neighbors(Oracle& O) {
  const int nf = O.re.nface;
  O.nbr.assign(O.n_elems * nf, -1);
  O.nbr_face.assign(O.n_elems * nf, -1);
  if (O.dim == 1) {
    // face 0 is the left vertex (local vertex 0), face 1 the right vertex (local vertex 1)
    std::map<int, std::pair<long, int>> seen;
    for (long e = 0; e < O.n_elems; ++e)
      for (int k = 0; k < 2; ++k) {
        int v = O.ev[e * 2 + k];
        auto it = seen.find(v);
        if (it == seen.end()) {
          seen[v] = {e, k};
        } else {
          long e2 = it->second.first;
          int k2 = it->second.second;
          if (O.nbr[e2 * nf + k2] >= 0) return false;
          O.nbr[e * nf + k] = (int)e2;
          O.nbr_face[e * nf + k] = k2;
          O.nbr[e2 * nf + k2] = (int)e;
          O.nbr_face[e2 * nf + k2] = k;
        }
      }
  } else {
    // face k joins local vertices k and k+1; neighbours share the unordered pair
    std::map<std::pair<int, int>, std::pair<long, int>> seen;
    for (long e = 0; e < O.n_elems; ++e)
      for (int k = 0; k < 3; ++k) {
        int a = O.ev[e * O.nv() + k], b = O.ev[e * O.nv() + (k + 1) % 3];
        std::pair<int, int> key(a < b ? a : b, a < b ? b : a);
        auto it = seen.find(key);
        if (it == seen.end()) {
          seen[key] = {e, k};
        } else {
          long e2 = it->second.first;
          int k2 = it->second.second;
          if (O.nbr[e2 * nf + k2] >= 0) return false;
          O.nbr[e * nf + k] = (int)e2;
          O.nbr_face[e * nf + k] = k2;
          O.nbr[e2 * nf + k2] = (int)e;
          O.nbr_face[e2 * nf + k2] = k;
        }
      }
  }
  return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// C interface used by the Python test harness (ctypes).
// ---------------------------------------------------------------------------
extern "C" {

void* orc_create(int problem, int p, long n_verts, const double* X, long n_elems, const int* ev,
                 double gamma, double kappa, double eps, int bc_mode, int q) {
  Oracle* O = new Oracle();
  O->problem = problem;
  O->dim = (problem == PROB_BURGERS1D) ? 1 : 2;
  O->m = (problem == PROB_BURGERS1D) ? 1 : 4;
  O->p = p;
  O->gamma = gamma;
  O->kappa = kappa;
  O->eps = eps;
  O->bc_mode = bc_mode;
  O->q = q;
  if ((problem != PROB_BURGERS1D && problem != PROB_EULER2D) || !build_ref(O->dim, p, O->re) ||
      (q != 1 && q != 2) || (q == 2 && (O->dim != 2 || !build_ref(2, 2, O->geo)))) {
    delete O;
    return nullptr;
  }
  O->n_verts = n_verts;
  O->n_elems = n_elems;
  O->X.assign(X, X + n_verts * O->dim);
  O->ev.assign(ev, ev + n_elems * O->nv());
  if (!build_neighbors(*O)) {
    delete O;
    return nullptr;
  }
  return O;
}

void orc_destroy(void* h) { delete (Oracle*)h; }

// sizes: nb, nu, nup, nxe, nq, nfq, ntrace, nface, N_u, N_x
void orc_sizes(void* h, long* out) {
  Oracle* O = (Oracle*)h;
  out[0] = O->re.nb;
  out[1] = O->nu();
  out[2] = O->nup();
  out[3] = O->nxe();
  out[4] = O->re.nq();
  out[5] = O->re.nfq();
  out[6] = O->re.ntrace;
  out[7] = O->re.nface;
  out[8] = O->Nu();
  out[9] = O->Nx();
}

void orc_neighbors(void* h, int* nbr, int* nbr_face) {
  Oracle* O = (Oracle*)h;
  std::memcpy(nbr, O->nbr.data(), sizeof(int) * O->nbr.size());
  std::memcpy(nbr_face, O->nbr_face.data(), sizeof(int) * O->nbr_face.size());
}

void orc_ref_nodes(void* h, double* nodes, int* face_nodes) {
  Oracle* O = (Oracle*)h;
  std::memcpy(nodes, O->re.nodes.data(), sizeof(double) * O->re.nodes.size());
  for (int k = 0; k < O->re.nface; ++k)
    for (int j = 0; j < O->re.ntrace; ++j) face_nodes[k * O->re.ntrace + j] = O->re.face_nodes[k][j];
}

void orc_ref_quadrature(void* h, double* vq, double* vw, double* ft, double* fw) {
  Oracle* O = (Oracle*)h;
  std::memcpy(vq, O->re.vq.data(), sizeof(double) * O->re.vq.size());
  std::memcpy(vw, O->re.vw.data(), sizeof(double) * O->re.vw.size());
  std::memcpy(ft, O->re.ft.data(), sizeof(double) * O->re.ft.size());
  std::memcpy(fw, O->re.fw.data(), sizeof(double) * O->re.fw.size());
}

void orc_ref_basis(void* h, int npts, const double* xi, double* phi, double* dphi) {
  Oracle* O = (Oracle*)h;
  const int nb = O->re.nb, dim = O->dim;
  for (int q = 0; q < npts; ++q)
    for (int i = 0; i < nb; ++i) {
      phi[q * nb + i] = O->re.phi(i, &xi[q * dim]);
      for (int d = 0; d < dim; ++d) dphi[(q * nb + i) * dim + d] = O->re.dphi(i, &xi[q * dim], d);
    }
}

void orc_gauss_legendre(int n, double* x, double* w) {
  std::vector<double> gx, gw;
  gauss_legendre(n, gx, gw);
  for (int i = 0; i < n; ++i) {
    x[i] = gx[i];
    w[i] = gw[i];
  }
}

void orc_euler_flux(double gamma, const double* U, double* f, double* P) {
  Oracle O;
  O.gamma = gamma;
  euler_flux(O, U, f, *P);
}

void orc_euler_roe(double gamma, const double* Up, const double* Um, const double* n, double* H) {
  euler_roe(gamma, Up, Um, n, H);
}

double orc_burgers_roe(double up, double um, double n) { return burgers_roe(up, um, n); }

void orc_freestream(double gamma, const double* mu, double* U) { euler_freestream(gamma, mu, U); }

// Element residual and Jacobians; JU, JUp, Jx, Ne, dNe may be NULL.
// Returns 1 if the evaluation point is non-physical, else 0.
int orc_element(void* h, long e, const double* Ue, const double* Up, const double* xe, const double* mu,
                double* Re, double* JU, double* JUp, double* Jx, double* Ne, double* dNe) {
  Oracle* O = (Oracle*)h;
  bool np = false;
  element_eval(*O, e, Ue, Up, xe, mu, Re, JU, JUp, Jx, Ne, dNe, &np);
  return np ? 1 : 0;
}

void orc_element_physical(void* h, long e, const double* Ue, const double* Up, const double* xe,
                          const double* mu, double* Re) {
  element_residual_physical(*(Oracle*)h, e, Ue, Up, xe, mu, Re);
}

void orc_gather(void* h, const double* U, const double* x, long e, double* Ue, double* Up, double* xe) {
  gather(*(Oracle*)h, U, x, e, Ue, Up, xe);
}

void orc_gather_rows(void* h, int ku, const double* Phi, int kx, const double* Psi, long e, double* Phie,
                     double* Phip, double* Psie) {
  gather_rows(*(Oracle*)h, ku, Phi, kx, Psi, e, Phie, Phip, Psie);
}

// Global residual R = sum_e P_e R_e (Eq. hdm_elem) and distortion N (Eq. dist_elem0).
int orc_global_residual(void* h, const double* U, const double* x, const double* mu, double* R, double* N) {
  Oracle* O = (Oracle*)h;
  const int nu = O->nu(), nup = O->nup(), nx = O->nxe();
  int bad_count = 0;
  std::vector<double> Ue(nu), Up(nup), xe(nx);
  for (long e = 0; e < O->n_elems; ++e) {
    gather(*O, U, x, e, Ue.data(), Up.data(), xe.data());
    bool np = false;
    double Ne = 0.0;
    element_eval(*O, e, Ue.data(), Up.data(), xe.data(), mu, R + e * nu, nullptr, nullptr, nullptr,
                 N ? &Ne : nullptr, nullptr, &np);
    if (N) N[e] = Ne;
    if (np) ++bad_count;
  }
  return bad_count;
}

// Dense global Jacobians dR/dU (N_u x N_u), dR/dx (N_u x N_x), dN/dx (N_e x N_x),
// assembled from the element Jacobians as in Eqs. hdm_elem_jac1, hdm_elem_jac2.
// For small meshes only (the test harness).
int orc_global_jacobian(void* h, const double* U, const double* x, const double* mu, double* dRdU,
                        double* dRdx, double* dNdx) {
  Oracle* O = (Oracle*)h;
  const RefElem& re = O->re;
  const int nu = O->nu(), nup = O->nup(), nx = O->nxe(), m = O->m, nt = re.ntrace;
  const long Nu = O->Nu(), Nx = O->Nx();
  std::memset(dRdU, 0, sizeof(double) * Nu * Nu);
  std::memset(dRdx, 0, sizeof(double) * Nu * Nx);
  std::memset(dNdx, 0, sizeof(double) * O->n_elems * Nx);
  std::vector<double> Ue(nu), Up(nup), xe(nx), Re(nu), JU(nu * nu), JUp(nu * nup), Jx(nu * nx), dN(nx);
  int bad_count = 0;
  for (long e = 0; e < O->n_elems; ++e) {
    gather(*O, U, x, e, Ue.data(), Up.data(), xe.data());
    bool np = false;
    double Ne = 0.0;
    element_eval(*O, e, Ue.data(), Up.data(), xe.data(), mu, Re.data(), JU.data(), JUp.data(), Jx.data(), &Ne,
                 dN.data(), &np);
    if (np) ++bad_count;
    for (int i = 0; i < nu; ++i) {
      long gi = e * nu + i;
      for (int j = 0; j < nu; ++j) dRdU[gi * Nu + e * nu + j] += JU[i * nu + j];
      for (int k = 0; k < re.nface; ++k) {
        long e2 = O->nbr[e * re.nface + k];
        int k2 = O->nbr_face[e * re.nface + k];
        if (e2 < 0) continue;
        for (int j = 0; j < nt; ++j)
          for (int a = 0; a < m; ++a) {
            long gj = e2 * nu + re.face_nodes[k2][nt - 1 - j] * m + a;
            dRdU[gi * Nu + gj] += JUp[i * nup + (k * nt + j) * m + a];
          }
      }
      const int* vv = &O->ev[e * O->nv()];
      for (int v = 0; v < O->nv(); ++v)
        for (int c = 0; c < O->dim; ++c) dRdx[gi * Nx + vv[v] * O->dim + c] += Jx[i * nx + v * O->dim + c];
    }
    const int* vv = &O->ev[e * O->nv()];
    for (int v = 0; v < O->nv(); ++v)
      for (int c = 0; c < O->dim; ++c) dNdx[e * Nx + vv[v] * O->dim + c] += dN[v * O->dim + c];
  }
  return bad_count;
}

// Weighted reduced quantities S~, T~, H (full symmetric k x k, row-major), J~.
// nnz < 0: all elements with rho = 1. Returns the number of non-physical elements.
int orc_reduced(void* h, int ku, const double* Phi, int kx, const double* Psi, long nnz, const int* elems,
                const double* rho, const double* w, const double* tau, const double* mu, double* S, double* T,
                double* H, double* J, int nthreads) {
  Oracle* O = (Oracle*)h;
  return reduced_assemble(*O, ku, Phi, kx, Psi, nnz, elems, rho, w, tau, mu, true, S, T, H, J, nthreads);
}

// J~ only (residual-only pass). Returns the number of non-physical elements.
int orc_objective(void* h, int ku, const double* Phi, int kx, const double* Psi, long nnz, const int* elems,
                  const double* rho, const double* w, const double* tau, const double* mu, double* J,
                  int nthreads) {
  Oracle* O = (Oracle*)h;
  return reduced_assemble(*O, ku, Phi, kx, Psi, nnz, elems, rho, w, tau, mu, false, nullptr, nullptr, nullptr, J,
                          nthreads);
}

// LM solve (Sec. 3.2.3): optional w-only initialisation (Remark rem:solver) from
// w_guess with tau = tau0, then the joint (w, tau) iteration.
// info[16]: 0 status, 1 init iters, 2 main iters, 3 line-search trials, 4 shifts,
//           5 J, 6 |S|, 7 |T|, 8 |g| at start of main phase, 9 init status.
// hist: J after every accepted step (init then main), at most 2*(max_iters+1) values.
// trace (may be null): rows of lm_phase's trace, at most 2*(max_iters+1) rows of ku+kx+3 values;
// ntrace receives the row count.
int orc_solve(void* h, int ku, const double* Phi, int kx, const double* Psi, long nnz, const int* elems,
              const double* rho, const double* mu, const double* w_guess, const double* tau0, int do_init,
              double tol, int max_iters, double* w, double* tau, double* info, double* hist, int* nhist,
              int nthreads, double* trace, int* ntrace) {
  Oracle* O = (Oracle*)h;
  Problem P{O, ku, kx, Phi, Psi, nnz, elems, rho, mu, nthreads};
  for (int c = 0; c < ku; ++c) w[c] = w_guess[c];
  for (int c = 0; c < kx; ++c) tau[c] = tau0 ? tau0[c] : 0.0;
  std::vector<double> S(ku), T(kx > 0 ? kx : 1), hv, tr;
  std::vector<double>* trp = trace ? &tr : nullptr;
  double J = 0.0;
  PhaseStats s0, s1;
  if (do_init) {
    lm_phase(P, false, w, tau, tol, max_iters, s0, hv, &J, S.data(), T.data(), trp);
    if (s0.status == ST_NONPHYS_START) {
      info[0] = ST_NONPHYS_START;
      *nhist = 0;
      if (ntrace) *ntrace = 0;
      return ST_NONPHYS_START;
    }
  }
  lm_phase(P, true, w, tau, tol, max_iters, s1, hv, &J, S.data(), T.data(), trp);
  double ns = 0.0, nt = 0.0;
  for (int c = 0; c < ku; ++c) ns += S[c] * S[c];
  for (int c = 0; c < kx; ++c) nt += T[c] * T[c];
  info[0] = s1.status;
  info[1] = s0.iters;
  info[2] = s1.iters;
  info[3] = s0.trials + s1.trials;
  info[4] = s0.shifts + s1.shifts;
  info[5] = J;
  info[6] = std::sqrt(ns);
  info[7] = std::sqrt(nt);
  info[8] = s1.g0;
  info[9] = s0.status;
  *nhist = (int)hv.size();
  for (size_t i = 0; i < hv.size(); ++i) hist[i] = hv[i];
  if (trace) {
    for (size_t i = 0; i < tr.size(); ++i) trace[i] = tr[i];
    *ntrace = (int)(tr.size() / (size_t)(ku + kx + 3));
  }
  return s1.status;
}

// Operation counts of the element residual (work accounting, see Cnt): out[0] the
// value's operations of R_e, out[1] the derivative's along the direction seeded by
// dUe, dUp, dxe (each may be NULL: that input's derivative is then structurally
// zero). Returns 1 if the state is non-physical.
int orc_count_element(void* h, long e, const double* Ue, const double* Up, const double* xe, const double* mu,
                      const double* dUe, const double* dUp, const double* dxe, long long* out) {
  Oracle* O = (Oracle*)h;
  const int nu = O->nu(), nup = O->nup(), nx = O->nxe();
  std::vector<Cnt> cU(nu), cUp(nup), cx(nx), cR(nu);
  for (int i = 0; i < nu; ++i) cU[i] = dUe ? Cnt(Ue[i], dUe[i], false) : Cnt(Ue[i]);
  for (int i = 0; i < nup; ++i) cUp[i] = dUp ? Cnt(Up[i], dUp[i], false) : Cnt(Up[i]);
  for (int i = 0; i < nx; ++i) cx[i] = dxe ? Cnt(xe[i], dxe[i], false) : Cnt(xe[i]);
  bool np = false;
  g_cnt = CntTally();
  element_residual<Cnt>(*O, e, cU.data(), cUp.data(), cx.data(), mu, cR.data(), &np);
  out[0] = g_cnt.prim;
  out[1] = g_cnt.tan;
  return np ? 1 : 0;
}

// Operation counts of one pointwise routine at a state (work accounting, see Cnt):
// which = 0 the Euler flux f(U) with U seeded by d; 1 the Euler Roe flux
// H(U+, U-; n) with U+ seeded by d; 2 the Burgers Roe flux with u+ seeded;
// 3 the Euler Roe flux with both U+ and U- seeded by d; 4 the Euler Roe flux with
// U- seeded by d.
// out[0] value operations, out[1] derivative operations.
void orc_count_pointwise(void* h, int which, const double* Up, const double* Um, const double* n, const double* d,
                         long long* out) {
  Oracle* O = (Oracle*)h;
  g_cnt = CntTally();
  if (which == 0) {
    Cnt U[4], f[8], P;
    for (int a = 0; a < 4; ++a) U[a] = Cnt(Up[a], d[a], false);
    euler_flux<Cnt>(*O, U, f, P);
  } else if (which == 1 || which == 3 || which == 4) {
    Cnt a4[4], b4[4], nn[2], H[4];
    for (int a = 0; a < 4; ++a) {
      a4[a] = which != 4 ? Cnt(Up[a], d[a], false) : Cnt(Up[a]);
      b4[a] = which >= 3 ? Cnt(Um[a], d[a], false) : Cnt(Um[a]);
    }
    nn[0] = Cnt(n[0]);
    nn[1] = Cnt(n[1]);
    euler_roe<Cnt>(O->gamma, a4, b4, nn, H);
  } else {
    Cnt up(Up[0], d[0], false), um(Um[0]), nn(n[0]);
    burgers_roe<Cnt>(up, um, nn);
  }
  out[0] = g_cnt.prim;
  out[1] = g_cnt.tan;
}

int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"

extern "C" void orc_shear_state(double gamma, double x, double y, double* U) {
  euler_shear_state(gamma, x, y, U);
}
