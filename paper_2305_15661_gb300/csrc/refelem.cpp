#include "refelem.h"

#include <cmath>

namespace ift {

// Golub-Welsch: the Gauss-Legendre points are the eigenvalues of the symmetric
// tridiagonal Jacobi matrix of the Legendre recurrence (off-diagonal
// k / sqrt(4k^2 - 1)); each weight is 2 v_0^2 for the normalised eigenvector v.
// The eigenproblem is solved with cyclic Jacobi rotations (n <= 10 here).
void gauss_legendre_gw(int n, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> A(n * n, 0.0), V(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int k = 1; k < n; ++k) {
    double b = k / std::sqrt(4.0 * k * k - 1.0);
    A[(k - 1) * n + k] = b;
    A[k * n + k - 1] = b;
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-34) break;
    for (int pp = 0; pp < n; ++pp)
      for (int q = pp + 1; q < n; ++q) {
        double apq = A[pp * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (A[q * n + q] - A[pp * n + pp]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A R  (columns p, q)
          double akp = A[k * n + pp], akq = A[k * n + q];
          A[k * n + pp] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- R^T A (rows p, q)
          double apk = A[pp * n + k], aqk = A[q * n + k];
          A[pp * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V R
          double vkp = V[k * n + pp], vkq = V[k * n + q];
          V[k * n + pp] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (A[idx[j] * n + idx[j]] < A[idx[i] * n + idx[i]]) {
        int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
      }
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    int c = idx[i];
    x[i] = A[c * n + c];
    double v0 = V[0 * n + c];
    w[i] = 2.0 * v0 * v0;
  }
  // symmetrise the rule (the Legendre points are symmetric about 0)
  for (int i = 0; i < n / 2; ++i) {
    double xs = 0.5 * (x[n - 1 - i] - x[i]);
    double ws = 0.5 * (w[i] + w[n - 1 - i]);
    x[i] = -xs;
    x[n - 1 - i] = xs;
    w[i] = ws;
    w[n - 1 - i] = ws;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

namespace {

// 1-D Lagrange basis on the equispaced points j/p (p >= 1) and its derivative.
double lag1(int p, int j, double t) {
  double r = 1.0;
  for (int m = 0; m <= p; ++m)
    if (m != j) r *= (t - (double)m / p) / ((double)(j - m) / p);
  return r;
}
double dlag1(int p, int j, double t) {
  double s = 0.0;
  for (int l = 0; l <= p; ++l) {
    if (l == j) continue;
    double r = 1.0 / ((double)(j - l) / p);
    for (int m = 0; m <= p; ++m)
      if (m != j && m != l) r *= (t - (double)m / p) / ((double)(j - m) / p);
    s += r;
  }
  return s;
}

// Silvester's formula: for barycentric multi-index (a1, a2, a3), a1+a2+a3 = p,
// phi = prod_t prod_{q < a_t} (p lambda_t - q) / (q + 1), lambda = (1-r-s, r, s).
// Returns the value and d/dlambda_t for t = 0..2.
void silvester(int p, const int a[3], const double lam[3], double& val, double dl[3]) {
  double f[3], df[3];
  for (int t = 0; t < 3; ++t) {
    double v = 1.0, d = 0.0;
    for (int q = 0; q < a[t]; ++q) {
      double fac = (p * lam[t] - q) / (q + 1.0);
      double dfac = p / (q + 1.0);
      d = d * fac + v * dfac;
      v *= fac;
    }
    f[t] = v;
    df[t] = d;
  }
  val = f[0] * f[1] * f[2];
  dl[0] = df[0] * f[1] * f[2];
  dl[1] = f[0] * df[1] * f[2];
  dl[2] = f[0] * f[1] * df[2];
}

}  // namespace

bool build_tables(int dim, int p, RefTables& t) {
  t.dim = dim;
  t.p = p;
  const int n1d = p + 2;
  std::vector<double> gx, gw;
  gauss_legendre_gw(n1d, gx, gw);
  if (dim == 1) {
    if (p < 0 || p > 6) return false;
    t.nb = p + 1;
    t.nodes.clear();
    for (int j = 0; j <= p; ++j) t.nodes.push_back(p == 0 ? 0.5 : (double)j / p);
    t.nq = n1d;
    t.qxi.resize(n1d);
    t.qw.resize(n1d);
    for (int q = 0; q < n1d; ++q) {
      t.qxi[q] = 0.5 * (1.0 + gx[q]);
      t.qw[q] = 0.5 * gw[q];
    }
    t.B.assign(t.nq * t.nb, 0.0);
    t.D.assign(t.nq * t.nb, 0.0);
    for (int q = 0; q < t.nq; ++q)
      for (int i = 0; i < t.nb; ++i) {
        t.B[q * t.nb + i] = (p == 0) ? 1.0 : lag1(p, i, t.qxi[q]);
        t.D[q * t.nb + i] = t.qw[q] * ((p == 0) ? 0.0 : dlag1(p, i, t.qxi[q]));
      }
    t.nface = 2;
    t.ntrace = 1;
    t.nfq = 1;
    t.ft = {0.0};
    t.fw = {1.0};
    t.Lt = {1.0};
    t.face_nodes = {0, p == 0 ? 0 : p};
  } else if (dim == 2) {
    if (p < 1 || p > 6) return false;
    t.nb = (p + 1) * (p + 2) / 2;
    // barycentric multi-indices in node order
    std::vector<int> mi;
    auto add = [&](int a1, int a2, int a3) {
      mi.push_back(a1);
      mi.push_back(a2);
      mi.push_back(a3);
    };
    add(p, 0, 0);
    add(0, p, 0);
    add(0, 0, p);
    for (int s = 1; s < p; ++s) add(p - s, s, 0);  // edge 0: v0 -> v1
    for (int s = 1; s < p; ++s) add(0, p - s, s);  // edge 1: v1 -> v2
    for (int s = 1; s < p; ++s) add(s, 0, p - s);  // edge 2: v2 -> v0
    for (int j = 1; j < p; ++j)
      for (int i = 1; i + j < p; ++i) add(p - i - j, i, j);
    if ((int)mi.size() != 3 * t.nb) return false;
    t.nodes.resize(t.nb * 2);
    for (int i = 0; i < t.nb; ++i) {
      t.nodes[2 * i] = (double)mi[3 * i + 1] / p;
      t.nodes[2 * i + 1] = (double)mi[3 * i + 2] / p;
    }
    // collapsed Gauss rule: r = (1+a)(1-b)/4, s = (1+b)/2, weight w_a w_b (1-b)/8
    t.nq = n1d * n1d;
    t.qxi.resize(2 * t.nq);
    t.qw.resize(t.nq);
    for (int ib = 0; ib < n1d; ++ib)
      for (int ia = 0; ia < n1d; ++ia) {
        int q = ib * n1d + ia;
        double a = gx[ia], b = gx[ib];
        t.qxi[2 * q] = 0.25 * (1.0 + a) * (1.0 - b);
        t.qxi[2 * q + 1] = 0.5 * (1.0 + b);
        t.qw[q] = gw[ia] * gw[ib] * (1.0 - b) / 8.0;
      }
    t.B.assign(t.nq * t.nb, 0.0);
    t.D.assign(2 * t.nq * t.nb, 0.0);
    for (int q = 0; q < t.nq; ++q) {
      double r = t.qxi[2 * q], s = t.qxi[2 * q + 1];
      double lam[3] = {1.0 - r - s, r, s};
      for (int i = 0; i < t.nb; ++i) {
        double v, dl[3];
        silvester(p, &mi[3 * i], lam, v, dl);
        t.B[q * t.nb + i] = v;
        // d/dr = dphi/dlam1 - dphi/dlam0, d/ds = dphi/dlam2 - dphi/dlam0
        t.D[(0 * t.nq + q) * t.nb + i] = t.qw[q] * (dl[1] - dl[0]);
        t.D[(1 * t.nq + q) * t.nb + i] = t.qw[q] * (dl[2] - dl[0]);
      }
    }
    t.nface = 3;
    t.ntrace = p + 1;
    t.nfq = n1d;
    t.ft.resize(n1d);
    t.fw.resize(n1d);
    for (int f = 0; f < n1d; ++f) {
      t.ft[f] = 0.5 * (1.0 + gx[f]);
      t.fw[f] = 0.5 * gw[f];
    }
    t.Lt.resize(n1d * t.ntrace);
    for (int f = 0; f < n1d; ++f)
      for (int j = 0; j < t.ntrace; ++j) t.Lt[f * t.ntrace + j] = lag1(p, j, t.ft[f]);
    t.face_nodes.assign(3 * t.ntrace, 0);
    for (int k = 0; k < 3; ++k) {
      t.face_nodes[k * t.ntrace + 0] = k;
      for (int s = 1; s < p; ++s) t.face_nodes[k * t.ntrace + s] = 3 + k * (p - 1) + (s - 1);
      t.face_nodes[k * t.ntrace + p] = (k + 1) % 3;
    }
  } else {
    return false;
  }
  t.face_pos.assign(t.nface * t.nb, -1);
  for (int k = 0; k < t.nface; ++k)
    for (int j = 0; j < t.ntrace; ++j) {
      int node = t.face_nodes[k * t.ntrace + j];
      // for p = 0 in 1-D both faces carry the single node
      t.face_pos[k * t.nb + node] = j;
    }
  return true;
}

// Quadratic Lagrange shape functions on the triangle in barycentric form, with
// l0 = 1 - r - s, l1 = r, l2 = s: vertices N_v = l_v (2 l_v - 1), edge midpoints
// N = 4 l_a l_b; their gradients with respect to (r, s).
static void quad_shape_grad(double r, double s, double g[6][2]) {
  const double l0 = 1.0 - r - s, l1 = r, l2 = s;
  g[0][0] = -(4.0 * l0 - 1.0);
  g[0][1] = -(4.0 * l0 - 1.0);
  g[1][0] = 4.0 * l1 - 1.0;
  g[1][1] = 0.0;
  g[2][0] = 0.0;
  g[2][1] = 4.0 * l2 - 1.0;
  g[3][0] = 4.0 * (l0 - l1);  // edge 0-1: 4 l0 l1
  g[3][1] = -4.0 * l1;
  g[4][0] = 4.0 * l2;         // edge 1-2: 4 l1 l2
  g[4][1] = 4.0 * l1;
  g[5][0] = -4.0 * l2;        // edge 2-0: 4 l2 l0
  g[5][1] = 4.0 * (l0 - l2);
}

void build_curved_tables(const RefTables& t, std::vector<double>& gdv, std::vector<double>& gtf) {
  static const double V[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
  gdv.assign((size_t)t.nq * 12, 0.0);
  for (int q = 0; q < t.nq; ++q) {
    double g[6][2];
    quad_shape_grad(t.qxi[2 * q], t.qxi[2 * q + 1], g);
    for (int j = 0; j < 6; ++j)
      for (int c = 0; c < 2; ++c) gdv[(q * 6 + j) * 2 + c] = g[j][c];
  }
  gtf.assign((size_t)3 * t.nfq * 6, 0.0);
  for (int k = 0; k < 3; ++k) {
    const int k1 = (k + 1) % 3;
    const double dv[2] = {V[k1][0] - V[k][0], V[k1][1] - V[k][1]};
    for (int f = 0; f < t.nfq; ++f) {
      const double tt = t.ft[f];
      double g[6][2];
      quad_shape_grad(V[k][0] + tt * dv[0], V[k][1] + tt * dv[1], g);
      for (int j = 0; j < 6; ++j) gtf[(k * t.nfq + f) * 6 + j] = g[j][0] * dv[0] + g[j][1] * dv[1];
    }
  }
}

}  // namespace ift
