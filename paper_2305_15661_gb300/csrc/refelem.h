// Reference-element tables of the nodal DG discretisation (Sec. 2.3).
//
// Nodes: equispaced Lagrange nodes (1-D: [0,1]; triangle: vertices
// (0,0),(1,0),(0,1), then edge-interior nodes edge by edge, edge k running from
// vertex k to vertex k+1, then interior nodes). Quadrature: Gauss-Legendre with
// p+2 points (Golub-Welsch), collapsed Gauss rule on the triangle. The tables are
// built here on the host and copied to the device once per context.
#pragma once
#include <vector>

namespace ift {

struct RefTables {
  int dim = 1, p = 1, nb = 0, nq = 0, nfq = 0, nface = 0, ntrace = 0;
  std::vector<double> nodes;      // nb x dim
  std::vector<double> qxi;        // nq x dim volume points
  std::vector<double> qw;         // nq volume weights (master measure)
  std::vector<double> B;          // nq x nb       phi_i(xi_q)
  std::vector<double> D;          // dim x nq x nb w_q d phi_i / d xi_r (xi_q)
  std::vector<double> ft, fw;     // nfq face parameters in [0,1] and weights (sum 1)
  std::vector<double> Lt;         // nfq x ntrace  ell_j(t_f): trace basis along a face
  std::vector<int> face_nodes;    // nface x ntrace trace nodes in the face's direction
  std::vector<int> face_pos;      // nface x nb: position of node i on face k, or -1
};

// Gauss-Legendre points (ascending) and weights on [-1, 1].
void gauss_legendre_gw(int n, std::vector<double>& x, std::vector<double>& w);

bool build_tables(int dim, int p, RefTables& t);

// Curved (q = 2) triangles: derivatives of the six quadratic geometry shape
// functions N_j (vertices, then the midpoints of edges 0-1, 1-2, 2-0) at the volume
// points of t, gdv[(q * 6 + j) * 2 + c] = dN_j/dxi_c, and along each face k at its
// points, gtf[((k * nfq + f) * 6 + j] = dN_j/dt with xi(t) = V_k + t (V_{k+1} - V_k).
void build_curved_tables(const RefTables& t, std::vector<double>& gdv, std::vector<double>& gtf);

}  // namespace ift
