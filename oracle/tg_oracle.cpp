// Oracle for finite-element Galerkin assembly on simplex meshes.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg may load this library.  It shares no code,
// header, table or constant with the CUDA library: everything here is
// derived from the method's definition, in FP64, and written to be checked
// by eye against the paper:
//
//   * Local matrices by quadrature, Eq. (matlclquad) of SM A.2 (the concrete
//     form of Eq. (kloc1) and Algorithm 1): geometry J and |det J|, the
//     push-forward G = J^{-T} grad(B^), coefficient at the quadrature points,
//     then the weighted sum over the points.
//   * Global matrix by the classic scatter-add of Eq. (scatter_add),
//     element by element in input order, (a, b) in row-major order, into a
//     dictionary of keys (std::map keyed by (row, col)).  The paper states
//     that its routing-matrix Reduce (Algorithm 2) computes exactly this sum,
//     so this is the reference for the Reduce.
//   * Load vector by the same quadrature (second line of Eq. (matlclquad)).
//   * Vector P1 elasticity from the bilinear form of Hooke's law
//     (SM B.1, Benchmark II): int lambda div u div v + 2 mu eps(u):eps(v).
//   * Gradients of a scalar objective L = sum_s gvals[s] * vals[s] (or the
//     adjoint outer product lambda U^T of Eq. (adj)) with respect to the
//     coefficients and the node coordinates, from the analytic derivative of
//     the quadrature formula (d|det J| = |det J| tr(J^{-1} dJ),
//     dG = -J^{-T} dJ^T G).
//
// Readings where the paper is silent (quadrature rules, P2 basis, reference
// tetrahedron) are the ones the design document lists; every rule and basis
// below is pinned by the test suite (exactness on monomials, reference
// matrices, invariants, finite differences).
//
// Build: g++ -O2 -ffp-contract=off -shared -fPIC (no fast-math).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

namespace {

enum { EL_P1_TRI = 0, EL_P2_TRI = 1, EL_P1_TET = 2, EL_P1_TET_VEC3 = 3 };
enum { LAYOUT_PER_ELEMENT = 0, LAYOUT_PER_QP = 1, LAYOUT_PER_NODE = 2, LAYOUT_CONSTANT = 3 };

struct Rule {
  int nq = 0;
  int dim = 0;
  std::vector<double> w;  // nq
  std::vector<double> x;  // nq * dim reference coordinates
};

// ---------------------------------------------------------------------------
// Quadrature rules on the reference simplex {x_i >= 0, sum x_i <= 1}.

// Triangle, 3 points (1/6,1/6), (2/3,1/6), (1/6,2/3), weights 1/6: degree 2.
Rule rule_tri3() {
  Rule r;
  r.nq = 3;
  r.dim = 2;
  r.w = {1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
  r.x = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  return r;
}

// Triangle, 6 points, degree 4: two symmetric orbits of barycentric points
// (1-2a, a, a) with weight wA each and (1-2b, b, b) with weight wB each.
// Instead of typing a table, the four unknowns are solved from the four
// moment conditions that make a fully symmetric rule exact to degree 4:
// the invariants 1, e2, e3, e2^2 (e2 = l0 l1 + l1 l2 + l2 l0, e3 = l0 l1 l2)
// integrate on the reference triangle to 1/2, 1/8, 1/120, 1/30.
void tri6_residual(const double u[4], double r[4]) {
  const double a = u[0], b = u[1], wA = u[2], wB = u[3];
  const double e2a = 2.0 * a - 3.0 * a * a, e2b = 2.0 * b - 3.0 * b * b;
  const double e3a = (1.0 - 2.0 * a) * a * a, e3b = (1.0 - 2.0 * b) * b * b;
  r[0] = 3.0 * wA + 3.0 * wB - 0.5;
  r[1] = 3.0 * wA * e2a + 3.0 * wB * e2b - 1.0 / 8.0;
  r[2] = 3.0 * wA * e3a + 3.0 * wB * e3b - 1.0 / 120.0;
  r[3] = 3.0 * wA * e2a * e2a + 3.0 * wB * e2b * e2b - 1.0 / 30.0;
}

bool solve4(double A[4][4], double rhs[4], double out[4]) {
  // Gaussian elimination with partial pivoting.
  double M[4][5];
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) M[i][j] = A[i][j];
    M[i][4] = rhs[i];
  }
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int i = c + 1; i < 4; ++i)
      if (std::fabs(M[i][c]) > std::fabs(M[p][c])) p = i;
    if (M[p][c] == 0.0) return false;
    for (int j = 0; j < 5; ++j) std::swap(M[c][j], M[p][j]);
    for (int i = c + 1; i < 4; ++i) {
      const double f = M[i][c] / M[c][c];
      for (int j = c; j < 5; ++j) M[i][j] -= f * M[c][j];
    }
  }
  for (int i = 3; i >= 0; --i) {
    double s = M[i][4];
    for (int j = i + 1; j < 4; ++j) s -= M[i][j] * out[j];
    out[i] = s / M[i][i];
  }
  return true;
}

Rule rule_tri6() {
  double u[4] = {0.45, 0.09, 0.11, 0.055};  // starting guess near the known orbits
  for (int it = 0; it < 60; ++it) {
    double r[4];
    tri6_residual(u, r);
    double J[4][4];
    for (int k = 0; k < 4; ++k) {
      double up[4], um[4], rp[4], rm[4];
      std::memcpy(up, u, sizeof(up));
      std::memcpy(um, u, sizeof(um));
      const double h = 1e-7;
      up[k] += h;
      um[k] -= h;
      tri6_residual(up, rp);
      tri6_residual(um, rm);
      for (int i = 0; i < 4; ++i) J[i][k] = (rp[i] - rm[i]) / (2.0 * h);
    }
    double du[4];
    double neg[4] = {-r[0], -r[1], -r[2], -r[3]};
    if (!solve4(J, neg, du)) break;
    for (int k = 0; k < 4; ++k) u[k] += du[k];
  }
  const double a = u[0], b = u[1], wA = u[2], wB = u[3];
  Rule q;
  q.nq = 6;
  q.dim = 2;
  // (xi, eta) = (l1, l2).  Orbit a first, then orbit b; within an orbit the
  // distinguished barycentric coordinate 1-2a sits at l0, l1, l2 in turn.
  q.x = {a, a, 1.0 - 2.0 * a, a, a, 1.0 - 2.0 * a,
         b, b, 1.0 - 2.0 * b, b, b, 1.0 - 2.0 * b};
  q.w = {wA, wA, wA, wB, wB, wB};
  return q;
}

// Tetrahedron, 4 points, degree 2: barycentric (a, b, b, b) and its
// permutations, a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20, weights 1/24.
// Point q has its large coordinate at barycentric index q (l0 = 1 - sum xi).
Rule rule_tet4() {
  const double s5 = std::sqrt(5.0);
  const double a = (5.0 + 3.0 * s5) / 20.0, b = (5.0 - s5) / 20.0;
  Rule r;
  r.nq = 4;
  r.dim = 3;
  r.w = {1.0 / 24.0, 1.0 / 24.0, 1.0 / 24.0, 1.0 / 24.0};
  r.x = {b, b, b, a, b, b, b, a, b, b, b, a};
  return r;
}

Rule rule_for(int el) {
  switch (el) {
    case EL_P1_TRI: return rule_tri3();
    case EL_P2_TRI: return rule_tri6();
    default: return rule_tet4();
  }
}

int nv_of(int el) { return el == EL_P1_TRI ? 3 : el == EL_P2_TRI ? 6 : 4; }
int dim_of(int el) { return (el == EL_P1_TRI || el == EL_P2_TRI) ? 2 : 3; }

// ---------------------------------------------------------------------------
// Reference basis: values phi[a] and gradients dphi[a*dim + s] at x.
void basis(int el, const double* x, double* phi, double* dphi) {
  if (el == EL_P1_TRI) {
    phi[0] = 1.0 - x[0] - x[1];
    phi[1] = x[0];
    phi[2] = x[1];
    const double g[6] = {-1, -1, 1, 0, 0, 1};
    for (int i = 0; i < 6; ++i) dphi[i] = g[i];
  } else if (el == EL_P2_TRI) {
    const double l0 = 1.0 - x[0] - x[1], l1 = x[0], l2 = x[1];
    const double g0[2] = {-1, -1}, g1[2] = {1, 0}, g2[2] = {0, 1};
    // vertex functions l_i (2 l_i - 1)
    phi[0] = l0 * (2.0 * l0 - 1.0);
    phi[1] = l1 * (2.0 * l1 - 1.0);
    phi[2] = l2 * (2.0 * l2 - 1.0);
    // edge functions 4 l0 l1, 4 l1 l2, 4 l2 l0
    phi[3] = 4.0 * l0 * l1;
    phi[4] = 4.0 * l1 * l2;
    phi[5] = 4.0 * l2 * l0;
    for (int s = 0; s < 2; ++s) {
      dphi[0 * 2 + s] = (4.0 * l0 - 1.0) * g0[s];
      dphi[1 * 2 + s] = (4.0 * l1 - 1.0) * g1[s];
      dphi[2 * 2 + s] = (4.0 * l2 - 1.0) * g2[s];
      dphi[3 * 2 + s] = 4.0 * (l1 * g0[s] + l0 * g1[s]);
      dphi[4 * 2 + s] = 4.0 * (l2 * g1[s] + l1 * g2[s]);
      dphi[5 * 2 + s] = 4.0 * (l0 * g2[s] + l2 * g0[s]);
    }
  } else {
    phi[0] = 1.0 - x[0] - x[1] - x[2];
    phi[1] = x[0];
    phi[2] = x[1];
    phi[3] = x[2];
    const double g[12] = {-1, -1, -1, 1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int i = 0; i < 12; ++i) dphi[i] = g[i];
  }
}

// ---------------------------------------------------------------------------
// Geometry of an affine simplex from its vertex coordinates X[v*dim + r]
// (the first dim+1 nodes): J[r][c] = X[c+1][r] - X[0][r], det by cofactor
// expansion, inverse by the adjugate.
struct Geo {
  int dim;
  double J[3][3];
  double Jinv[3][3];
  double det;
};

Geo geometry(int dim, const double* X) {
  Geo g;
  g.dim = dim;
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c) g.J[r][c] = X[(c + 1) * dim + r] - X[0 * dim + r];
  if (dim == 2) {
    g.det = g.J[0][0] * g.J[1][1] - g.J[0][1] * g.J[1][0];
    g.Jinv[0][0] = g.J[1][1] / g.det;
    g.Jinv[0][1] = -g.J[0][1] / g.det;
    g.Jinv[1][0] = -g.J[1][0] / g.det;
    g.Jinv[1][1] = g.J[0][0] / g.det;
  } else {
    const double(*J)[3] = g.J;
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    g.det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    // adjugate: Jinv[i][j] = cofactor[j][i] / det
    double cof[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        cof[i][j] = J[i1][j1] * J[i2][j2] - J[i1][j2] * J[i2][j1];
      }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) g.Jinv[i][j] = cof[j][i] / g.det;
  }
  return g;
}

// G[r][a] = sum_s Jinv[s][r] * dphi[a][s]   (i.e. J^{-T} grad(phi^_a))
void push_forward(const Geo& g, int nv, const double* dphi, double G[3][6]) {
  for (int r = 0; r < g.dim; ++r)
    for (int a = 0; a < nv; ++a) {
      double s = 0.0;
      for (int t = 0; t < g.dim; ++t) s += g.Jinv[t][r] * dphi[a * g.dim + t];
      G[r][a] = s;
    }
}

double coef_at(const double* v, int layout, int64_t e, int q, int nq) {
  switch (layout) {
    case LAYOUT_PER_QP: return v[e * nq + q];
    case LAYOUT_PER_ELEMENT: return v[e];
    default: return v[0];
  }
}

void gather_X(int dim, int nv, const int32_t* cells, const double* coords, int64_t e, double* X) {
  for (int a = 0; a < nv; ++a)
    for (int r = 0; r < dim; ++r) X[a * dim + r] = coords[(int64_t)cells[e * nv + a] * dim + r];
}

// Local scalar matrix, Eq. (matlclquad) plus the mass term c u v:
// K[a][b] = sum_q w_q |det J| ( kappa_q G_qa . G_qb + c phi_a(x_q) phi_b(x_q) ).
void scalar_local(int el, const Rule& R, const double* X, const double* kq, double c, double* K) {
  const int nv = nv_of(el), dim = dim_of(el);
  const Geo g = geometry(dim, X);
  const double adet = std::fabs(g.det);
  for (int i = 0; i < nv * nv; ++i) K[i] = 0.0;
  for (int q = 0; q < R.nq; ++q) {
    double phi[6], dphi[18], G[3][6];
    basis(el, &R.x[q * dim], phi, dphi);
    push_forward(g, nv, dphi, G);
    for (int a = 0; a < nv; ++a)
      for (int b = 0; b < nv; ++b) {
        double gg = 0.0;
        for (int r = 0; r < dim; ++r) gg += G[r][a] * G[r][b];
        K[a * nv + b] += R.w[q] * adet * (kq[q] * gg + c * phi[a] * phi[b]);
      }
  }
}

// Local elasticity matrix (12 x 12), local DoF index 3*a + i:
// K[(a,i),(b,j)] = sum_q w_q |det J| ( lam_q g_ai g_bj + mu_q g_aj g_bi + mu_q delta_ij g_a . g_b ).
void elastic_local(const Rule& R, const double* X, const double* lq, const double* mq, double* K) {
  const Geo g = geometry(3, X);
  const double adet = std::fabs(g.det);
  for (int i = 0; i < 144; ++i) K[i] = 0.0;
  for (int q = 0; q < R.nq; ++q) {
    double phi[6], dphi[18], G[3][6];
    basis(EL_P1_TET, &R.x[q * 3], phi, dphi);
    push_forward(g, 4, dphi, G);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double gab = 0.0;
        for (int r = 0; r < 3; ++r) gab += G[r][a] * G[r][b];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            const double v = lq[q] * G[i][a] * G[j][b] + mq[q] * G[j][a] * G[i][b] + (i == j ? mq[q] * gab : 0.0);
            K[(3 * a + i) * 12 + (3 * b + j)] += R.w[q] * adet * v;
          }
      }
  }
}

typedef std::map<std::pair<int64_t, int64_t>, double> Dok;

}  // namespace

struct orc_csr {
  int64_t nrows;
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

static orc_csr* freeze(const Dok& dok, int64_t nrows) {
  orc_csr* m = new orc_csr;
  m->nrows = nrows;
  m->row_ptr.assign(nrows + 1, 0);
  m->col.reserve(dok.size());
  m->val.reserve(dok.size());
  for (const auto& kv : dok) {
    m->row_ptr[kv.first.first + 1] += 1;
    m->col.push_back((int32_t)kv.first.second);
    m->val.push_back(kv.second);
  }
  for (int64_t i = 0; i < nrows; ++i) m->row_ptr[i + 1] += m->row_ptr[i];
  return m;
}

extern "C" {

int orc_quadrature(int el, double* w, double* x) {
  const Rule R = rule_for(el);
  for (int q = 0; q < R.nq; ++q) {
    w[q] = R.w[q];
    for (int s = 0; s < R.dim; ++s) x[q * R.dim + s] = R.x[q * R.dim + s];
  }
  return R.nq;
}

void orc_basis(int el, const double* x, double* phi, double* dphi) { basis(el, x, phi, dphi); }

// One scalar element matrix (kq holds the coefficient at each quadrature point).
void orc_element_matrix(int el, const double* X, const double* kq, double c, double* K) {
  scalar_local(el, rule_for(el), X, kq, c, K);
}

void orc_elastic_element_matrix(const double* X, const double* lq, const double* mq, double* K) {
  elastic_local(rule_tet4(), X, lq, mq, K);
}

// Scalar bilinear assembly by scatter-add into a DOK.  row_mask (optional,
// length N) restricts the recorded rows; every element is still evaluated.
orc_csr* orc_assemble_bilinear(int el, int64_t E, int64_t N, const int32_t* cells, const double* coords,
                               const double* kappa, int kappa_layout, double c, const uint8_t* row_mask) {
  const Rule R = rule_for(el);
  const int nv = nv_of(el), dim = dim_of(el);
  Dok dok;
  std::vector<double> X(nv * dim), kq(R.nq), K(nv * nv);
  for (int64_t e = 0; e < E; ++e) {
    gather_X(dim, nv, cells, coords, e, X.data());
    for (int q = 0; q < R.nq; ++q) kq[q] = coef_at(kappa, kappa_layout, e, q, R.nq);
    scalar_local(el, R, X.data(), kq.data(), c, K.data());
    for (int a = 0; a < nv; ++a) {
      const int64_t gi = cells[e * nv + a];
      if (row_mask && !row_mask[gi]) continue;
      for (int b = 0; b < nv; ++b) {
        const int64_t gj = cells[e * nv + b];
        dok[std::make_pair(gi, gj)] += K[a * nv + b];
      }
    }
  }
  return freeze(dok, N);
}

// Vector P1 elasticity; DoF = 3 * node + component.  row_mask is per node.
orc_csr* orc_assemble_elasticity(int64_t E, int64_t N, const int32_t* cells, const double* coords, const double* lam,
                                 const double* mu, int layout, const uint8_t* row_mask) {
  const Rule R = rule_tet4();
  Dok dok;
  double X[12], lq[4], mq[4], K[144];
  for (int64_t e = 0; e < E; ++e) {
    gather_X(3, 4, cells, coords, e, X);
    for (int q = 0; q < 4; ++q) {
      lq[q] = coef_at(lam, layout, e, q, 4);
      mq[q] = coef_at(mu, layout, e, q, 4);
    }
    elastic_local(R, X, lq, mq, K);
    for (int a = 0; a < 4; ++a) {
      const int64_t na = cells[e * 4 + a];
      if (row_mask && !row_mask[na]) continue;
      for (int i = 0; i < 3; ++i)
        for (int b = 0; b < 4; ++b)
          for (int j = 0; j < 3; ++j) {
            const int64_t nb = cells[e * 4 + b];
            dok[std::make_pair(3 * na + i, 3 * nb + j)] += K[(3 * a + i) * 12 + (3 * b + j)];
          }
    }
  }
  return freeze(dok, 3 * N);
}

int64_t orc_csr_nrows(const orc_csr* m) { return m->nrows; }
int64_t orc_csr_nnz(const orc_csr* m) { return (int64_t)m->col.size(); }
void orc_csr_export(const orc_csr* m, int64_t* row_ptr, int32_t* col, double* val) {
  std::memcpy(row_ptr, m->row_ptr.data(), sizeof(int64_t) * (m->nrows + 1));
  std::memcpy(col, m->col.data(), sizeof(int32_t) * m->col.size());
  std::memcpy(val, m->val.data(), sizeof(double) * m->val.size());
}
void orc_csr_free(orc_csr* m) { delete m; }

// Load vector F[g(a)*ncomp + k] += sum_q w_q |det J| f_k(x_q) phi_a(x_q).
// f layouts: PER_QP f[(e*Q + q)*ncomp + k]; PER_NODE f[node*ncomp + k]
// interpolated with the element's own basis; CONSTANT f[k].
void orc_assemble_load(int el, int64_t E, int64_t N, const int32_t* cells, const double* coords, const double* f,
                       int f_layout, int ncomp, double* F) {
  const int gel = (el == EL_P1_TET_VEC3) ? EL_P1_TET : el;
  const Rule R = rule_for(gel);
  const int nv = nv_of(gel), dim = dim_of(gel);
  for (int64_t i = 0; i < N * ncomp; ++i) F[i] = 0.0;
  std::vector<double> X(nv * dim);
  for (int64_t e = 0; e < E; ++e) {
    gather_X(dim, nv, cells, coords, e, X.data());
    const Geo g = geometry(dim, X.data());
    const double adet = std::fabs(g.det);
    for (int q = 0; q < R.nq; ++q) {
      double phi[6], dphi[18];
      basis(gel, &R.x[q * dim], phi, dphi);
      for (int k = 0; k < ncomp; ++k) {
        double fq;
        if (f_layout == LAYOUT_PER_QP) {
          fq = f[(e * R.nq + q) * ncomp + k];
        } else if (f_layout == LAYOUT_PER_NODE) {
          fq = 0.0;
          for (int b = 0; b < nv; ++b) fq += f[(int64_t)cells[e * nv + b] * ncomp + k] * phi[b];
        } else {
          fq = f[k];
        }
        for (int a = 0; a < nv; ++a) F[(int64_t)cells[e * nv + a] * ncomp + k] += R.w[q] * adet * fq * phi[a];
      }
    }
  }
}

// Gradients of L = sum_e sum_ab W^e_ab K^e_ab for the scalar bilinear form.
// W^e_ab = gvals[(g_a, g_b)] looked up in the CSR (g_row_ptr, g_col) when
// gvals is given, else lam[g_a] * U[g_b] (the adjoint outer product).
// grad_kappa has kappa's layout (NULL to skip); grad_coords is [N][dim];
// grad_c a single value.  All outputs are overwritten.
int orc_assemble_backward(int el, int64_t E, int64_t N, const int32_t* cells, const double* coords,
                          const double* kappa, int kappa_layout, double c, const int64_t* g_row_ptr,
                          const int32_t* g_col, const double* gvals, const double* lam, const double* U,
                          double* grad_kappa, double* grad_coords, double* grad_c) {
  const Rule R = rule_for(el);
  const int nv = nv_of(el), dim = dim_of(el);
  if (grad_kappa) {
    const int64_t n = kappa_layout == LAYOUT_PER_QP ? E * R.nq : kappa_layout == LAYOUT_PER_ELEMENT ? E : 1;
    for (int64_t i = 0; i < n; ++i) grad_kappa[i] = 0.0;
  }
  if (grad_coords)
    for (int64_t i = 0; i < N * dim; ++i) grad_coords[i] = 0.0;
  double gc = 0.0;
  std::vector<double> X(nv * dim), W(nv * nv);
  for (int64_t e = 0; e < E; ++e) {
    gather_X(dim, nv, cells, coords, e, X.data());
    for (int a = 0; a < nv; ++a)
      for (int b = 0; b < nv; ++b) {
        const int64_t ga = cells[e * nv + a], gb = cells[e * nv + b];
        double w = 0.0;
        if (gvals) {
          for (int64_t s = g_row_ptr[ga]; s < g_row_ptr[ga + 1]; ++s)
            if (g_col[s] == gb) w = gvals[s];
        } else {
          w = lam[ga] * U[gb];
        }
        W[a * nv + b] = w;
      }
    const Geo g = geometry(dim, X.data());
    const double adet = std::fabs(g.det);
    double dLdJ_pre[3][3] = {{0}};  // accumulates the bracket before the J^{-T} factor
    for (int q = 0; q < R.nq; ++q) {
      double phi[6], dphi[18], G[3][6];
      basis(el, &R.x[q * dim], phi, dphi);
      push_forward(g, nv, dphi, G);
      const double kq = coef_at(kappa, kappa_layout, e, q, R.nq);
      // P_q = G W_s G^T, with W_s the symmetric part of W
      double P[3][3] = {{0}};
      for (int r = 0; r < dim; ++r)
        for (int s = 0; s < dim; ++s) {
          double v = 0.0;
          for (int a = 0; a < nv; ++a)
            for (int b = 0; b < nv; ++b)
              v += G[r][a] * 0.5 * (W[a * nv + b] + W[b * nv + a]) * G[s][b];
          P[r][s] = v;
        }
      double trP = 0.0;
      for (int r = 0; r < dim; ++r) trP += P[r][r];
      double wm = 0.0;  // W : (phi phi^T)
      for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) wm += W[a * nv + b] * phi[a] * phi[b];
      if (grad_kappa) {
        const double v = R.w[q] * adet * trP;
        if (kappa_layout == LAYOUT_PER_QP) grad_kappa[e * R.nq + q] += v;
        else if (kappa_layout == LAYOUT_PER_ELEMENT) grad_kappa[e] += v;
        else grad_kappa[0] += v;
      }
      gc += R.w[q] * adet * wm;
      const double alpha = R.w[q] * adet * kq;
      for (int r = 0; r < dim; ++r)
        for (int s = 0; s < dim; ++s)
          dLdJ_pre[r][s] += alpha * ((r == s ? trP : 0.0) - 2.0 * P[r][s]) + (r == s ? R.w[q] * adet * c * wm : 0.0);
    }
    if (grad_coords) {
      // dL/dJ = pre * J^{-T};  column j of dL/dJ belongs to vertex j+1, vertex 0 gets minus the sum.
      double dJ[3][3];
      for (int r = 0; r < dim; ++r)
        for (int s = 0; s < dim; ++s) {
          double v = 0.0;
          for (int t = 0; t < dim; ++t) v += dLdJ_pre[r][t] * g.Jinv[s][t];
          dJ[r][s] = v;
        }
      for (int j = 0; j < dim; ++j)
        for (int r = 0; r < dim; ++r) {
          grad_coords[(int64_t)cells[e * nv + j + 1] * dim + r] += dJ[r][j];
          grad_coords[(int64_t)cells[e * nv + 0] * dim + r] -= dJ[r][j];
        }
    }
  }
  if (grad_c) *grad_c = gc;
  return 0;
}

// Gradients of L = sum_i sum_k gF[i*ncomp + k] F[i*ncomp + k] for the load
// vector: grad_f (layout of f) and grad_coords [N][dim] (overwritten).  F
// depends on the coordinates through |det J| only: dL/dJ = L_e J^{-T}.
int orc_load_backward(int el, int64_t E, int64_t N, const int32_t* cells, const double* coords, const double* f,
                      int f_layout, int ncomp, const double* gF, double* grad_f, double* grad_coords) {
  const int gel = (el == EL_P1_TET_VEC3) ? EL_P1_TET : el;
  const Rule R = rule_for(gel);
  const int nv = nv_of(gel), dim = dim_of(gel);
  const int64_t nf = f_layout == LAYOUT_PER_QP ? E * R.nq * ncomp : f_layout == LAYOUT_PER_NODE ? N * ncomp : ncomp;
  if (grad_f)
    for (int64_t i = 0; i < nf; ++i) grad_f[i] = 0.0;
  if (grad_coords)
    for (int64_t i = 0; i < N * dim; ++i) grad_coords[i] = 0.0;
  std::vector<double> X(nv * dim);
  for (int64_t e = 0; e < E; ++e) {
    gather_X(dim, nv, cells, coords, e, X.data());
    const Geo g = geometry(dim, X.data());
    const double adet = std::fabs(g.det);
    double Le = 0.0;
    for (int q = 0; q < R.nq; ++q) {
      double phi[6], dphi[18];
      basis(gel, &R.x[q * dim], phi, dphi);
      for (int k = 0; k < ncomp; ++k) {
        // s = sum_a gF[g_a, k] phi_a(x_q): the weight of f_k(x_q) in L
        double s = 0.0;
        for (int a = 0; a < nv; ++a) s += gF[(int64_t)cells[e * nv + a] * ncomp + k] * phi[a];
        double fq;
        if (f_layout == LAYOUT_PER_QP) {
          fq = f[(e * R.nq + q) * ncomp + k];
          if (grad_f) grad_f[(e * R.nq + q) * ncomp + k] += R.w[q] * adet * s;
        } else if (f_layout == LAYOUT_PER_NODE) {
          fq = 0.0;
          for (int b = 0; b < nv; ++b) {
            fq += f[(int64_t)cells[e * nv + b] * ncomp + k] * phi[b];
            if (grad_f) grad_f[(int64_t)cells[e * nv + b] * ncomp + k] += R.w[q] * adet * s * phi[b];
          }
        } else {
          fq = f[k];
          if (grad_f) grad_f[k] += R.w[q] * adet * s;
        }
        Le += R.w[q] * adet * fq * s;
      }
    }
    if (grad_coords) {
      for (int j = 0; j < dim; ++j)
        for (int r = 0; r < dim; ++r) {
          const double v = Le * g.Jinv[j][r];  // (L_e J^{-T})[r][j]
          grad_coords[(int64_t)cells[e * nv + j + 1] * dim + r] += v;
          grad_coords[(int64_t)cells[e * nv + 0] * dim + r] -= v;
        }
    }
  }
  return 0;
}

// Gradients of L = sum_e sum W^e K^e for vector P1 elasticity with respect to
// lambda, mu (layout PER_ELEMENT or PER_QP) and the coordinates.  W^e is
// looked up in (g_row_ptr, g_col, gvals) at DoF level, or lam_adj[ga] U[gb].
// Uses dL/dJ = (L_e I - G Gamma^T) J^{-T}, Gamma = dL_e/dG at fixed |det J|.
int orc_elasticity_backward(int64_t E, int64_t N, const int32_t* cells, const double* coords, const double* lam,
                            const double* mu, int layout, const int64_t* g_row_ptr, const int32_t* g_col,
                            const double* gvals, const double* lam_adj, const double* U, double* grad_lam,
                            double* grad_mu, double* grad_coords) {
  const Rule R = rule_tet4();
  const int64_t nc = layout == LAYOUT_PER_QP ? E * 4 : E;
  for (int64_t i = 0; i < nc; ++i) {
    if (grad_lam) grad_lam[i] = 0.0;
    if (grad_mu) grad_mu[i] = 0.0;
  }
  if (grad_coords)
    for (int64_t i = 0; i < N * 3; ++i) grad_coords[i] = 0.0;
  double X[12], W[144];
  for (int64_t e = 0; e < E; ++e) {
    gather_X(3, 4, cells, coords, e, X);
    for (int A = 0; A < 12; ++A)
      for (int B = 0; B < 12; ++B) {
        const int64_t gA = 3 * (int64_t)cells[e * 4 + A / 3] + A % 3;
        const int64_t gB = 3 * (int64_t)cells[e * 4 + B / 3] + B % 3;
        double w = 0.0;
        if (gvals) {
          for (int64_t s = g_row_ptr[gA]; s < g_row_ptr[gA + 1]; ++s)
            if (g_col[s] == gB) w = gvals[s];
        } else {
          w = lam_adj[gA] * U[gB];
        }
        W[A * 12 + B] = w;
      }
    const Geo g = geometry(3, X);
    const double adet = std::fabs(g.det);
    double phi[6], dphi[18], G[3][6];
    basis(EL_P1_TET, &R.x[0], phi, dphi);  // P1 gradients do not depend on the point
    push_forward(g, 4, dphi, G);
    // T1 = sum W_{ai,bj} g_ai g_bj, T2 = sum W_{ai,bj} g_aj g_bi, T3 = sum_{ab} (sum_i W_{ai,bi}) g_a.g_b
    double T1 = 0, T2 = 0, T3 = 0;
    double dT1[3][4] = {{0}}, dT2[3][4] = {{0}}, dT3[3][4] = {{0}};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            const double w = W[(3 * a + i) * 12 + 3 * b + j];
            T1 += w * G[i][a] * G[j][b];
            T2 += w * G[j][a] * G[i][b];
            dT1[i][a] += w * G[j][b];
            dT1[j][b] += w * G[i][a];
            dT2[j][a] += w * G[i][b];
            dT2[i][b] += w * G[j][a];
            if (i == j) {
              for (int r = 0; r < 3; ++r) {
                T3 += w * G[r][a] * G[r][b];
                dT3[r][a] += w * G[r][b];
                dT3[r][b] += w * G[r][a];
              }
            }
          }
    double sl = 0.0, sm = 0.0;  // sum_q w_q lam_q, sum_q w_q mu_q
    for (int q = 0; q < 4; ++q) {
      const double lq = coef_at(lam, layout, e, q, 4), mq = coef_at(mu, layout, e, q, 4);
      sl += R.w[q] * lq;
      sm += R.w[q] * mq;
      const int64_t idx = layout == LAYOUT_PER_QP ? e * 4 + q : e;
      if (grad_lam) grad_lam[idx] += R.w[q] * adet * T1;
      if (grad_mu) grad_mu[idx] += R.w[q] * adet * (T2 + T3);
    }
    if (grad_coords) {
      const double Le = adet * (sl * T1 + sm * (T2 + T3));
      double Gam[3][4];
      for (int r = 0; r < 3; ++r)
        for (int a = 0; a < 4; ++a) Gam[r][a] = adet * (sl * dT1[r][a] + sm * (dT2[r][a] + dT3[r][a]));
      double pre[3][3];
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) {
          double v = 0.0;
          for (int a = 0; a < 4; ++a) v += G[r][a] * Gam[s][a];
          pre[r][s] = (r == s ? Le : 0.0) - v;
        }
      for (int j = 0; j < 3; ++j)
        for (int r = 0; r < 3; ++r) {
          double v = 0.0;
          for (int t = 0; t < 3; ++t) v += pre[r][t] * g.Jinv[j][t];
          grad_coords[(int64_t)cells[e * 4 + j + 1] * 3 + r] += v;
          grad_coords[(int64_t)cells[e * 4 + 0] * 3 + r] -= v;
        }
    }
  }
  return 0;
}

}  // extern "C"
