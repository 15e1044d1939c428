// Oracle for finite element assembly: a plain, slow, obviously correct CPU
// implementation in FP64.  TEST INFRASTRUCTURE ONLY: the product library never
// links, loads or calls this file, and this file shares no code, header,
// table or constant with the CUDA path.
//
// What it computes (Sec. 4.1, Eq. 1-3 of Cui, Guo & Liu, "GPU Accelerated
// Finite Element Assembly with Runtime Compilation"):
//   * the weak form  (grad v, sigma grad u) + lambda (v, u) = (v, f)   (Eq. 2)
//     with sigma = kappa I per element (kappa-diffusion), plus the linear
//     elasticity form on vector P1 elements;
//   * the assembled system A x = b (Eq. 3): A_ij is the sum over every element
//     containing dofs i and j of its local entry, b_i the sum over every element
//     containing dof i of its local load entry.
// Steps, in the order the paper gives them (Sec. 5, the description of
// Algorithm 1): per element, take the vertex coordinates and global indices,
// evaluate the integrand at every quadrature point and sum into a local
// matrix and load vector, then add the local values into the global matrix
// and vector.  Here the global matrix is CSR: each local entry is added at the
// position found by a binary search of its column in its row (the sparse
// variant of Algorithm 1 searches the row for the column the same way).
//
// Conventions fixed here because the paper is silent:
//   * P2 dofs: vertex dofs are node ids; the dof of edge (a, b), a < b, is
//     N + rank of (a, b) in lexicographic order over all mesh edges; local
//     order v0..v3, then edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3);
//   * vector dofs interleaved: dof = ndpn * scalar_dof + component;
//   * the CSR pattern holds every coupled pair, ascending columns, zeros kept;
//   * matrix integrals use the 11-point degree-4 rule (exact for every matrix
//     integrand here: affine tets, element-constant coefficients, degree <= 4);
//     the load vector uses the rule the caller asks for (1, 4 or 11 points);
//   * |det J| is used; elements with det J <= 0 are counted and reported.
//
// Gradients: forward-mode dual numbers with 13 directions (the 12 vertex
// coordinates of one element and its kappa) carried through the very same
// element routine; nothing is hand-differentiated here.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------- duals
constexpr int ND = 13;
struct Dual {
  double v;
  double d[ND];
  Dual() : v(0) { for (int i = 0; i < ND; ++i) d[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < ND; ++i) d[i] = 0; }
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) { Dual r(a.v / b.v); for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
inline Dual dsin(const Dual& a) { Dual r(std::sin(a.v)); double c = std::cos(a.v); for (int i = 0; i < ND; ++i) r.d[i] = c * a.d[i]; return r; }
inline Dual dabs(const Dual& a) { return a.v < 0 ? -a : a; }
inline double val(const Dual& a) { return a.v; }
inline double dsin(double a) { return std::sin(a); }
inline double dabs(double a) { return std::fabs(a); }
inline double val(double a) { return a; }

// ---------------------------------------------------------------- rules
// Quadrature rules on a tetrahedron: barycentric points and weights that sum
// to 1, so that  int_T g = |T| sum_q w_q g(x_q).
//   1 point : centroid, degree 1.
//   4 points: permutations of (a, b, b, b), a = (5 + 3 sqrt 5)/20,
//             b = (5 - sqrt 5)/20, weight 1/4 each, degree 2 (Stroud T3:2-1).
//   11 points (Keast 1986, degree 4), weights on the reference tet of volume
//             1/6 times 6: centroid -74/5625; permutations of
//             (11/14, 1/14, 1/14, 1/14) 343/45000; permutations of
//             (c1, c1, c2, c2), c1,2 = (1 +- sqrt(5/14))/4, 56/2250.
struct Rule { int n; double bary[11][4]; double w[11]; };

Rule make_rule(int npts) {
  Rule r{};
  r.n = 0;
  if (npts == 1) {
    r.n = 1;
    for (int i = 0; i < 4; ++i) r.bary[0][i] = 0.25;
    r.w[0] = 1.0;
  } else if (npts == 4) {
    double a = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, b = (5.0 - std::sqrt(5.0)) / 20.0;
    r.n = 4;
    for (int q = 0; q < 4; ++q) {
      for (int i = 0; i < 4; ++i) r.bary[q][i] = (i == q) ? a : b;
      r.w[q] = 0.25;
    }
  } else if (npts == 11) {
    r.n = 11;
    for (int i = 0; i < 4; ++i) r.bary[0][i] = 0.25;
    r.w[0] = 6.0 * (-74.0 / 5625.0);
    for (int q = 0; q < 4; ++q) {
      for (int i = 0; i < 4; ++i) r.bary[1 + q][i] = (i == q) ? 11.0 / 14.0 : 1.0 / 14.0;
      r.w[1 + q] = 6.0 * (343.0 / 45000.0);
    }
    double c1 = (1.0 + std::sqrt(5.0 / 14.0)) / 4.0, c2 = (1.0 - std::sqrt(5.0 / 14.0)) / 4.0;
    // the 6 ways to choose which two barycentric slots hold c1
    const int pr[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int q = 0; q < 6; ++q) {
      for (int i = 0; i < 4; ++i) r.bary[5 + q][i] = c2;
      r.bary[5 + q][pr[q][0]] = c1;
      r.bary[5 + q][pr[q][1]] = c1;
      r.w[5 + q] = 6.0 * (56.0 / 2250.0);
    }
  }
  return r;
}

// local edge k of a tet joins vertices EDGE[k][0] < EDGE[k][1]
const int EDGE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// Values of the scalar basis at barycentric point L (order 1 or 2).
void basis(int order, const double L[4], double* phi) {
  if (order == 1) {
    for (int a = 0; a < 4; ++a) phi[a] = L[a];
  } else {
    for (int a = 0; a < 4; ++a) phi[a] = L[a] * (2.0 * L[a] - 1.0);
    for (int k = 0; k < 6; ++k) phi[4 + k] = 4.0 * L[EDGE[k][0]] * L[EDGE[k][1]];
  }
}

// dphi[a][i] = d phi_a / d lambda_i at barycentric point L.
void basis_dlambda(int order, const double L[4], double dphi[10][4]) {
  for (int a = 0; a < 10; ++a)
    for (int i = 0; i < 4; ++i) dphi[a][i] = 0.0;
  if (order == 1) {
    for (int a = 0; a < 4; ++a) dphi[a][a] = 1.0;
  } else {
    for (int a = 0; a < 4; ++a) dphi[a][a] = 4.0 * L[a] - 1.0;
    for (int k = 0; k < 6; ++k) {
      int p = EDGE[k][0], q = EDGE[k][1];
      dphi[4 + k][p] = 4.0 * L[q];
      dphi[4 + k][q] = 4.0 * L[p];
    }
  }
}

struct Form {
  int order;      // 1 or 2
  int kind;       // 0 Poisson/diffusion (+ mass_coef * mass), 1 elasticity
  int ndpn;       // dofs per scalar dof: 1, or 3 for elasticity
  double mass_coef;
  int f_kind;     // 0 none, 1 constant (scalar p0 / vector p0..p2), 2 p0 sin(pi x) sin(pi y) sin(pi z)
  double f_param[4];
  Rule mrule;     // matrix rule (11 points)
  Rule lrule;     // load rule (caller's)
};

// Element routine: local matrix Ke (nl x nl, row-major) and load Fe (nl) for
// vertex coordinates X[4][3].  Row index = ndpn * a + i (test function
// phi_a e_i), column index = ndpn * b + j (trial function phi_b e_j).
// Returns det J.
template <class T>
T element(const Form& F, const T X[4][3], T kappa, T lam, T mu, T* Ke, T* Fe) {
  const int nb = (F.order == 1) ? 4 : 10;
  const int nl = nb * F.ndpn;
  // J = [x1 - x0, x2 - x0, x3 - x0] (columns)
  T J[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) J[r][c] = X[c + 1][r] - X[0][r];
  // adjugate by cofactors: adj[c][r] = cofactor C[r][c]
  T adj[3][3];
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  T det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  T vol = dabs(det) / T(6.0);
  // grad lambda_i for i = 1..3 is row i-1 of J^{-1} = adj / det;
  // grad lambda_0 = -(sum of the others)
  T gl[4][3];
  for (int i = 1; i < 4; ++i)
    for (int c = 0; c < 3; ++c) gl[i][c] = adj[i - 1][c] / det;
  for (int c = 0; c < 3; ++c) gl[0][c] = -(gl[1][c] + gl[2][c] + gl[3][c]);

  for (int i = 0; i < nl * nl; ++i) Ke[i] = T(0.0);
  for (int i = 0; i < nl; ++i) Fe[i] = T(0.0);

  // ---- matrix: sum over quadrature points of the weak-form integrand
  for (int q = 0; q < F.mrule.n; ++q) {
    const double* L = F.mrule.bary[q];
    double dl[10][4];
    basis_dlambda(F.order, L, dl);
    double phi[10];
    basis(F.order, L, phi);
    T gphi[10][3];  // physical gradients at the point
    for (int a = 0; a < nb; ++a)
      for (int c = 0; c < 3; ++c) {
        T s(0.0);
        for (int i = 0; i < 4; ++i) s += T(dl[a][i]) * gl[i][c];
        gphi[a][c] = s;
      }
    T wq = T(F.mrule.w[q]) * vol;
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) {
        if (F.kind == 0) {
          T dot = gphi[a][0] * gphi[b][0] + gphi[a][1] * gphi[b][1] + gphi[a][2] * gphi[b][2];
          T v = kappa * dot + T(F.mass_coef * phi[a] * phi[b]);
          Ke[a * nl + b] += wq * v;
        } else {
          T dot = gphi[a][0] * gphi[b][0] + gphi[a][1] * gphi[b][1] + gphi[a][2] * gphi[b][2];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              T v = lam * gphi[a][i] * gphi[b][j] + mu * gphi[a][j] * gphi[b][i];
              if (i == j) v += mu * dot;
              Ke[(3 * a + i) * nl + (3 * b + j)] += wq * v;
            }
        }
      }
  }

  // ---- load: sum over quadrature points of f(x_q) phi_a(x_q)
  if (F.f_kind != 0) {
    for (int q = 0; q < F.lrule.n; ++q) {
      const double* L = F.lrule.bary[q];
      double phi[10];
      basis(F.order, L, phi);
      T xq[3];
      for (int c = 0; c < 3; ++c) {
        T s(0.0);
        for (int v = 0; v < 4; ++v) s += T(L[v]) * X[v][c];
        xq[c] = s;
      }
      T wq = T(F.lrule.w[q]) * vol;
      if (F.kind == 0) {
        T f;
        if (F.f_kind == 1) {
          f = T(F.f_param[0]);
        } else {
          f = T(F.f_param[0]) * dsin(T(M_PI) * xq[0]) * dsin(T(M_PI) * xq[1]) * dsin(T(M_PI) * xq[2]);
        }
        for (int a = 0; a < nb; ++a) Fe[a] += wq * f * T(phi[a]);
      } else {
        for (int a = 0; a < nb; ++a)
          for (int i = 0; i < 3; ++i) {
            T f;
            if (F.f_kind == 1) {
              f = T(F.f_param[i]);
            } else {
              f = T(F.f_param[i]) * dsin(T(M_PI) * xq[0]) * dsin(T(M_PI) * xq[1]) * dsin(T(M_PI) * xq[2]);
            }
            Fe[3 * a + i] += wq * f * T(phi[a]);
          }
      }
    }
  }
  return det;
}

// Position of column `col` in CSR row `row` by binary search; -1 if absent.
int64_t find_pos(const int32_t* row_ptr, const int32_t* col_idx, int64_t row, int64_t col) {
  const int32_t* b = col_idx + row_ptr[row];
  const int32_t* e = col_idx + row_ptr[row + 1];
  const int32_t* p = std::lower_bound(b, e, (int32_t)col);
  if (p == e || *p != col) return -1;
  return p - col_idx;
}

Form make_form(int order, int kind, double mass_coef, int f_kind, const double* f_param, int npts) {
  Form F{};
  F.order = order;
  F.kind = kind;
  F.ndpn = (kind == 1) ? 3 : 1;
  F.mass_coef = mass_coef;
  F.f_kind = f_kind;
  for (int i = 0; i < 4; ++i) F.f_param[i] = f_param ? f_param[i] : 0.0;
  F.mrule = make_rule(11);
  F.lrule = make_rule(npts);
  return F;
}

}  // namespace

extern "C" {

// Quadrature rule export (barycentric points npts x 4, weights summing to 1).
// Returns the number of points, 0 for an unsupported count.
int orc_rule(int npts, double* bary, double* w) {
  Rule r = make_rule(npts);
  for (int q = 0; q < r.n; ++q) {
    for (int i = 0; i < 4; ++i) bary[4 * q + i] = r.bary[q][i];
    w[q] = r.w[q];
  }
  return r.n;
}

// P2 element->dof table (SoA, 10 x E): vertex dofs are the node ids, edge
// dofs N + rank of the (min, max) vertex pair among all unique mesh edges in
// lexicographic order.  Returns the number of unique edges.
int64_t orc_p2_dofs(int64_t n_nodes, int64_t n_elems, const int32_t* tets, int32_t* edof) {
  std::vector<uint64_t> keys;
  keys.reserve(6 * n_elems);
  for (int64_t e = 0; e < n_elems; ++e)
    for (int k = 0; k < 6; ++k) {
      uint64_t a = (uint32_t)tets[EDGE[k][0] * n_elems + e];
      uint64_t b = (uint32_t)tets[EDGE[k][1] * n_elems + e];
      if (a > b) std::swap(a, b);
      keys.push_back((a << 32) | b);
    }
  std::vector<uint64_t> uniq(keys);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  for (int64_t e = 0; e < n_elems; ++e) {
    for (int v = 0; v < 4; ++v) edof[v * n_elems + e] = tets[v * n_elems + e];
    for (int k = 0; k < 6; ++k) {
      uint64_t key = keys[6 * e + k];
      int64_t rank = std::lower_bound(uniq.begin(), uniq.end(), key) - uniq.begin();
      edof[(4 + k) * n_elems + e] = (int32_t)(n_nodes + rank);
    }
  }
  return (int64_t)uniq.size();
}

// CSR pattern of the assembled matrix: every pair of dofs that share an
// element, built by sorting and de-duplicating 64-bit (row, col) keys.
// edof: nb x E SoA element->scalar-dof table; scalar dof d expands to the
// ndpn dofs ndpn*d + c.  On success *row_ptr_out (ndof+1) and *col_idx_out
// (nnz) are malloc'd here; release them with orc_free.  Returns nnz.
int64_t orc_pattern(int64_t ndof_scalar, int64_t n_elems, int nb, const int32_t* edof, int ndpn,
                    int32_t** row_ptr_out, int32_t** col_idx_out) {
  const int64_t ndof = ndof_scalar * ndpn;
  std::vector<uint64_t> keys;
  keys.reserve((size_t)n_elems * nb * nb * ndpn * ndpn);
  for (int64_t e = 0; e < n_elems; ++e)
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b)
        for (int i = 0; i < ndpn; ++i)
          for (int j = 0; j < ndpn; ++j) {
            uint64_t r = (uint64_t)edof[a * n_elems + e] * ndpn + i;
            uint64_t c = (uint64_t)edof[b * n_elems + e] * ndpn + j;
            keys.push_back(r * (uint64_t)ndof + c);
          }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  int64_t nnz = (int64_t)keys.size();
  int32_t* rp = (int32_t*)std::calloc(ndof + 1, sizeof(int32_t));
  int32_t* ci = (int32_t*)std::malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  for (int64_t k = 0; k < nnz; ++k) {
    rp[keys[k] / ndof + 1] += 1;
    ci[k] = (int32_t)(keys[k] % ndof);
  }
  for (int64_t r = 0; r < ndof; ++r) rp[r + 1] += rp[r];
  *row_ptr_out = rp;
  *col_idx_out = ci;
  return nnz;
}

void orc_free(void* p) { std::free(p); }

// Assembled matrix values (CSR, given pattern) and load vector.
//   coords: x, y, z arrays of n_nodes; edof: nb x E SoA scalar dof table;
//   kind 0: -div(kappa grad u) + mass_coef u (kappa per element, or kappa_const
//   when kappa is NULL); kind 1: linear elasticity with per-element Lame
//   parameters (or constants when NULL), vector P1/P2;
//   npts: load rule (1, 4 or 11).
// Returns the number of elements with det J <= 0, or -1 if a local entry has
// no slot in the pattern.
int64_t orc_assemble(int64_t n_nodes, const double* x, const double* y, const double* z,
                     int64_t n_elems, const int32_t* tets, int order, const int32_t* edof,
                     int kind, double mass_coef, const double* kappa, double kappa_const,
                     const double* lam, double lam_const, const double* mu, double mu_const,
                     int f_kind, const double* f_param, int npts,
                     int64_t ndof, const int32_t* row_ptr, const int32_t* col_idx,
                     double* values, double* rhs) {
  (void)n_nodes;
  Form F = make_form(order, kind, mass_coef, f_kind, f_param, npts);
  const int nb = (order == 1) ? 4 : 10;
  const int nl = nb * F.ndpn;
  std::fill(values, values + row_ptr[ndof], 0.0);
  std::fill(rhs, rhs + ndof, 0.0);
  std::vector<double> Ke(nl * nl), Fe(nl);
  int64_t bad = 0;
  for (int64_t e = 0; e < n_elems; ++e) {
    double X[4][3];
    for (int v = 0; v < 4; ++v) {
      int32_t n = tets[v * n_elems + e];
      X[v][0] = x[n]; X[v][1] = y[n]; X[v][2] = z[n];
    }
    double k = kappa ? kappa[e] : kappa_const;
    double l = lam ? lam[e] : lam_const;
    double m = mu ? mu[e] : mu_const;
    double det = element<double>(F, X, k, l, m, Ke.data(), Fe.data());
    if (!(det > 0)) ++bad;
    for (int a = 0; a < nl; ++a) {
      int64_t ra = (int64_t)edof[(a / F.ndpn) * n_elems + e] * F.ndpn + a % F.ndpn;
      rhs[ra] += Fe[a];
      for (int b = 0; b < nl; ++b) {
        int64_t cb = (int64_t)edof[(b / F.ndpn) * n_elems + e] * F.ndpn + b % F.ndpn;
        int64_t p = find_pos(row_ptr, col_idx, ra, cb);
        if (p < 0) return -1;
        values[p] += Ke[a * nl + b];
      }
    }
  }
  return bad;
}

// Local matrices and load vectors of a list of elements (nl x nl row-major
// and nl per element), for element-level checks.
void orc_local(const double* Xall /* n x 4 x 3 */, int64_t n, int order, int kind,
               double mass_coef, const double* kappa, const double* lam, const double* mu,
               int f_kind, const double* f_param, int npts, double* Ke_out, double* Fe_out,
               double* det_out) {
  Form F = make_form(order, kind, mass_coef, f_kind, f_param, npts);
  const int nb = (order == 1) ? 4 : 10;
  const int nl = nb * F.ndpn;
  for (int64_t e = 0; e < n; ++e) {
    double X[4][3];
    for (int v = 0; v < 4; ++v)
      for (int c = 0; c < 3; ++c) X[v][c] = Xall[12 * e + 3 * v + c];
    double det = element<double>(F, X, kappa ? kappa[e] : 1.0, lam ? lam[e] : 1.0,
                                 mu ? mu[e] : 1.0, Ke_out + e * nl * nl, Fe_out + e * nl);
    if (det_out) det_out[e] = det;
  }
}

// Selected rows of the assembled system by brute force over all elements,
// without a pattern: for each requested row (sorted ascending, unique) every
// element that holds the row's dof adds its local row.  Output is COO
// (row, col, value) sorted by (row, col) plus rhs per requested row; the
// arrays are malloc'd here (release with orc_free).  Returns the entry count.
int64_t orc_rows(const double* x, const double* y, const double* z, int64_t n_elems,
                 const int32_t* tets, int order, const int32_t* edof, int kind,
                 double mass_coef, const double* kappa, double kappa_const, const double* lam,
                 double lam_const, const double* mu, double mu_const, int f_kind,
                 const double* f_param, int npts, const int64_t* rows, int64_t nrows,
                 int64_t** r_out, int64_t** c_out, double** v_out, double* rhs_out) {
  Form F = make_form(order, kind, mass_coef, f_kind, f_param, npts);
  const int nb = (order == 1) ? 4 : 10;
  const int nl = nb * F.ndpn;
  std::vector<std::pair<std::pair<int64_t, int64_t>, double>> acc;
  std::vector<double> Ke(nl * nl), Fe(nl);
  for (int64_t i = 0; i < nrows; ++i) rhs_out[i] = 0.0;
  std::vector<int64_t> sel(nl);
  for (int64_t e = 0; e < n_elems; ++e) {
    bool any = false;
    for (int a = 0; a < nl; ++a) {
      int64_t ra = (int64_t)edof[(a / F.ndpn) * n_elems + e] * F.ndpn + a % F.ndpn;
      const int64_t* p = std::lower_bound(rows, rows + nrows, ra);
      sel[a] = (p != rows + nrows && *p == ra) ? (p - rows) : -1;
      any = any || sel[a] >= 0;
    }
    if (!any) continue;
    double X[4][3];
    for (int v = 0; v < 4; ++v) {
      int32_t n = tets[v * n_elems + e];
      X[v][0] = x[n]; X[v][1] = y[n]; X[v][2] = z[n];
    }
    element<double>(F, X, kappa ? kappa[e] : kappa_const, lam ? lam[e] : lam_const,
                    mu ? mu[e] : mu_const, Ke.data(), Fe.data());
    for (int a = 0; a < nl; ++a) {
      if (sel[a] < 0) continue;
      int64_t ra = rows[sel[a]];
      rhs_out[sel[a]] += Fe[a];
      for (int b = 0; b < nl; ++b) {
        int64_t cb = (int64_t)edof[(b / F.ndpn) * n_elems + e] * F.ndpn + b % F.ndpn;
        acc.push_back({{ra, cb}, Ke[a * nl + b]});
      }
    }
  }
  // stable sort keeps element order inside each (row, col) group
  std::stable_sort(acc.begin(), acc.end(),
                   [](const auto& p, const auto& q) { return p.first < q.first; });
  std::vector<int64_t> R, C;
  std::vector<double> V;
  for (size_t k = 0; k < acc.size(); ++k) {
    if (!R.empty() && R.back() == acc[k].first.first && C.back() == acc[k].first.second) {
      V.back() += acc[k].second;
    } else {
      R.push_back(acc[k].first.first);
      C.push_back(acc[k].first.second);
      V.push_back(acc[k].second);
    }
  }
  int64_t n = (int64_t)R.size();
  *r_out = (int64_t*)std::malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  *c_out = (int64_t*)std::malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  *v_out = (double*)std::malloc(sizeof(double) * (n > 0 ? n : 1));
  for (int64_t k = 0; k < n; ++k) {
    (*r_out)[k] = R[k];
    (*c_out)[k] = C[k];
    (*v_out)[k] = V[k];
  }
  return n;
}

// Gradient of L = sum_p grad_values[p] * values[p] + sum_i grad_rhs[i] * rhs[i]
// with respect to the per-element kappa and the node coordinates, for the
// scalar forms (kind 0).  Each element is run through the element routine in
// dual numbers seeded with its 12 vertex coordinates and its kappa.
// grad_values / grad_rhs may be NULL (treated as zero).  grad_x is 3 x N SoA.
// Returns -1 if a local entry has no slot in the pattern, else 0.
int64_t orc_assemble_grad(int64_t n_nodes, const double* x, const double* y, const double* z,
                          int64_t n_elems, const int32_t* tets, int order, const int32_t* edof,
                          double mass_coef, const double* kappa, double kappa_const, int f_kind,
                          const double* f_param, int npts, int64_t ndof, const int32_t* row_ptr,
                          const int32_t* col_idx, const double* grad_values, const double* grad_rhs,
                          double* grad_kappa, double* grad_x) {
  Form F = make_form(order, 0, mass_coef, f_kind, f_param, npts);
  (void)ndof;
  const int nl = (order == 1) ? 4 : 10;
  std::fill(grad_x, grad_x + 3 * n_nodes, 0.0);
  std::vector<Dual> Ke(nl * nl), Fe(nl);
  for (int64_t e = 0; e < n_elems; ++e) {
    Dual X[4][3];
    int32_t nid[4];
    for (int v = 0; v < 4; ++v) {
      nid[v] = tets[v * n_elems + e];
      double xv[3] = {x[nid[v]], y[nid[v]], z[nid[v]]};
      for (int c = 0; c < 3; ++c) {
        X[v][c] = Dual(xv[c]);
        X[v][c].d[3 * v + c] = 1.0;
      }
    }
    Dual k(kappa ? kappa[e] : kappa_const);
    k.d[12] = 1.0;
    element<Dual>(F, X, k, Dual(1.0), Dual(1.0), Ke.data(), Fe.data());
    double dL[ND];
    for (int i = 0; i < ND; ++i) dL[i] = 0.0;
    for (int a = 0; a < nl; ++a) {
      int64_t ra = edof[a * n_elems + e];
      double gf = grad_rhs ? grad_rhs[ra] : 0.0;
      for (int i = 0; i < ND; ++i) dL[i] += gf * Fe[a].d[i];
      if (!grad_values) continue;
      for (int b = 0; b < nl; ++b) {
        int64_t p = find_pos(row_ptr, col_idx, ra, edof[b * n_elems + e]);
        if (p < 0) return -1;
        double gv = grad_values[p];
        for (int i = 0; i < ND; ++i) dL[i] += gv * Ke[a * nl + b].d[i];
      }
    }
    if (grad_kappa) grad_kappa[e] = dL[12];
    for (int v = 0; v < 4; ++v)
      for (int c = 0; c < 3; ++c) grad_x[c * n_nodes + nid[v]] += dL[3 * v + c];
  }
  return 0;
}


}  // extern "C"

namespace {

// ---------------------------------------------------------------- 2-D triangles
// The paper's worked example (Sec. 4.1-4.2): P1 triangles, Eq. 1 with a
// matrix coefficient sigma(x, y) and a mass term lambda u, load f.
//   sigma(x, y) = S0 + x Sx + y Sy (2 x 2, row-major, affine in x and y);
//   f(x, y) = f0 + f1 x + f2 y + f3 x^2 + f4 x y + f5 y^2.
// The bilinear form (grad v, sigma grad u): row = test function phi_a,
// column = trial function phi_b, so A is not symmetric when sigma is not.
// Triangle rules (barycentric points, weights summing to 1):
//   1 point: centroid (degree 1); 3 points: permutations of (2/3, 1/6, 1/6),
//   weight 1/3 (degree 2); 6 points (degree 4): permutations of
//   (a, a, 1 - 2a) for a = (8 - sqrt 10 +- sqrt(38 - 44 sqrt(2/5))) / 18 with
//   weights (620 +- sqrt(213125 - 53320 sqrt 10)) / 3720.
// Matrix integrals use the 6-point rule (exact: integrands of degree <= 2);
// the load uses the caller's rule.
struct TriRule { int n; double bary[6][3]; double w[6]; };

TriRule make_tri_rule(int npts) {
  TriRule r{};
  if (npts == 1) {
    r.n = 1;
    for (int i = 0; i < 3; ++i) r.bary[0][i] = 1.0 / 3.0;
    r.w[0] = 1.0;
  } else if (npts == 3) {
    r.n = 3;
    for (int q = 0; q < 3; ++q) {
      for (int i = 0; i < 3; ++i) r.bary[q][i] = (i == q) ? 2.0 / 3.0 : 1.0 / 6.0;
      r.w[q] = 1.0 / 3.0;
    }
  } else if (npts == 6) {
    r.n = 6;
    const double s10 = std::sqrt(10.0), t = std::sqrt(38.0 - 44.0 * std::sqrt(0.4));
    const double a[2] = {(8.0 - s10 + t) / 18.0, (8.0 - s10 - t) / 18.0};
    const double u = std::sqrt(213125.0 - 53320.0 * s10);
    const double w[2] = {(620.0 + u) / 3720.0, (620.0 - u) / 3720.0};
    int q = 0;
    for (int c = 0; c < 2; ++c)
      for (int odd = 0; odd < 3; ++odd, ++q) {
        for (int i = 0; i < 3; ++i) r.bary[q][i] = (i == odd) ? 1.0 - 2.0 * a[c] : a[c];
        r.w[q] = w[c];
      }
  }
  return r;
}

struct Form2D {
  double S0[4], Sx[4], Sy[4];
  double lambda;
  double f[6];
  TriRule mrule, lrule;
};

// Local 3 x 3 matrix (row-major) and load of one triangle; returns det J.
double element_tri(const Form2D& F, const double X[3][2], double* Ke, double* Fe) {
  // J = [x1 - x0, x2 - x0] (columns); grad lambda_1,2 = rows of J^{-1}
  const double J[2][2] = {{X[1][0] - X[0][0], X[2][0] - X[0][0]}, {X[1][1] - X[0][1], X[2][1] - X[0][1]}};
  const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double area = std::fabs(det) / 2.0;
  double g[3][2];
  g[1][0] = J[1][1] / det;
  g[1][1] = -J[0][1] / det;
  g[2][0] = -J[1][0] / det;
  g[2][1] = J[0][0] / det;
  g[0][0] = -(g[1][0] + g[2][0]);
  g[0][1] = -(g[1][1] + g[2][1]);
  for (int i = 0; i < 9; ++i) Ke[i] = 0.0;
  for (int i = 0; i < 3; ++i) Fe[i] = 0.0;
  for (int q = 0; q < F.mrule.n; ++q) {
    const double* L = F.mrule.bary[q];
    const double x = L[0] * X[0][0] + L[1] * X[1][0] + L[2] * X[2][0];
    const double y = L[0] * X[0][1] + L[1] * X[1][1] + L[2] * X[2][1];
    double sig[4];
    for (int k = 0; k < 4; ++k) sig[k] = F.S0[k] + x * F.Sx[k] + y * F.Sy[k];
    const double wq = F.mrule.w[q] * area;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double sg0 = sig[0] * g[b][0] + sig[1] * g[b][1];
        const double sg1 = sig[2] * g[b][0] + sig[3] * g[b][1];
        Ke[3 * a + b] += wq * (g[a][0] * sg0 + g[a][1] * sg1 + F.lambda * L[a] * L[b]);
      }
  }
  for (int q = 0; q < F.lrule.n; ++q) {
    const double* L = F.lrule.bary[q];
    const double x = L[0] * X[0][0] + L[1] * X[1][0] + L[2] * X[2][0];
    const double y = L[0] * X[0][1] + L[1] * X[1][1] + L[2] * X[2][1];
    const double fv = F.f[0] + F.f[1] * x + F.f[2] * y + F.f[3] * x * x + F.f[4] * x * y + F.f[5] * y * y;
    const double wq = F.lrule.w[q] * area;
    for (int a = 0; a < 3; ++a) Fe[a] += wq * fv * L[a];
  }
  return det;
}

Form2D make_form2d(const double* S0, const double* Sx, const double* Sy, double lambda, const double* f, int npts) {
  Form2D F{};
  for (int k = 0; k < 4; ++k) {
    F.S0[k] = S0[k];
    F.Sx[k] = Sx[k];
    F.Sy[k] = Sy[k];
  }
  F.lambda = lambda;
  for (int k = 0; k < 6; ++k) F.f[k] = f[k];
  F.mrule = make_tri_rule(6);
  F.lrule = make_tri_rule(npts);
  return F;
}

}  // namespace

extern "C" {

int orc_tri_rule(int npts, double* bary, double* w) {
  TriRule r = make_tri_rule(npts);
  for (int q = 0; q < r.n; ++q) {
    for (int i = 0; i < 3; ++i) bary[3 * q + i] = r.bary[q][i];
    w[q] = r.w[q];
  }
  return r.n;
}

// Local matrices (n x 3 x 3) and loads (n x 3) of triangles X (n x 3 x 2).
void orc_local_tri(const double* Xall, int64_t n, const double* S0, const double* Sx, const double* Sy,
                   double lambda, const double* f, int npts, double* Ke, double* Fe, double* det) {
  Form2D F = make_form2d(S0, Sx, Sy, lambda, f, npts);
  for (int64_t e = 0; e < n; ++e) {
    double X[3][2];
    for (int v = 0; v < 3; ++v)
      for (int c = 0; c < 2; ++c) X[v][c] = Xall[6 * e + 2 * v + c];
    const double d = element_tri(F, X, Ke + 9 * e, Fe + 3 * e);
    if (det) det[e] = d;
  }
}

// Assembled CSR values and load of the 2-D problem (Eq. 3); tris: 3 x E SoA.
// Returns the number of triangles with det J <= 0, or -1 on a missing slot.
int64_t orc_assemble_tri(int64_t n_nodes, const double* x, const double* y, int64_t n_elems, const int32_t* tris,
                         const double* S0, const double* Sx, const double* Sy, double lambda, const double* f,
                         int npts, const int32_t* row_ptr, const int32_t* col_idx, double* values, double* rhs) {
  Form2D F = make_form2d(S0, Sx, Sy, lambda, f, npts);
  std::fill(values, values + row_ptr[n_nodes], 0.0);
  std::fill(rhs, rhs + n_nodes, 0.0);
  int64_t bad = 0;
  double Ke[9], Fe[3];
  for (int64_t e = 0; e < n_elems; ++e) {
    double X[3][2];
    int32_t nd[3];
    for (int v = 0; v < 3; ++v) {
      nd[v] = tris[v * n_elems + e];
      X[v][0] = x[nd[v]];
      X[v][1] = y[nd[v]];
    }
    if (!(element_tri(F, X, Ke, Fe) > 0)) ++bad;
    for (int a = 0; a < 3; ++a) {
      rhs[nd[a]] += Fe[a];
      for (int b = 0; b < 3; ++b) {
        const int64_t p = find_pos(row_ptr, col_idx, nd[a], nd[b]);
        if (p < 0) return -1;
        values[p] += Ke[3 * a + b];
      }
    }
  }
  return bad;
}

}  // extern "C"

// ---------------------------------------------------------------- user coefficients
// Scalar form  -div(kappa_T k(x) grad u) + mass_coef u = f(x)  on P1/P2 tets,
// with k and f caller-supplied point functions.  The paper's system compiles
// the user's symbolic weak form into the kernel at run time (Sec. 5, runtime
// compilation); whatever the compiled kernel does, the integrals it must
// reach are these, taken literally:
//   * stiffness: sum over the caller's rule of w_q |T| kappa_T k(x_q)
//     grad phi_a(x_q) . grad phi_b(x_q); when k is absent (k = 1) the
//     11-point rule is used instead, which is exact for it;
//   * mass: 11-point rule (exact for P1 and P2 on affine tets);
//   * load: sum over the caller's rule of w_q |T| f(x_q) phi_a(x_q)
//     (zero when f is absent).
namespace {

typedef double (*PointFn)(double, double, double);

double element_user(int order, double mass_coef, double kappa_T, PointFn kfn, PointFn ffn, int npts,
                    const double X[4][3], double* Ke, double* Fe) {
  const int nb = (order == 1) ? 4 : 10;
  double J[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) J[r][c] = X[c + 1][r] - X[0][r];
  // J^{-1} by cofactors
  double adj[3][3];
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  const double vol = std::fabs(det) / 6.0;
  double gl[4][3];
  for (int i = 1; i < 4; ++i)
    for (int c = 0; c < 3; ++c) gl[i][c] = adj[i - 1][c] / det;
  for (int c = 0; c < 3; ++c) gl[0][c] = -(gl[1][c] + gl[2][c] + gl[3][c]);
  for (int i = 0; i < nb * nb; ++i) Ke[i] = 0.0;
  for (int i = 0; i < nb; ++i) Fe[i] = 0.0;

  auto point = [&](const double* L, double xq[3]) {
    for (int c = 0; c < 3; ++c) {
      xq[c] = 0.0;
      for (int v = 0; v < 4; ++v) xq[c] += L[v] * X[v][c];
    }
  };
  // stiffness
  const Rule ks = make_rule(kfn ? npts : 11);
  for (int q = 0; q < ks.n; ++q) {
    const double* L = ks.bary[q];
    double dl[10][4];
    basis_dlambda(order, L, dl);
    double gphi[10][3];
    for (int a = 0; a < nb; ++a)
      for (int c = 0; c < 3; ++c) {
        gphi[a][c] = 0.0;
        for (int i = 0; i < 4; ++i) gphi[a][c] += dl[a][i] * gl[i][c];
      }
    double k = kappa_T;
    if (kfn) {
      double xq[3];
      point(L, xq);
      k *= kfn(xq[0], xq[1], xq[2]);
    }
    const double wq = ks.w[q] * vol;
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b)
        Ke[a * nb + b] += wq * k * (gphi[a][0] * gphi[b][0] + gphi[a][1] * gphi[b][1] + gphi[a][2] * gphi[b][2]);
  }
  // mass
  if (mass_coef != 0.0) {
    const Rule ms = make_rule(11);
    for (int q = 0; q < ms.n; ++q) {
      double phi[10];
      basis(order, ms.bary[q], phi);
      const double wq = ms.w[q] * vol;
      for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b) Ke[a * nb + b] += wq * mass_coef * phi[a] * phi[b];
    }
  }
  // load
  if (ffn) {
    const Rule ls = make_rule(npts);
    for (int q = 0; q < ls.n; ++q) {
      double phi[10], xq[3];
      basis(order, ls.bary[q], phi);
      point(ls.bary[q], xq);
      const double wq = ls.w[q] * vol;
      const double f = ffn(xq[0], xq[1], xq[2]);
      for (int a = 0; a < nb; ++a) Fe[a] += wq * f * phi[a];
    }
  }
  return det;
}

}  // namespace

extern "C" {

// Assembled CSR values and load of the user-coefficient scalar form (see
// element_user).  kappa: per-element kappa_T, or kappa_const when NULL;
// kfn / ffn may be NULL.  Returns the count of elements with det J <= 0, or
// -1 if a local entry has no slot in the pattern.
int64_t orc_assemble_user(int64_t n_nodes, const double* x, const double* y, const double* z, int64_t n_elems,
                          const int32_t* tets, int order, const int32_t* edof, double mass_coef,
                          const double* kappa, double kappa_const, PointFn kfn, PointFn ffn, int npts,
                          int64_t ndof, const int32_t* row_ptr, const int32_t* col_idx, double* values,
                          double* rhs) {
  (void)n_nodes;
  const int nb = (order == 1) ? 4 : 10;
  std::fill(values, values + row_ptr[ndof], 0.0);
  std::fill(rhs, rhs + ndof, 0.0);
  std::vector<double> Ke(nb * nb), Fe(nb);
  int64_t bad = 0;
  for (int64_t e = 0; e < n_elems; ++e) {
    double X[4][3];
    for (int v = 0; v < 4; ++v) {
      const int32_t n = tets[v * n_elems + e];
      X[v][0] = x[n];
      X[v][1] = y[n];
      X[v][2] = z[n];
    }
    const double det = element_user(order, mass_coef, kappa ? kappa[e] : kappa_const, kfn, ffn, npts, X,
                                    Ke.data(), Fe.data());
    if (!(det > 0)) ++bad;
    for (int a = 0; a < nb; ++a) {
      const int64_t ra = edof[a * n_elems + e];
      rhs[ra] += Fe[a];
      for (int b = 0; b < nb; ++b) {
        const int64_t p = find_pos(row_ptr, col_idx, ra, edof[b * n_elems + e]);
        if (p < 0) return -1;
        values[p] += Ke[a * nb + b];
      }
    }
  }
  return bad;
}

// Local matrices (nb x nb) and loads (nb) of a list of elements for the
// user-coefficient form; kappa_T = 1.
void orc_local_user(const double* Xall /* n x 4 x 3 */, int64_t n, int order, double mass_coef, PointFn kfn,
                    PointFn ffn, int npts, double* Ke_out, double* Fe_out) {
  const int nb = (order == 1) ? 4 : 10;
  for (int64_t e = 0; e < n; ++e) {
    double X[4][3];
    for (int v = 0; v < 4; ++v)
      for (int c = 0; c < 3; ++c) X[v][c] = Xall[12 * e + 3 * v + c];
    element_user(order, mass_coef, 1.0, kfn, ffn, npts, X, Ke_out + e * nb * nb, Fe_out + e * nb);
  }
}

}  // extern "C"

// ---------------------------------------------------------------- Dirichlet conditions
// Closing the loop to a solve (the paper assembles the pure Neumann operator
// and leaves solving out): for every dof d of the list, row d becomes the
// identity row with right-hand side g_d, and column d is eliminated from the
// other rows, rhs_i -= A_id g_d, A_id = 0 (A stays symmetric).  The textbook
// elimination, done literally: first the right-hand-side corrections with the
// original values, then the zeroing.
extern "C" void orc_dirichlet(int64_t ndof, const int32_t* row_ptr, const int32_t* col_idx, double* values,
                              double* rhs, int64_t n, const int32_t* dofs, const double* g) {
  std::vector<char> fixed(ndof, 0);
  std::vector<double> gv(ndof, 0.0);
  for (int64_t k = 0; k < n; ++k) {
    fixed[dofs[k]] = 1;
    gv[dofs[k]] = g ? g[k] : 0.0;
  }
  for (int64_t i = 0; i < ndof; ++i) {
    if (fixed[i]) continue;
    for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
      if (fixed[col_idx[p]]) rhs[i] -= values[p] * gv[col_idx[p]];
  }
  for (int64_t i = 0; i < ndof; ++i)
    for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      const int32_t c = col_idx[p];
      if (fixed[i]) values[p] = (c == i) ? 1.0 : 0.0;
      else if (fixed[c]) values[p] = 0.0;
    }
  for (int64_t i = 0; i < ndof; ++i)
    if (fixed[i]) rhs[i] = gv[i];
}

// ---------------------------------------------------------------- CPU baseline
// Not a checker: the timing baseline of the benchmark on all host cores.  The
// element loop of orc_assemble (same element routine, same binary-search
// scatter), with the elements split over OpenMP threads: each thread adds
// into its own zeroed copy of the values and the load vector, and the copies
// are then summed position by position.  Without OpenMP it runs on one
// thread.  Returns the number of elements with det J <= 0, or -1.
#ifdef _OPENMP
#include <omp.h>
#endif
extern "C" int64_t orc_assemble_par(const double* x, const double* y, const double* z, int64_t n_elems,
                                    const int32_t* tets, int order, const int32_t* edof, int kind,
                                    double mass_coef, const double* kappa, double kappa_const, const double* lam,
                                    double lam_const, const double* mu, double mu_const, int f_kind,
                                    const double* f_param, int npts, int64_t ndof, const int32_t* row_ptr,
                                    const int32_t* col_idx, double* values, double* rhs, int nthreads,
                                    int* used_threads) {
  Form F = make_form(order, kind, mass_coef, f_kind, f_param, npts);
  const int nb = (order == 1) ? 4 : 10;
  const int nl = nb * F.ndpn;
  const int64_t nnz = row_ptr[ndof];
  int T = 1;
#ifdef _OPENMP
  T = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
  std::vector<std::vector<double>> V(T), R(T);
  int64_t bad = 0, missing = 0;
#pragma omp parallel num_threads(T) reduction(+ : bad, missing)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    V[t].assign(nnz, 0.0);
    R[t].assign(ndof, 0.0);
    std::vector<double> Ke(nl * nl), Fe(nl);
#pragma omp for schedule(static)
    for (int64_t e = 0; e < n_elems; ++e) {
      double X[4][3];
      for (int v = 0; v < 4; ++v) {
        int32_t n = tets[v * n_elems + e];
        X[v][0] = x[n]; X[v][1] = y[n]; X[v][2] = z[n];
      }
      double det = element<double>(F, X, kappa ? kappa[e] : kappa_const, lam ? lam[e] : lam_const,
                                   mu ? mu[e] : mu_const, Ke.data(), Fe.data());
      if (!(det > 0)) ++bad;
      for (int a = 0; a < nl; ++a) {
        int64_t ra = (int64_t)edof[(a / F.ndpn) * n_elems + e] * F.ndpn + a % F.ndpn;
        R[t][ra] += Fe[a];
        for (int b = 0; b < nl; ++b) {
          int64_t cb = (int64_t)edof[(b / F.ndpn) * n_elems + e] * F.ndpn + b % F.ndpn;
          int64_t p = find_pos(row_ptr, col_idx, ra, cb);
          if (p < 0) ++missing;
          else V[t][p] += Ke[a * nl + b];
        }
      }
    }
  }
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t p = 0; p < nnz; ++p) {
    double s = 0.0;
    for (int t = 0; t < T; ++t) s += V[t][p];
    values[p] = s;
  }
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t i = 0; i < ndof; ++i) {
    double s = 0.0;
    for (int t = 0; t < T; ++t) s += R[t][i];
    rhs[i] = s;
  }
  if (used_threads) *used_threads = T;
  return missing ? -1 : bad;
}
