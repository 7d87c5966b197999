// Host-side setup of one (BDM_k, dP_{k-1}) level on the structured triangle mesh (Case 3 of Sec. 3):
// H(div)-conforming velocity (vector P_k with continuous normal components, Sec. 2.1), discontinuous
// P_{k-1} pressure, the symmetric interior-penalty form of Eq. (DiscontBilinearForm) over interior
// edges, the no-flux condition u . n = 0 as Dirichlet rows on boundary-edge DoFs (Eq.
// StokesBCforDGFEM1), canonical transfers and extended cell Vanka patches (Sec. 3.1).
//
// DoFs (shared with the whole library's conventions):
//  * per edge (oriented from its lower to its higher vertex id), the normal flux
//    v(x_j) . rot(x_b - x_a), rot(x, y) = (y, -x), at x_j = x_a + (j+1)/(k+2) (x_b - x_a), j = 0..k;
//  * per cell, the moments int_ref vhat . q over the reference cell, q in Nedelec's first-kind space
//    of degree k - 1 (vector P_{k-2}, then (-y, x) times the homogeneous P_{k-2}), orthogonalised in
//    L^2 of the reference cell and scaled to norms in [1, 2) by powers of two (a well-scaled basis);
//  * per cell, the pressure at the equispaced P_{k-1} nodes (one at the centroid for k = 1).
//  Cells carry the reference basis by the contravariant Piola map v = J vhat / det J, under which
//  the scaled normal flux is invariant; a cell traversing an edge against its orientation sees the
//  edge's DoFs with the opposite sign at mirrored points.
//  Order: edges (horizontal, vertical, diagonal; lexicographic), then each cell's interior moments,
//  then each cell's pressures (cells: lower triangles, then upper, lexicographic).
// The penalty is alpha = (k + 1)(k + 2) (the paper asks for a sufficiently large one): twice the
// k-dependence (k + 1)(k + 2) / 2 of the trace inverse inequality on triangles, below which a_h stops
// being coercive on this mesh family.
#include <algorithm>
#include <array>
#include <cmath>
#include <exception>
#include <map>
#include <stdexcept>
#include <thread>
#include <utility>
#include <vector>

#include "vk_internal.h"

namespace vk {

namespace {

// vector monomials of P_k^2: (component, p, q) with p + q <= k, q outer
struct VMono {
  int c, p, q;
};

std::vector<VMono> vmonos(int k) {
  std::vector<VMono> m;
  for (int c = 0; c < 2; ++c)
    for (int q = 0; q <= k; ++q)
      for (int p = 0; p + q <= k; ++p) m.push_back({c, p, q});
  return m;
}

// Nedelec first-kind space of degree k - 1 spanned by monomial pairs, as sums of terms (component, p, q,
// coefficient): P_{k-2}^2 (x then y component per monomial, q outer), then (-y, x) times the homogeneous
// monomials of degree k - 2
struct Term {
  int c, p, q;
  double w;
};
std::vector<std::vector<Term>> nedelec_monomial(int k) {
  std::vector<std::vector<Term>> out;
  for (int q = 0; q <= k - 2; ++q)
    for (int p = 0; p + q <= k - 2; ++p) {
      out.push_back({{0, p, q, 1.0}});
      out.push_back({{1, p, q, 1.0}});
    }
  if (k >= 2)
    for (int q = 0; q <= k - 2; ++q) {
      const int p = k - 2 - q;
      out.push_back({{0, p, q + 1, -1.0}, {1, p + 1, q, 1.0}});   // (-y, x) x^p y^q
    }
  return out;
}

double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

const int kEdge[3][2] = {{1, 2}, {0, 2}, {0, 1}};   // local edge i opposite vertex i, traversed a -> b
const double kVert[3][2] = {{0, 0}, {1, 0}, {0, 1}};

// Double-double numbers (an unevaluated sum hi + lo, about 106 significant bits) from the error-free
// transformations of Knuth (TwoSum) and Dekker (TwoProduct, here through a fused multiply-add): the
// reference basis is the inverse of a Vandermonde-type matrix whose condition number grows to 1e9 at
// k = 5, so it is solved in this precision and rounded once to FP64.
struct DD {
  double hi = 0.0, lo = 0.0;
};
DD two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
DD fast_two_sum(double a, double b) {
  const double s = a + b;
  return {s, b - (s - a)};
}
DD operator+(DD a, DD b) {
  DD s = two_sum(a.hi, b.hi);
  const DD t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
DD operator-(DD a) { return {-a.hi, -a.lo}; }
DD operator-(DD a, DD b) { return a + (-b); }
DD operator*(DD a, DD b) {
  const double p = a.hi * b.hi;
  double e = std::fma(a.hi, b.hi, -p);
  e += a.hi * b.lo + a.lo * b.hi;
  return fast_two_sum(p, e);
}
DD operator/(DD a, DD b) {
  // three quotient digits, each from the remainder of the previous ones
  const double q1 = a.hi / b.hi;
  DD r = a - b * DD{q1, 0.0};
  const double q2 = r.hi / b.hi;
  r = r - b * DD{q2, 0.0};
  const double q3 = r.hi / b.hi;
  return fast_two_sum(q1, q2) + DD{q3, 0.0};
}
DD dd(double x) { return {x, 0.0}; }
DD dd_ratio(double a, double b) { return dd(a) / dd(b); }   // a, b integers exactly representable
DD dd_pow(DD x, int p) {
  DD r = dd(1.0);
  for (int i = 0; i < p; ++i) r = r * x;
  return r;
}

// Gaussian elimination with partial pivoting in double-double: solves A X = B (n x n, n x nrhs, row
// major, both overwritten; X in B).
void lu_solve_dd(int n, std::vector<DD>& A, std::vector<DD>& B, int nrhs) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[size_t(r) * n + c].hi) > std::fabs(A[size_t(p) * n + c].hi)) p = r;
    if (A[size_t(p) * n + c].hi == 0.0) throw std::runtime_error("BDM: singular Vandermonde");
    if (p != c) {
      for (int j = 0; j < n; ++j) std::swap(A[size_t(c) * n + j], A[size_t(p) * n + j]);
      for (int j = 0; j < nrhs; ++j) std::swap(B[size_t(c) * nrhs + j], B[size_t(p) * nrhs + j]);
    }
    for (int r = c + 1; r < n; ++r) {
      if (A[size_t(r) * n + c].hi == 0.0) continue;
      const DD f = A[size_t(r) * n + c] / A[size_t(c) * n + c];
      for (int j = c; j < n; ++j) A[size_t(r) * n + j] = A[size_t(r) * n + j] - f * A[size_t(c) * n + j];
      for (int j = 0; j < nrhs; ++j) B[size_t(r) * nrhs + j] = B[size_t(r) * nrhs + j] - f * B[size_t(c) * nrhs + j];
    }
  }
  for (int c = n - 1; c >= 0; --c)
    for (int j = 0; j < nrhs; ++j) {
      DD s = B[size_t(c) * nrhs + j];
      for (int m = c + 1; m < n; ++m) s = s - A[size_t(c) * n + m] * B[size_t(m) * nrhs + j];
      B[size_t(c) * nrhs + j] = s / A[size_t(c) * n + c];
    }
}

// Test functions of the interior moments: the monomial-generated Nedelec functions orthogonalised in
// L^2 of the reference triangle (Gram-Schmidt in their order, double-double), each scaled by the power of
// two 2^-floor(t / 2), t = floor(log2 |q|^2), so that its norm lies in [1, 2).  Inner products from
// int x^a y^b = a! b! / (a + b + 2)!.
struct TermD {
  int c, p, q;
  DD w;
};
std::vector<std::vector<TermD>> nedelec(int k) {
  const auto base = nedelec_monomial(k);
  // dense coefficient vectors over (component, p, q) with p + q <= k - 1
  const int d = std::max(k - 1, 0), side = d + 1;
  auto at = [&](int c, int p, int q) { return (c * side + p) * side + q; };
  const size_t len = size_t(2) * side * side;
  auto inner = [&](const std::vector<DD>& a, const std::vector<DD>& b) {
    DD s;
    for (int c = 0; c < 2; ++c)
      for (int p = 0; p <= d; ++p)
        for (int q = 0; p + q <= d; ++q) {
          const DD u = a[at(c, p, q)];
          if (u.hi == 0.0) continue;
          for (int r = 0; r <= d; ++r)
            for (int t = 0; r + t <= d; ++t) {
              const DD v = b[at(c, r, t)];
              if (v.hi != 0.0) s = s + u * v * dd_ratio(fact(p + r) * fact(q + t), fact(p + r + q + t + 2));
            }
        }
    return s;
  };
  std::vector<std::vector<DD>> e;
  std::vector<DD> n2;
  for (const auto& f : base) {
    std::vector<DD> v(len);
    for (const Term& t : f) v[at(t.c, t.p, t.q)] = dd(t.w);
    for (size_t j = 0; j < e.size(); ++j) {
      const DD cj = inner(v, e[j]) / n2[j];
      for (size_t x = 0; x < len; ++x)
        if (e[j][x].hi != 0.0) v[x] = v[x] - cj * e[j][x];
    }
    n2.push_back(inner(v, v));
    e.push_back(std::move(v));
  }
  std::vector<std::vector<TermD>> out;
  for (size_t j = 0; j < e.size(); ++j) {
    const int t = std::ilogb(n2[j].hi + n2[j].lo);   // floor(log2 |q|^2) of the rounded norm
    const int h = t >= 0 ? t / 2 : -((-t + 1) / 2);    // floor(t / 2)
    const DD sc = dd(std::ldexp(1.0, -h));
    std::vector<TermD> f;
    for (int c = 0; c < 2; ++c)
      for (int p = 0; p <= d; ++p)
        for (int q = 0; p + q <= d; ++q) {
          // exact zeros of the rational coefficients come out as rounding residue of order 1e-30
          const DD w = e[j][at(c, p, q)];
          if (std::fabs(w.hi) > 1e-20) f.push_back({c, p, q, sc * w});
        }
    out.push_back(std::move(f));
  }
  return out;
}

constexpr int kMaxNb = 42;   // (k + 1)(k + 2) for k = 5

// Reference BDM_k basis: coefficient matrix C[m][i] of monomial m in basis function i (dual to the DoFs
// in local order: edge e point j at e (k+1) + j, then the Nedelec moments).
struct RefBDM {
  int k = 0, n = 0;
  std::vector<VMono> mono;
  std::vector<double> C;   // n x n
  std::vector<DD> Cd;      // the same in double-double
  // value (component c) and reference derivative d/dx_d of basis i at (x, y)
  void eval(double x, double y, double* val /*[n][2]*/, double* grad /*[n][2][2] or null*/) const {
    double mv[kMaxNb], mdx[kMaxNb], mdy[kMaxNb];
    for (int m = 0; m < n; ++m) {
      const VMono& t = mono[m];
      mv[m] = std::pow(x, t.p) * std::pow(y, t.q);
      mdx[m] = t.p > 0 ? t.p * std::pow(x, t.p - 1) * std::pow(y, t.q) : 0.0;
      mdy[m] = t.q > 0 ? t.q * std::pow(x, t.p) * std::pow(y, t.q - 1) : 0.0;
    }
    for (int i = 0; i < n; ++i) {
      double v[2] = {0, 0}, g[2][2] = {{0, 0}, {0, 0}};
      for (int m = 0; m < n; ++m) {
        const double c = C[size_t(m) * n + i];
        if (c == 0.0) continue;
        const int comp = mono[m].c;
        v[comp] += c * mv[m];
        g[comp][0] += c * mdx[m];
        g[comp][1] += c * mdy[m];
      }
      val[2 * i] = v[0];
      val[2 * i + 1] = v[1];
      if (grad)
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) grad[4 * i + 2 * a + b] = g[a][b];
    }
  }
};

RefBDM make_ref(int k) {
  RefBDM R;
  R.k = k;
  R.mono = vmonos(k);
  const int n = int(R.mono.size());
  R.n = n;
  if (n > kMaxNb) throw std::runtime_error("BDM: order too high");
  // V[dof][monomial]: the DoF functionals applied to the monomials, in double-double (the edge points
  // (j+1)/(k+2) and the moments a! b! / (a+b+2)! are exact ratios of integers)
  std::vector<DD> V(size_t(n) * n);
  int row = 0;
  for (int e = 0; e < 3; ++e) {
    const double* a = kVert[kEdge[e][0]];
    const double* b = kVert[kEdge[e][1]];
    const double nu[2] = {b[1] - a[1], -(b[0] - a[0])};
    for (int j = 0; j <= k; ++j, ++row) {
      const DD t = dd_ratio(j + 1, k + 2);
      const DD x = dd(a[0]) + t * dd(b[0] - a[0]), y = dd(a[1]) + t * dd(b[1] - a[1]);
      for (int m = 0; m < n; ++m) {
        const VMono& mm = R.mono[m];
        V[size_t(row) * n + m] = dd_pow(x, mm.p) * dd_pow(y, mm.q) * dd(nu[mm.c]);
      }
    }
  }
  for (const auto& q : nedelec(k)) {
    for (int m = 0; m < n; ++m) {
      const VMono& mm = R.mono[m];
      DD s;
      for (const TermD& t : q)
        if (t.c == mm.c)
          s = s + t.w * dd_ratio(fact(mm.p + t.p) * fact(mm.q + t.q), fact(mm.p + t.p + mm.q + t.q + 2));
      V[size_t(row) * n + m] = s;
    }
    ++row;
  }
  if (row != n) throw std::runtime_error("BDM: DoF count mismatch");
  // V C = I
  std::vector<DD> C(size_t(n) * n);
  for (int i = 0; i < n; ++i) C[size_t(i) * n + i] = dd(1.0);
  lu_solve_dd(n, V, C, n);
  R.C.resize(size_t(n) * n);
  for (size_t i = 0; i < C.size(); ++i) R.C[i] = C[i].hi + C[i].lo;
  R.Cd = std::move(C);
  return R;
}

struct Geo {
  double x0[2], J[2][2], Ji[2][2], det;
};

// cell c: lower (i,j),(i+1,j),(i,j+1) for c < N^2, else upper (i+1,j),(i+1,j+1),(i,j+1); vertex ids
void cell_vertices(int N, int c, int v[3][2]) {
  const int q = c % (N * N), i = q % N, j = q / N;
  if (c < N * N) {
    v[0][0] = i; v[0][1] = j; v[1][0] = i + 1; v[1][1] = j; v[2][0] = i; v[2][1] = j + 1;
  } else {
    v[0][0] = i + 1; v[0][1] = j; v[1][0] = i + 1; v[1][1] = j + 1; v[2][0] = i; v[2][1] = j + 1;
  }
}

Geo geometry(const int v[3][2], double h) {
  Geo g;
  g.x0[0] = h * v[0][0];
  g.x0[1] = h * v[0][1];
  g.J[0][0] = h * (v[1][0] - v[0][0]);
  g.J[0][1] = h * (v[2][0] - v[0][0]);
  g.J[1][0] = h * (v[1][1] - v[0][1]);
  g.J[1][1] = h * (v[2][1] - v[0][1]);
  g.det = g.J[0][0] * g.J[1][1] - g.J[0][1] * g.J[1][0];
  g.Ji[0][0] = g.J[1][1] / g.det;
  g.Ji[0][1] = -g.J[0][1] / g.det;
  g.Ji[1][0] = -g.J[1][0] / g.det;
  g.Ji[1][1] = g.J[0][0] / g.det;
  return g;
}

// Mesh combinatorics of the DoF layout.
struct BdmMesh {
  int N, k, nh, nvv, ndg, nedge, ncell, per_e, per_c, nq, n_edge, n_int, n_u, n_p, ndof;
  explicit BdmMesh(int N_, int k_) : N(N_), k(k_) {
    nh = N * (N + 1);
    nvv = N * (N + 1);
    ndg = N * N;
    nedge = nh + nvv + ndg;
    ncell = 2 * N * N;
    per_e = k + 1;
    per_c = (k + 1) * (k - 1);
    nq = k * (k + 1) / 2;
    n_edge = nedge * per_e;
    n_int = ncell * per_c;
    n_u = n_edge + n_int;
    n_p = ncell * nq;
    ndof = n_u + n_p;
  }
  int vid(int x, int y) const { return y * (N + 1) + x; }
  // edge index of the segment between two vertices (any order)
  int edge(int ax, int ay, int bx, int by) const {
    if (ay == by) return std::min(ay, by) * N + std::min(ax, bx);                        // horizontal
    if (ax == bx) return nh + std::min(ay, by) * (N + 1) + ax;                            // vertical
    // diagonal (i+1, j) - (i, j+1)
    const int j = std::min(ay, by), i = std::min(ax, bx);
    return nh + nvv + j * N + i;
  }
  // the edge's endpoints in orientation order (lower vertex id first)
  void edge_ends(int e, int& ax, int& ay, int& bx, int& by) const {
    if (e < nh) {
      const int j = e / N, i = e % N;
      ax = i; ay = j; bx = i + 1; by = j;
    } else if (e < nh + nvv) {
      const int q = e - nh, j = q / (N + 1), i = q % (N + 1);
      ax = i; ay = j; bx = i; by = j + 1;
    } else {
      const int q = e - nh - nvv, j = q / N, i = q % N;
      ax = i + 1; ay = j; bx = i; by = j + 1;   // vid(i+1, j) < vid(i, j+1)
    }
    if (vid(ax, ay) > vid(bx, by)) {
      std::swap(ax, bx);
      std::swap(ay, by);
    }
  }
  // local DoFs of cell c: global index and sign, velocity first; then the pressure DoFs
  void cell_dofs(int c, std::vector<int>& dof, std::vector<double>& sgn) const {
    int v[3][2];
    cell_vertices(N, c, v);
    dof.clear();
    sgn.clear();
    for (int e = 0; e < 3; ++e) {
      const int* a = v[kEdge[e][0]];
      const int* b = v[kEdge[e][1]];
      const int ge = edge(a[0], a[1], b[0], b[1]);
      const bool same = vid(a[0], a[1]) < vid(b[0], b[1]);
      for (int j = 0; j <= k; ++j) {
        dof.push_back(ge * per_e + (same ? j : k - j));
        sgn.push_back(same ? 1.0 : -1.0);
      }
    }
    for (int m = 0; m < per_c; ++m) {
      dof.push_back(n_edge + c * per_c + m);
      sgn.push_back(1.0);
    }
  }
  int pdof(int c, int m) const { return n_u + c * nq + m; }
};

// P_{k-1} pressure basis (equispaced nodes, t outer / s inner) at a reference point
void pressure_basis(int k, double x, double y, double* out) {
  const int d = k - 1;
  if (d == 0) {
    out[0] = 1.0;
    return;
  }
  std::vector<std::array<int, 3>> al;
  for (int t = 0; t <= d; ++t)
    for (int s = 0; s + t <= d; ++s) al.push_back({d - s - t, s, t});
  const double lam[3] = {1.0 - x - y, x, y};
  for (size_t a = 0; a < al.size(); ++a) {
    double v = 1.0;
    for (int i = 0; i < 3; ++i)
      for (int m = 1; m <= al[a][i]; ++m) v *= (d * lam[i] - (m - 1)) / m;
    out[a] = v;
  }
}

// Gauss-Legendre on [0, 1] by Newton on the three-term recurrence (independent of host_fem's copy)
void gauss01(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int n = 2; n <= q; ++n) {
        const double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (z + 1.0);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct Trip {
  int r, c;
  double v;
};

void to_csr(int n, int m, std::vector<Trip>& t, HostCsr& A, double drop) {
  std::sort(t.begin(), t.end(), [](const Trip& a, const Trip& b) { return a.r != b.r ? a.r < b.r : a.c < b.c; });
  A.nrows = n;
  A.ncols = m;
  A.ptr.assign(n + 1, 0);
  A.col.clear();
  A.val.clear();
  for (size_t e = 0; e < t.size();) {
    size_t f = e;
    double s = 0.0;
    while (f < t.size() && t[f].r == t[e].r && t[f].c == t[e].c) s += t[f++].v;
    if (std::fabs(s) > drop || drop < 0) {
      A.ptr[t[e].r + 1]++;
      A.col.push_back(t[e].c);
      A.val.push_back(s);
    }
    e = f;
  }
  for (int i = 0; i < n; ++i) A.ptr[i + 1] += A.ptr[i];
}

// Cell block of one cell shape without DoF signs: A_e = 2 nu int eps(phi_j):eps(phi_i) (nb x nb) and
// B_e = -int psi_q div phi_i (nq x nb), collapsed Gauss rule of k + 2 points per direction.
void cell_block(const RefBDM& R, int k, const Geo& G, double nu, std::vector<double>& Ae, std::vector<double>& Be) {
  const int nb = R.n, nq = k * (k + 1) / 2;
  Ae.assign(size_t(nb) * nb, 0.0);
  Be.assign(size_t(nq) * nb, 0.0);
  std::vector<double> gx, gw, val(2 * nb), grad(4 * nb), ps(nq), dv(nb);
  std::vector<std::array<double, 3>> eps(nb);   // e11, e22, e12 of each Piola-mapped function
  gauss01(k + 2, gx, gw);
  for (int iu = 0; iu < k + 2; ++iu)
    for (int iv = 0; iv < k + 2; ++iv) {
      const double xr = gx[iu], yr = gx[iv] * (1.0 - gx[iu]);
      const double w = gw[iu] * gw[iv] * (1.0 - gx[iu]) * std::fabs(G.det);
      R.eval(xr, yr, val.data(), grad.data());
      pressure_basis(k, xr, yr, ps.data());
      for (int i = 0; i < nb; ++i) {
        double gp[2][2];   // physical gradient J (grad vhat) J^{-1} / det J
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            double s = 0.0;
            for (int p = 0; p < 2; ++p)
              for (int q = 0; q < 2; ++q) s += G.J[a][p] * grad[4 * i + 2 * p + q] * G.Ji[q][b];
            gp[a][b] = s / G.det;
          }
        eps[i] = {gp[0][0], gp[1][1], 0.5 * (gp[0][1] + gp[1][0])};
        dv[i] = gp[0][0] + gp[1][1];
      }
      for (int i = 0; i < nb; ++i) {
        for (int j = 0; j < nb; ++j)
          Ae[size_t(i) * nb + j] +=
              2.0 * nu * w * (eps[i][0] * eps[j][0] + eps[i][1] * eps[j][1] + 2.0 * eps[i][2] * eps[j][2]);
        for (int q = 0; q < nq; ++q) Be[size_t(q) * nb + i] -= w * ps[q] * dv[i];
      }
    }
}

// Interior-edge block of Eq. (DiscontBilinearForm) without DoF signs, over the functions of the two
// cells (c1's first): with jt(w) = (w_1 - w_2) . t and the average {eps} taken against t (.) n_1,
//   -2 nu int [ jt(v) t^T{eps(u)}n_1 + jt(u) t^T{eps(v)}n_1 ] + (2 nu alpha / h_e) int jt(u) jt(v) / 2
// by Gauss-Legendre with k + 1 points.
void edge_block(const RefBDM& R, int k, const double A[2], const double B[2], const Geo G[2], double nu, double alpha,
                std::vector<double>& Ee) {
  const int nb = R.n, nn = 2 * nb;
  const double tau[2] = {B[0] - A[0], B[1] - A[1]};
  const double he = std::hypot(tau[0], tau[1]);
  const double tt[2] = {tau[0] / he, tau[1] / he};
  // outward normal of c1: the unit normal pointing away from c1's centroid
  const double cx = G[0].x0[0] + (G[0].J[0][0] + G[0].J[0][1]) / 3.0;
  const double cy = G[0].x0[1] + (G[0].J[1][0] + G[0].J[1][1]) / 3.0;
  double n1[2] = {tt[1], -tt[0]};
  if (n1[0] * (cx - A[0]) + n1[1] * (cy - A[1]) > 0) {
    n1[0] = -n1[0];
    n1[1] = -n1[1];
  }
  std::vector<double> ex, ew, val(2 * nb), grad(4 * nb);
  gauss01(k + 1, ex, ew);
  std::vector<double> JT(size_t(k + 1) * nn), AV(size_t(k + 1) * nn);
  for (int side = 0; side < 2; ++side) {
    const Geo& g = G[side];
    for (int p = 0; p <= k; ++p) {
      const double dx = A[0] + ex[p] * tau[0] - g.x0[0], dy = A[1] + ex[p] * tau[1] - g.x0[1];
      R.eval(g.Ji[0][0] * dx + g.Ji[0][1] * dy, g.Ji[1][0] * dx + g.Ji[1][1] * dy, val.data(), grad.data());
      for (int i = 0; i < nb; ++i) {
        double vp[2], gp[2][2];
        for (int a = 0; a < 2; ++a) vp[a] = (g.J[a][0] * val[2 * i] + g.J[a][1] * val[2 * i + 1]) / g.det;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            double s = 0.0;
            for (int pp = 0; pp < 2; ++pp)
              for (int q = 0; q < 2; ++q) s += g.J[a][pp] * grad[4 * i + 2 * pp + q] * g.Ji[q][b];
            gp[a][b] = s / g.det;
          }
        double ten = 0.0;   // t^T eps n_1 with eps = (gp + gp^T) / 2
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) ten += tt[a] * 0.5 * (gp[a][b] + gp[b][a]) * n1[b];
        JT[size_t(p) * nn + side * nb + i] = (side == 0 ? 1.0 : -1.0) * (vp[0] * tt[0] + vp[1] * tt[1]);
        AV[size_t(p) * nn + side * nb + i] = 0.5 * ten;
      }
    }
  }
  Ee.assign(size_t(nn) * nn, 0.0);
  for (int i = 0; i < nn; ++i)
    for (int j = 0; j < nn; ++j) {
      double s = 0.0;
      for (int p = 0; p <= k; ++p) {
        const double* jt = &JT[size_t(p) * nn];
        const double* av = &AV[size_t(p) * nn];
        s += ew[p] * he * (-2.0 * nu * (av[j] * jt[i] + jt[j] * av[i]) + nu * alpha / he * jt[j] * jt[i]);
      }
      Ee[size_t(i) * nn + j] = s;
    }
}

// Run f(t, lo, hi) over the nthreads consecutive chunks of [0, n), one thread each.
template <class F>
void chunks(int n, int nthreads, F&& f) {
  std::vector<std::thread> th;
  std::vector<std::exception_ptr> err(nthreads);   // a worker's exception goes to the caller
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      try {
        f(t, int(int64_t(n) * t / nthreads), int(int64_t(n) * (t + 1) / nthreads));
      } catch (...) {
        err[t] = std::current_exception();
      }
    });
  for (auto& x : th) x.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

}  // namespace

void build_level_bdm(int N, int k, double nu, bool with_patches, int nthreads, HostLevel& L) {
  if (k < 1 || k > 5) throw std::runtime_error("BDM order k must be in 1..5");
  const BdmMesh M(N, k);
  const RefBDM R = make_ref(k);
  const int nb = R.n, nq = M.nq, nn = 2 * nb;
  L.N = N;
  L.k = k;
  L.cell = 2;
  L.ncell_lower = N * N;
  L.nv1 = L.np1 = 0;
  L.n_u = M.n_u;
  L.n_p = M.n_p;
  L.ndof = M.ndof;
  const double h = 1.0 / N, alpha = double((k + 1) * (k + 2));
  // no-flux rows: the DoFs of boundary edges
  L.dir.assign(L.ndof, 0);
  for (int e = 0; e < M.nedge; ++e) {
    int ax, ay, bx, by;
    M.edge_ends(e, ax, ay, bx, by);
    const bool bnd = (ax == bx && (ax == 0 || ax == N)) || (ay == by && (ay == 0 || ay == N));
    if (bnd)
      for (int j = 0; j <= k; ++j) L.dir[e * M.per_e + j] = 1;
  }
  // cells of each edge (ascending) and the edge type: 0 horizontal, 1 vertical, 2 diagonal
  std::vector<int> c_of_e(size_t(M.nedge) * 2, -1);
  for (int c = 0; c < M.ncell; ++c) {
    int v[3][2];
    cell_vertices(N, c, v);
    for (int e = 0; e < 3; ++e) {
      const int* a = v[kEdge[e][0]];
      const int* b = v[kEdge[e][1]];
      const int ge = M.edge(a[0], a[1], b[0], b[1]);
      (c_of_e[2 * ge] < 0 ? c_of_e[2 * ge] : c_of_e[2 * ge + 1]) = c;
    }
  }
  auto etype = [&](int e) { return e < M.nh ? 0 : e < M.nh + M.nvv ? 1 : 2; };
  // The mesh is a lattice of two cell shapes, and every interior edge of one type joins a lower cell
  // (c1) to an upper cell (c2) in the same local position: one block per shape and per edge type,
  // computed on its first occurrence.
  std::vector<double> Ae[2], Be[2], Ee[3];
  for (int s = 0; s < 2; ++s) {
    int v[3][2];
    cell_vertices(N, s * N * N, v);
    cell_block(R, k, geometry(v, h), nu, Ae[s], Be[s]);
  }
  for (int e = 0; e < M.nedge; ++e) {
    const int t = etype(e);
    if (c_of_e[2 * e + 1] < 0 || !Ee[t].empty()) continue;
    int ax, ay, bx, by;
    M.edge_ends(e, ax, ay, bx, by);
    const double A[2] = {h * ax, h * ay}, B[2] = {h * bx, h * by};
    Geo G[2];
    for (int s = 0; s < 2; ++s) {
      int v[3][2];
      cell_vertices(N, c_of_e[2 * e + s], v);
      G[s] = geometry(v, h);
    }
    edge_block(R, k, A, B, G, nu, alpha, Ee[t]);
  }
  // row incidences: (kind, block, local index); kind 0 velocity of a cell, 1 pressure of a cell,
  // 2 one of the 2 nb functions of an interior edge's cell pair
  struct Inc {
    int kind, id, li;
  };
  std::vector<int> iptr(L.ndof + 1, 0);
  std::vector<int> dof;
  std::vector<double> sgn;
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int> fill;
    std::vector<Inc> inc;
    if (pass == 1) {
      for (int r = 0; r < L.ndof; ++r) iptr[r + 1] += iptr[r];
      fill.assign(iptr.begin(), iptr.end() - 1);
      inc.resize(iptr.back());
    }
    auto add = [&](int r, int kind, int id, int li) {
      if (pass == 0)
        iptr[r + 1]++;
      else
        inc[fill[r]++] = {kind, id, li};
    };
    for (int c = 0; c < M.ncell; ++c) {
      M.cell_dofs(c, dof, sgn);
      for (int i = 0; i < nb; ++i) add(dof[i], 0, c, i);
      for (int q = 0; q < nq; ++q) add(M.pdof(c, q), 1, c, q);
    }
    for (int e = 0; e < M.nedge; ++e) {
      if (c_of_e[2 * e + 1] < 0) continue;
      for (int s = 0; s < 2; ++s) {
        M.cell_dofs(c_of_e[2 * e + s], dof, sgn);
        for (int i = 0; i < nb; ++i) add(dof[i], 2, e, s * nb + i);
      }
    }
    if (pass == 1) {
      // rows: sum of the contributions of every incident block; Dirichlet rows become identity rows and
      // Dirichlet columns are dropped
      std::vector<std::vector<int>> tcol(std::max(1, std::min(nthreads, L.ndof / 2048 + 1)));
      std::vector<std::vector<double>> tval(tcol.size());
      std::vector<int> rowlen(L.ndof, 0);
      const int nt = int(tcol.size());
      chunks(L.ndof, nt, [&](int t, int lo, int hi) {
        std::vector<int>& oc = tcol[t];
        std::vector<double>& ov = tval[t];
        std::vector<std::pair<int, double>> acc;
        std::vector<int> d1, d2;
        std::vector<double> s1, s2;
        for (int r = lo; r < hi; ++r) {
          if (L.dir[r]) {
            oc.push_back(r);
            ov.push_back(1.0);
            rowlen[r] = 1;
            continue;
          }
          acc.clear();
          for (int x = iptr[r]; x < iptr[r + 1]; ++x) {
            const Inc& I = inc[x];
            if (I.kind == 2) {
              M.cell_dofs(c_of_e[2 * I.id], d1, s1);
              M.cell_dofs(c_of_e[2 * I.id + 1], d2, s2);
              const double si = I.li < nb ? s1[I.li] : s2[I.li - nb];
              const double* E = Ee[etype(I.id)].data() + size_t(I.li) * nn;
              for (int j = 0; j < nn; ++j) {
                const int g = j < nb ? d1[j] : d2[j - nb];
                if (!L.dir[g]) acc.push_back({g, si * (j < nb ? s1[j] : s2[j - nb]) * E[j]});
              }
              continue;
            }
            M.cell_dofs(I.id, d1, s1);
            const int sh = I.id < N * N ? 0 : 1;
            if (I.kind == 0) {
              const double si = s1[I.li];
              for (int j = 0; j < nb; ++j)
                if (!L.dir[d1[j]]) acc.push_back({d1[j], si * s1[j] * Ae[sh][size_t(I.li) * nb + j]});
              for (int q = 0; q < nq; ++q) acc.push_back({M.pdof(I.id, q), si * Be[sh][size_t(q) * nb + I.li]});
            } else {
              for (int j = 0; j < nb; ++j)
                if (!L.dir[d1[j]]) acc.push_back({d1[j], s1[j] * Be[sh][size_t(I.li) * nb + j]});
            }
          }
          std::sort(acc.begin(), acc.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
          int n = 0;
          for (size_t a = 0; a < acc.size();) {
            size_t b = a;
            double s = 0.0;
            while (b < acc.size() && acc[b].first == acc[a].first) s += acc[b++].second;
            if (s != 0.0) {
              oc.push_back(acc[a].first);
              ov.push_back(s);
              ++n;
            }
            a = b;
          }
          rowlen[r] = n;
        }
      });
      L.A.nrows = L.A.ncols = L.ndof;
      L.A.ptr.assign(L.ndof + 1, 0);
      for (int r = 0; r < L.ndof; ++r) L.A.ptr[r + 1] = L.A.ptr[r] + rowlen[r];
      L.A.col.clear();
      L.A.val.clear();
      L.A.col.reserve(L.A.ptr.back());
      L.A.val.reserve(L.A.ptr.back());
      for (int t = 0; t < nt; ++t) {
        L.A.col.insert(L.A.col.end(), tcol[t].begin(), tcol[t].end());
        L.A.val.insert(L.A.val.end(), tval[t].begin(), tval[t].end());
      }
    }
  }
  if (!with_patches) return;
  // extended cell patches (Sec. 3.1): each cell's pressures and the free velocity DoFs of the cell
  // and of its edge neighbours, ascending
  L.patch_ptr.assign(1, 0);
  L.patch_dofs.clear();
  L.patch_kind.clear();
  std::vector<int> vel;
  for (int c = 0; c < M.ncell; ++c) {
    int v[3][2];
    cell_vertices(N, c, v);
    std::vector<int> nbr = {c};
    for (int e = 0; e < 3; ++e) {
      const int* a = v[kEdge[e][0]];
      const int* b = v[kEdge[e][1]];
      const int ge = M.edge(a[0], a[1], b[0], b[1]);
      for (int s = 0; s < 2; ++s)
        if (c_of_e[2 * ge + s] >= 0) nbr.push_back(c_of_e[2 * ge + s]);
    }
    vel.clear();
    for (int d : nbr) {
      M.cell_dofs(d, dof, sgn);
      for (int g : dof)
        if (!L.dir[g]) vel.push_back(g);
    }
    std::sort(vel.begin(), vel.end());
    vel.erase(std::unique(vel.begin(), vel.end()), vel.end());
    for (int q = 0; q < nq; ++q) vel.push_back(M.pdof(c, q));
    L.patch_dofs.insert(L.patch_dofs.end(), vel.begin(), vel.end());
    L.patch_ptr.push_back(int(L.patch_dofs.size()));
    L.patch_kind.push_back(2);
  }
}

// Transfers between nested BDM levels (Sec. 3: the canonical interpolation of the natural embedding):
// every fine DoF functional applied to every coarse basis function.  The values are ratios of
// integers that the FP64 evaluation of the high-order basis would spoil by cancellation, so they are
// formed in double-double and rounded once: normal fluxes at the fine edge points, the moments of the
// pulled-back coarse function on each fine cell integrated exactly monomial by monomial, and the coarse
// pressure at the fine nodes.  The mesh is a lattice, so each local block depends only on the position
// of the fine point or cell inside its coarse cell and is computed once.
void build_transfer_bdm(const HostLevel& c, HostLevel& f) {
  const int k = f.k, Nc = c.N, Nf = f.N;
  if (Nf != 2 * Nc || c.k != k || c.cell != 2) throw std::runtime_error("BDM transfer: levels not nested");
  const BdmMesh Mc(Nc, k), Mf(Nf, k);
  const RefBDM R = make_ref(k);
  const int nb = R.n, nq = Mc.nq, dq = k - 1;
  const int D = 2 * (k + 2);   // fine edge points are multiples of 1 / D of the coarse width
  std::vector<Trip> t;
  std::vector<int> dof;
  std::vector<double> sgn;
  // coarse cell containing the point (X, Y) / S (coarse units; lower triangle on its diagonal), exact
  auto coarse_cell = [&](int64_t X, int64_t Y, int64_t S) {
    const int i = int(std::min<int64_t>(X / S, Nc - 1)), j = int(std::min<int64_t>(Y / S, Nc - 1));
    return (X - i * S) + (Y - j * S) <= S ? j * Nc + i : Nc * Nc + j * Nc + i;
  };
  // coarse-unit Piola values J vhat / det J (J integer) of the reference basis of coarse cell cc at the
  // point (X, Y) / S, in double-double
  auto coarse_vals = [&](int cc, int64_t X, int64_t Y, int64_t S, std::vector<DD>& out) {
    int v[3][2];
    cell_vertices(Nc, cc, v);
    const int J[2][2] = {{v[1][0] - v[0][0], v[2][0] - v[0][0]}, {v[1][1] - v[0][1], v[2][1] - v[0][1]}};
    const int det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const int64_t dx = X - v[0][0] * S, dy = Y - v[0][1] * S;
    const DD xr = dd_ratio(double((J[1][1] * dx - J[0][1] * dy) * det), double(S));   // det = +-1
    const DD yr = dd_ratio(double((-J[1][0] * dx + J[0][0] * dy) * det), double(S));
    std::vector<DD> xp(k + 1), yp(k + 1);
    xp[0] = yp[0] = dd(1.0);
    for (int p = 1; p <= k; ++p) {
      xp[p] = xp[p - 1] * xr;
      yp[p] = yp[p - 1] * yr;
    }
    out.assign(2 * nb, DD{});
    for (int i = 0; i < nb; ++i) {
      DD vh[2];
      for (int m = 0; m < nb; ++m) {
        const VMono& mm = R.mono[m];
        vh[mm.c] = vh[mm.c] + R.Cd[size_t(m) * nb + i] * (xp[mm.p] * yp[mm.q]);
      }
      for (int a = 0; a < 2; ++a) out[2 * i + a] = (dd(J[a][0]) * vh[0] + dd(J[a][1]) * vh[1]) * dd(det);
    }
  };
  // fine edge DoFs: the normal flux with rot(x_b - x_a) of the fine edge, in coarse units half of the
  // fine-unit vector; one block per (coarse cell shape, position in it, edge direction)
  std::map<std::array<int64_t, 5>, std::vector<double>> edge_memo;
  std::vector<DD> cv;
  for (int e = 0; e < Mf.nedge; ++e) {
    int ax, ay, bx, by;
    Mf.edge_ends(e, ax, ay, bx, by);
    for (int j = 0; j <= k; ++j) {
      // the point a + (j+1)/(k+2) (b - a) (fine units) in units of 1 / D of the coarse width: (k+2) a + (j+1)(b - a)
      const int64_t X = int64_t(ax) * (k + 2) + int64_t(j + 1) * (bx - ax);
      const int64_t Y = int64_t(ay) * (k + 2) + int64_t(j + 1) * (by - ay);
      const int cc = coarse_cell(X, Y, D);
      int v[3][2];
      cell_vertices(Nc, cc, v);
      const std::array<int64_t, 5> key = {cc < Nc * Nc ? 0 : 1, X - int64_t(v[0][0]) * D, Y - int64_t(v[0][1]) * D,
                                          bx - ax, by - ay};
      auto it = edge_memo.find(key);
      if (it == edge_memo.end()) {
        coarse_vals(cc, X, Y, D, cv);
        std::vector<double> val(nb);
        const DD nux = dd_ratio(by - ay, 2), nuy = dd_ratio(-(bx - ax), 2);
        for (int i = 0; i < nb; ++i) {
          const DD s = cv[2 * i] * nux + cv[2 * i + 1] * nuy;
          val[i] = s.hi + s.lo;
        }
        it = edge_memo.emplace(key, std::move(val)).first;
      }
      Mc.cell_dofs(cc, dof, sgn);
      for (int i = 0; i < nb; ++i)
        if (std::fabs(it->second[i]) > 1e-12) t.push_back({e * Mf.per_e + j, dof[i], sgn[i] * it->second[i]});
    }
  }
  // fine interior DoFs: int over the fine reference cell of (pulled-back coarse function) . q for the
  // Nedelec functions q.  With the fine cell's vertices f0 + Jf xhat (fine units) and the coarse cell's
  // c0 + Jc xhat (coarse units), the coarse reference coordinates are affine in the fine ones with
  // coefficients in Z / 2, the coarse basis is a polynomial there, and the pulled-back field is
  // adj(Jf) Jc vhat / (2 det Jc); the moments follow from int x^a y^b = a! b! / (a+b+2)!.
  const auto ned = nedelec(k);
  const int ni = Mf.per_c;
  const int dg = 2 * k;   // polynomial degree bound of the products
  auto pidx = [&](int p, int q) { return p * (dg + 1) + q; };
  std::map<std::array<int, 4>, std::vector<double>> mom_memo;
  for (int fc = 0; fc < Mf.ncell && ni > 0; ++fc) {
    int vf[3][2];
    cell_vertices(Nf, fc, vf);
    // fine centroid in coarse units: (sum of the fine vertices) / 6
    const int64_t sx = vf[0][0] + vf[1][0] + vf[2][0], sy = vf[0][1] + vf[1][1] + vf[2][1];
    const int cc = coarse_cell(sx, sy, 6);
    int vc[3][2];
    cell_vertices(Nc, cc, vc);
    const std::array<int, 4> key = {cc < Nc * Nc ? 0 : 1, fc < Nf * Nf ? 0 : 1, vf[0][0] - 2 * vc[0][0],
                                    vf[0][1] - 2 * vc[0][1]};
    auto it = mom_memo.find(key);
    if (it == mom_memo.end()) {
      const int Jf[2][2] = {{vf[1][0] - vf[0][0], vf[2][0] - vf[0][0]}, {vf[1][1] - vf[0][1], vf[2][1] - vf[0][1]}};
      const int Jc[2][2] = {{vc[1][0] - vc[0][0], vc[2][0] - vc[0][0]}, {vc[1][1] - vc[0][1], vc[2][1] - vc[0][1]}};
      const int detc = Jc[0][0] * Jc[1][1] - Jc[0][1] * Jc[1][0];
      // X (coarse units) = (f0 + Jf xf) / 2; coarse reference = adj(Jc) (X - c0) / det Jc
      const double o[2] = {0.5 * key[2], 0.5 * key[3]};   // f0 / 2 - c0
      const int adjc[2][2] = {{Jc[1][1], -Jc[0][1]}, {-Jc[1][0], Jc[0][0]}};
      std::vector<DD> xc(size_t(dg + 1) * (dg + 1)), yc(xc.size());
      for (int a = 0; a < 2; ++a) {
        std::vector<DD>& P = a == 0 ? xc : yc;
        P[pidx(0, 0)] = dd((adjc[a][0] * o[0] + adjc[a][1] * o[1]) * detc);
        P[pidx(1, 0)] = dd(0.5 * (adjc[a][0] * Jf[0][0] + adjc[a][1] * Jf[1][0]) * detc);
        P[pidx(0, 1)] = dd(0.5 * (adjc[a][0] * Jf[0][1] + adjc[a][1] * Jf[1][1]) * detc);
      }
      auto mul = [&](const std::vector<DD>& A, const std::vector<DD>& B) {
        std::vector<DD> C(A.size());
        for (int p = 0; p <= dg; ++p)
          for (int q = 0; p + q <= dg; ++q) {
            if (A[pidx(p, q)].hi == 0.0) continue;
            for (int r = 0; p + r <= dg; ++r)
              for (int s = 0; p + r + q + s <= dg; ++s)
                if (B[pidx(r, s)].hi != 0.0) C[pidx(p + r, q + s)] = C[pidx(p + r, q + s)] + A[pidx(p, q)] * B[pidx(r, s)];
          }
        return C;
      };
      std::vector<std::vector<DD>> xpow(k + 1), ypow(k + 1);
      xpow[0] = ypow[0] = std::vector<DD>(xc.size());
      xpow[0][0] = ypow[0][0] = dd(1.0);
      for (int p = 1; p <= k; ++p) {
        xpow[p] = mul(xpow[p - 1], xc);
        ypow[p] = mul(ypow[p - 1], yc);
      }
      std::vector<std::vector<DD>> mono(nb);
      for (int m = 0; m < nb; ++m) mono[m] = mul(xpow[R.mono[m].p], ypow[R.mono[m].q]);
      // pulled-back field: M vhat with M = adj(Jf) Jc / (2 det Jc)
      const int adjf[2][2] = {{Jf[1][1], -Jf[0][1]}, {-Jf[1][0], Jf[0][0]}};
      double M[2][2];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) M[a][b] = 0.5 * (adjf[a][0] * Jc[0][b] + adjf[a][1] * Jc[1][b]) / detc;
      std::vector<DD> intg(size_t(dg + 1) * (dg + 1));
      for (int p = 0; p <= dg; ++p)
        for (int q = 0; p + q <= dg; ++q) intg[pidx(p, q)] = dd_ratio(fact(p) * fact(q), fact(p + q + 2));
      std::vector<double> blk(size_t(ni) * nb);
      std::vector<DD> vh[2], u[2];
      for (int i = 0; i < nb; ++i) {
        for (int b = 0; b < 2; ++b) vh[b].assign(xc.size(), DD{});
        for (int m = 0; m < nb; ++m) {
          const DD cm = R.Cd[size_t(m) * nb + i];
          if (cm.hi == 0.0) continue;
          std::vector<DD>& V = vh[R.mono[m].c];
          for (size_t x = 0; x < V.size(); ++x)
            if (mono[m][x].hi != 0.0) V[x] = V[x] + cm * mono[m][x];
        }
        for (int a = 0; a < 2; ++a) {
          u[a].assign(xc.size(), DD{});
          for (size_t x = 0; x < xc.size(); ++x) u[a][x] = dd(M[a][0]) * vh[0][x] + dd(M[a][1]) * vh[1][x];
        }
        for (int m = 0; m < ni; ++m) {
          DD s;
          for (const TermD& tm : ned[m])
            for (int p = 0; p + tm.p <= dg; ++p)
              for (int q = 0; p + q + tm.p + tm.q <= dg; ++q) {
                const DD cf = u[tm.c][pidx(p, q)];
                if (cf.hi != 0.0) s = s + tm.w * cf * intg[pidx(p + tm.p, q + tm.q)];
              }
          blk[size_t(m) * nb + i] = s.hi + s.lo;
        }
      }
      it = mom_memo.emplace(key, std::move(blk)).first;
    }
    Mc.cell_dofs(cc, dof, sgn);
    for (int m = 0; m < ni; ++m)
      for (int i = 0; i < nb; ++i) {
        const double v = it->second[size_t(m) * nb + i];
        if (std::fabs(v) > 1e-12) t.push_back({Mf.n_edge + fc * ni + m, dof[i], sgn[i] * v});
      }
  }
  // pressure: the coarse P_{k-1} Lagrange basis at the fine nodes (fine node (s, t) / (k - 1) of the
  // fine reference cell; the centroid for k = 1), in the coarse cell of the fine centroid
  std::vector<double> ps(nq);
  for (int fc = 0; fc < Mf.ncell; ++fc) {
    int vf[3][2];
    cell_vertices(Nf, fc, vf);
    const int cc = coarse_cell(vf[0][0] + vf[1][0] + vf[2][0], vf[0][1] + vf[1][1] + vf[2][1], 6);
    int vc[3][2];
    cell_vertices(Nc, cc, vc);
    const int Jc[2][2] = {{vc[1][0] - vc[0][0], vc[2][0] - vc[0][0]}, {vc[1][1] - vc[0][1], vc[2][1] - vc[0][1]}};
    const int detc = Jc[0][0] * Jc[1][1] - Jc[0][1] * Jc[1][0];
    int m = 0;
    for (int tt = 0; tt <= dq; ++tt)
      for (int s = 0; s + tt <= dq; ++s, ++m) {
        // node in units of 1 / S coarse: S = 2 d (d = k - 1), or 6 for the centroid
        const int S = dq == 0 ? 6 : 2 * dq;
        int64_t X, Y;
        if (dq == 0) {
          X = vf[0][0] + vf[1][0] + vf[2][0];
          Y = vf[0][1] + vf[1][1] + vf[2][1];
        } else {
          X = int64_t(vf[0][0]) * dq + (vf[1][0] - vf[0][0]) * s + (vf[2][0] - vf[0][0]) * tt;
          Y = int64_t(vf[0][1]) * dq + (vf[1][1] - vf[0][1]) * s + (vf[2][1] - vf[0][1]) * tt;
        }
        const int64_t dx = X - int64_t(vc[0][0]) * S, dy = Y - int64_t(vc[0][1]) * S;
        const double xr = double((Jc[1][1] * dx - Jc[0][1] * dy) * detc) / S;
        const double yr = double((-Jc[1][0] * dx + Jc[0][0] * dy) * detc) / S;
        pressure_basis(k, xr, yr, ps.data());
        for (int q = 0; q < nq; ++q)
          if (std::fabs(ps[q]) > 1e-12) t.push_back({Mf.pdof(fc, m), Mc.pdof(cc, q), ps[q]});
      }
  }
  to_csr(f.ndof, c.ndof, t, f.P, -1.0);
  HostCsr& Rm = f.R;
  Rm.nrows = c.ndof;
  Rm.ncols = f.ndof;
  Rm.ptr.assign(Rm.nrows + 1, 0);
  for (int cc : f.P.col) Rm.ptr[cc + 1]++;
  for (int i = 0; i < Rm.nrows; ++i) Rm.ptr[i + 1] += Rm.ptr[i];
  Rm.col.resize(f.P.col.size());
  Rm.val.resize(f.P.col.size());
  std::vector<int> fill(Rm.ptr.begin(), Rm.ptr.end() - 1);
  for (int r = 0; r < f.P.nrows; ++r)
    for (int e = f.P.ptr[r]; e < f.P.ptr[r + 1]; ++e) {
      const int pos = fill[f.P.col[e]]++;
      Rm.col[pos] = r;
      Rm.val[pos] = f.P.val[e];
    }
}

// Load vector of the manufactured problem of Eq. (model_problem): f = 2 pi^2 nu u with
// u = (sin pi x cos pi y, -cos pi x sin pi y), p = 0, against the Piola-mapped basis (collapsed rule of
// k + 5 points per direction); u . n = 0 on the boundary, so the no-flux rows carry zero.
void manufactured_rhs_bdm(const HostLevel& L, double nu, std::vector<double>& b) {
  const int N = L.N, k = L.k;
  const BdmMesh M(N, k);
  const RefBDM R = make_ref(k);
  const int nb = R.n;
  const double h = 1.0 / N, pi = M_PI;
  std::vector<double> gx, gw, val(2 * nb);
  gauss01(k + 5, gx, gw);
  std::vector<int> dof;
  std::vector<double> sgn, loc(nb);
  b.assign(L.ndof, 0.0);
  for (int c = 0; c < M.ncell; ++c) {
    int v[3][2];
    cell_vertices(N, c, v);
    const Geo G = geometry(v, h);
    std::fill(loc.begin(), loc.end(), 0.0);
    for (size_t iu = 0; iu < gx.size(); ++iu)
      for (size_t iv = 0; iv < gx.size(); ++iv) {
        const double xr = gx[iu], yr = gx[iv] * (1.0 - gx[iu]);
        const double w = gw[iu] * gw[iv] * (1.0 - gx[iu]) * std::fabs(G.det);
        const double X = G.x0[0] + G.J[0][0] * xr + G.J[0][1] * yr, Y = G.x0[1] + G.J[1][0] * xr + G.J[1][1] * yr;
        const double f1 = 2 * pi * pi * nu * std::sin(pi * X) * std::cos(pi * Y);
        const double f2 = -2 * pi * pi * nu * std::cos(pi * X) * std::sin(pi * Y);
        R.eval(xr, yr, val.data(), nullptr);
        for (int i = 0; i < nb; ++i) {
          const double v1 = (G.J[0][0] * val[2 * i] + G.J[0][1] * val[2 * i + 1]) / G.det;
          const double v2 = (G.J[1][0] * val[2 * i] + G.J[1][1] * val[2 * i + 1]) / G.det;
          loc[i] += w * (v1 * f1 + v2 * f2);
        }
      }
    M.cell_dofs(c, dof, sgn);
    for (int i = 0; i < nb; ++i) b[dof[i]] += sgn[i] * loc[i];
  }
  for (int r = 0; r < L.ndof; ++r)
    if (L.dir[r]) b[r] = 0.0;
}

// Tables of the error integrals of vk_errors on the (BDM_k, dP_{k-1}) level: per cell its velocity DoFs
// and their signs (local order) and its pressure DoFs (relative to n_u); the collapsed rule of q points
// per direction; the reference basis values [Q][nb][2], reference gradients [Q][nb][2][2]
// (d vhat_c / d xhat_d) and the pressure basis [Q][nq] at its points.
void bdm_error_data(const HostLevel& L, int q, std::vector<int>& cv, std::vector<double>& sg, std::vector<int>& cp,
                    std::vector<double>& xi, std::vector<double>& eta, std::vector<double>& w,
                    std::vector<double>& val, std::vector<double>& grad, std::vector<double>& psi) {
  const int N = L.N, k = L.k;
  const BdmMesh M(N, k);
  const RefBDM R = make_ref(k);
  const int nb = R.n, nq = M.nq;
  std::vector<int> dof;
  std::vector<double> sgn;
  cv.resize(size_t(M.ncell) * nb);
  sg.resize(size_t(M.ncell) * nb);
  cp.resize(size_t(M.ncell) * nq);
  for (int c = 0; c < M.ncell; ++c) {
    M.cell_dofs(c, dof, sgn);
    std::copy(dof.begin(), dof.end(), cv.begin() + size_t(c) * nb);
    std::copy(sgn.begin(), sgn.end(), sg.begin() + size_t(c) * nb);
    for (int m = 0; m < nq; ++m) cp[size_t(c) * nq + m] = M.pdof(c, m) - M.n_u;
  }
  std::vector<double> gx, gw;
  gauss01(q, gx, gw);
  xi.clear();
  eta.clear();
  w.clear();
  for (int iu = 0; iu < q; ++iu)
    for (int iv = 0; iv < q; ++iv) {
      xi.push_back(gx[iu]);
      eta.push_back(gx[iv] * (1.0 - gx[iu]));
      w.push_back(gw[iu] * gw[iv] * (1.0 - gx[iu]));
    }
  const int Q = int(w.size());
  val.resize(size_t(Q) * nb * 2);
  grad.resize(size_t(Q) * nb * 4);
  psi.resize(size_t(Q) * nq);
  for (int t = 0; t < Q; ++t) {
    R.eval(xi[t], eta[t], &val[size_t(t) * nb * 2], &grad[size_t(t) * nb * 4]);
    pressure_basis(k, xi[t], eta[t], &psi[size_t(t) * nq]);
  }
}

// DoF locations of a (BDM_k, dP_{k-1}) level: the edge point of each normal-flux DoF (kind 3), the
// cell centroid for the interior moments (kind 4), the pressure node (kind 2).
void bdm_dof_coords(const HostLevel& L, double* xy, int8_t* kind) {
  const int N = L.N, k = L.k;
  const BdmMesh M(N, k);
  const double h = 1.0 / N;
  auto put = [&](int d, double x, double y, int8_t c) {
    if (xy) {
      xy[2 * int64_t(d)] = x;
      xy[2 * int64_t(d) + 1] = y;
    }
    if (kind) kind[d] = c;
  };
  for (int e = 0; e < M.nedge; ++e) {
    int ax, ay, bx, by;
    M.edge_ends(e, ax, ay, bx, by);
    for (int j = 0; j <= k; ++j) {
      const double t = double(j + 1) / (k + 2);
      put(e * M.per_e + j, h * (ax + t * (bx - ax)), h * (ay + t * (by - ay)), 3);
    }
  }
  const int dq = k - 1;
  for (int c = 0; c < M.ncell; ++c) {
    int v[3][2];
    cell_vertices(N, c, v);
    const double cx = h * (v[0][0] + v[1][0] + v[2][0]) / 3.0, cy = h * (v[0][1] + v[1][1] + v[2][1]) / 3.0;
    for (int m = 0; m < M.per_c; ++m) put(M.n_edge + c * M.per_c + m, cx, cy, 4);
    int m = 0;
    for (int t = 0; t <= dq; ++t)
      for (int s2 = 0; s2 + t <= dq; ++s2, ++m) {
        const double xr = dq == 0 ? 1.0 / 3.0 : double(s2) / dq, yr = dq == 0 ? 1.0 / 3.0 : double(t) / dq;
        put(M.pdof(c, m), h * (v[0][0] + (v[1][0] - v[0][0]) * xr + (v[2][0] - v[0][0]) * yr),
            h * (v[0][1] + (v[1][1] - v[0][1]) * xr + (v[2][1] - v[0][1]) * yr), 2);
      }
  }
}

}  // namespace vk
