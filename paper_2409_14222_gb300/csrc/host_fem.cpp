// Host-side setup of one Taylor-Hood (P_k, P_{k-1}) level on the structured triangle mesh:
// element matrices, CSR assembly with Dirichlet rows, canonical transfers and Vanka patch lists.
//
// Paper: arXiv 2409.14222.
//  * Weak form a(u,v) = 2 nu int eps(u):eps(v), b(v,p) = -int (div v) p   -- Eqs. (VariationalStokesa/b)
//  * Block system [[A, B^T], [B, 0]] per level, nested meshes by uniform refinement -- Sec. 3
//  * Coarsest grid squares cut from top left to bottom right                -- Sec. 4
//  * Canonical transfers P = diag(P^V, P^Q), R = P^T                        -- Sec. 3, grid transfers
//  * Vertex / edge / cell ("composite") Vanka patches                        -- Sec. 3.1
//
// Basis: Lagrange P_k on equispaced nodes in Silvester's product form over barycentric coordinates;
// integrals: collapsed (Duffy) Gauss-Legendre rule, exact for the polynomial degrees of both forms.
#include <algorithm>
#include <array>
#include <cmath>
#include <exception>
#include <stdexcept>
#include <thread>

#include "vk_internal.h"

namespace vk {

namespace {

struct CellShape {
  int e1x, e1y, e2x, e2y;  // v1 - v0, v2 - v0 in units of h
};
// lower-left triangle (i,j),(i+1,j),(i,j+1); upper-right (i+1,j),(i+1,j+1),(i,j+1)
constexpr CellShape kLower{1, 0, 0, 1};
constexpr CellShape kUpper{0, 1, -1, 1};

// Lattice multi-indices (alpha0, alpha1, alpha2) of the P_deg nodes, t outer, s inner.
std::vector<std::array<int, 3>> node_indices(int deg) {
  std::vector<std::array<int, 3>> out;
  for (int t = 0; t <= deg; ++t)
    for (int s = 0; s + t <= deg; ++s) out.push_back({deg - s - t, s, t});
  return out;
}

// Silvester's product: phi_alpha(l) = prod_i prod_{j < alpha_i} (deg*l_i - j)/(j+1).
void eval_basis(int deg, const std::vector<std::array<int, 3>>& al, double xi, double eta,
                double* val, double* dxi, double* deta) {
  const double lam[3] = {1.0 - xi - eta, xi, eta};
  double P[3][16], D[3][16];
  for (int i = 0; i < 3; ++i) {
    P[i][0] = 1.0;
    D[i][0] = 0.0;
    for (int m = 1; m <= deg; ++m) {
      double f = (deg * lam[i] - (m - 1)) / m;
      P[i][m] = P[i][m - 1] * f;
      D[i][m] = D[i][m - 1] * f + P[i][m - 1] * (double(deg) / m);
    }
  }
  for (size_t a = 0; a < al.size(); ++a) {
    const int a0 = al[a][0], a1 = al[a][1], a2 = al[a][2];
    val[a] = P[0][a0] * P[1][a1] * P[2][a2];
    if (dxi) {
      double d0 = D[0][a0] * P[1][a1] * P[2][a2];
      double d1 = P[0][a0] * D[1][a1] * P[2][a2];
      double d2 = P[0][a0] * P[1][a1] * D[2][a2];
      dxi[a] = d1 - d0;
      deta[a] = d2 - d0;
    }
  }
}

struct Element {
  int nb = 0, nq = 0;
  std::vector<double> A;  // (2nb x 2nb), local velocity DoF 2a + c
  std::vector<double> B;  // (nq x 2nb): b(phi_a e_c, psi_q)
};

Element make_element(int k, const CellShape& s, double h, double nu) {
  Element E;
  element_matrices(k, s.e1x, s.e1y, s.e2x, s.e2y, h, nu, E.A, E.B);
  E.nb = (k + 1) * (k + 2) / 2;
  E.nq = k * (k + 1) / 2;
  return E;
}

template <class F>
void parallel_for(int n, int nthreads, F&& f) {
  nthreads = std::max(1, std::min(nthreads, n / 4096 + 1));
  if (nthreads == 1) {
    f(0, n);
    return;
  }
  // an exception in a worker (out of host memory, say) is carried to the caller instead of ending
  // the process
  std::vector<std::thread> th;
  std::vector<std::exception_ptr> err(nthreads);
  for (int t = 0; t < nthreads; ++t) {
    int lo = int(int64_t(n) * t / nthreads), hi = int(int64_t(n) * (t + 1) / nthreads);
    th.emplace_back([&f, &err, t, lo, hi] {
      try {
        f(lo, hi);
      } catch (...) {
        err[t] = std::current_exception();
      }
    });
  }
  for (auto& x : th) x.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

struct Cells {
  int N;
  int count() const { return 2 * N * N; }
  // cell c: lower cells c = j*N + i, upper cells N*N + j*N + i
  void vertex0(int c, int& x, int& y, const CellShape*& s) const {
    int q = c % (N * N), i = q % N, j = q / N;
    if (c < N * N) {
      x = i; y = j; s = &kLower;
    } else {
      x = i + 1; y = j; s = &kUpper;
    }
  }
};

}  // namespace

void gauss_legendre01(int q, std::vector<double>& x, std::vector<double>& w) {
  // Gauss-Legendre on [-1, 1] by Newton's method on the three-term recurrence, mapped to [0, 1].
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double p1 = 0, p0 = 0, dp = 1;
    for (int it = 0; it < 100; ++it) {
      p0 = 1.0;
      p1 = z;
      for (int n = 2; n <= q; ++n) {
        double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    p0 = 1.0;
    p1 = z;
    for (int n = 2; n <= q; ++n) {
      double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
      p0 = p1;
      p1 = p2;
    }
    dp = q * (z * p1 - p0) / (z * z - 1.0);
    x[i] = 0.5 * (z + 1.0);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // (2 / ((1-z^2) P'^2)) * 1/2
  }
}

void element_matrices(int k, int e1x, int e1y, int e2x, int e2y, double h, double nu,
                      std::vector<double>& Aloc, std::vector<double>& Bloc) {
  const auto av = node_indices(k);
  const auto aq = node_indices(k - 1);
  const int nb = int(av.size()), nq = int(aq.size()), nv = 2 * nb;
  Aloc.assign(size_t(nv) * nv, 0.0);
  Bloc.assign(size_t(nq) * nv, 0.0);
  const double J00 = h * e1x, J01 = h * e2x, J10 = h * e1y, J11 = h * e2y;
  const double det = J00 * J11 - J01 * J10;
  const double T00 = J11 / det, T01 = -J10 / det, T10 = -J01 / det, T11 = J00 / det;  // J^{-T}
  // collapsed rule: xi = u, eta = v (1 - u), d(xi,eta) = (1 - u) du dv; degree 2k-1 in u, 2k-2 in v
  std::vector<double> gx, gw;
  const int q = k + 2;
  gauss_legendre01(q, gx, gw);
  std::vector<double> phi(nb), dxi(nb), deta(nb), psi(nq), gxp(nb), gyp(nb);
  for (int iu = 0; iu < q; ++iu)
    for (int iv = 0; iv < q; ++iv) {
      const double u = gx[iu], v = gx[iv];
      const double xi = u, eta = v * (1.0 - u);
      const double wq = gw[iu] * gw[iv] * (1.0 - u) * std::fabs(det);
      eval_basis(k, av, xi, eta, phi.data(), dxi.data(), deta.data());
      eval_basis(k - 1, aq, xi, eta, psi.data(), nullptr, nullptr);
      for (int a = 0; a < nb; ++a) {
        gxp[a] = T00 * dxi[a] + T01 * deta[a];
        gyp[a] = T10 * dxi[a] + T11 * deta[a];
      }
      for (int a = 0; a < nb; ++a)
        for (int c = 0; c < 2; ++c) {
          const double ga[2] = {gxp[a], gyp[a]};
          for (int b = 0; b < nb; ++b)
            for (int d = 0; d < 2; ++d) {
              const double gb[2] = {gxp[b], gyp[b]};
              // 2 eps(phi_a e_c):eps(phi_b e_d) = delta_cd grad.grad + d_d phi_a d_c phi_b
              double v2 = ga[d] * gb[c];
              if (c == d) v2 += ga[0] * gb[0] + ga[1] * gb[1];
              Aloc[size_t(2 * a + c) * nv + 2 * b + d] += nu * wq * v2;
            }
          for (int p = 0; p < nq; ++p) Bloc[size_t(p) * nv + 2 * a + c] -= wq * psi[p] * ga[c];
        }
    }
}

namespace {

// 1-D Lagrange basis on the equispaced nodes i/deg of [0, 1] and its derivative at x.
void lagrange_1d(int deg, double x, double* val, double* der) {
  for (int i = 0; i <= deg; ++i) {
    double v = 1.0, d = 0.0;
    for (int j = 0; j <= deg; ++j) {
      if (j == i) continue;
      const double den = double(i - j) / deg;
      const double f = (x - double(j) / deg) / den;
      d = d * f + v / den;   // product rule, accumulated factor by factor
      v *= f;
    }
    val[i] = v;
    if (der) der[i] = d;
  }
}

// Q_k / Q_{k-1} element of an axis-aligned square of side h (Case 2 of Sec. 3): local velocity node
// (s, t) has index t (k+1) + s and basis l_s(x) l_t(y); local DoF 2a + c; Gauss-Legendre rule of k + 1
// points per direction (exact for the degree-2k products of the bilinear forms).
Element make_quad_element(int k, double h, double nu) {
  Element E;
  const int n1 = k + 1, nb = n1 * n1, nq = k * k, nv = 2 * nb;
  E.nb = nb;
  E.nq = nq;
  E.A.assign(size_t(nv) * nv, 0.0);
  E.B.assign(size_t(nq) * nv, 0.0);
  std::vector<double> gx, gw;
  const int q = k + 1;
  gauss_legendre01(q, gx, gw);
  std::vector<double> lx(n1), dx(n1), ly(n1), dy(n1), mx(k), my(k), phi(nb), gxp(nb), gyp(nb), psi(nq);
  for (int iy = 0; iy < q; ++iy)
    for (int ix = 0; ix < q; ++ix) {
      lagrange_1d(k, gx[ix], lx.data(), dx.data());
      lagrange_1d(k, gx[iy], ly.data(), dy.data());
      lagrange_1d(k - 1, gx[ix], mx.data(), nullptr);
      lagrange_1d(k - 1, gx[iy], my.data(), nullptr);
      const double w = gw[ix] * gw[iy] * h * h;
      for (int t = 0; t < n1; ++t)
        for (int s2 = 0; s2 < n1; ++s2) {
          phi[t * n1 + s2] = lx[s2] * ly[t];
          gxp[t * n1 + s2] = dx[s2] * ly[t] / h;
          gyp[t * n1 + s2] = lx[s2] * dy[t] / h;
        }
      for (int u = 0; u < k; ++u)
        for (int r = 0; r < k; ++r) psi[u * k + r] = mx[r] * my[u];
      for (int a = 0; a < nb; ++a)
        for (int c = 0; c < 2; ++c) {
          const double ga[2] = {gxp[a], gyp[a]};
          for (int b = 0; b < nb; ++b)
            for (int d = 0; d < 2; ++d) {
              const double gb[2] = {gxp[b], gyp[b]};
              double v2 = ga[d] * gb[c];
              if (c == d) v2 += ga[0] * gb[0] + ga[1] * gb[1];
              E.A[size_t(2 * a + c) * nv + 2 * b + d] += nu * w * v2;
            }
          for (int p = 0; p < nq; ++p) E.B[size_t(p) * nv + 2 * a + c] -= w * psi[p] * ga[c];
        }
    }
  return E;
}

}  // namespace

// Cell -> node maps of the structured quadrilateral mesh: cell (i, j) = j N + i; local node (s, t) of
// Q_deg at lattice point (deg i + s, deg j + t), index t (deg+1) + s.
void cell_maps_quad(int N, int k, std::vector<int>& cv, std::vector<int>& cp) {
  const int n1 = k + 1, nv1 = k * N + 1, np1 = (k - 1) * N + 1, nb = n1 * n1, nq = k * k;
  cv.resize(size_t(N) * N * nb);
  cp.resize(size_t(N) * N * nq);
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      const int c = j * N + i;
      for (int t = 0; t < n1; ++t)
        for (int s = 0; s < n1; ++s) cv[size_t(c) * nb + t * n1 + s] = (k * j + t) * nv1 + k * i + s;
      for (int u = 0; u < k; ++u)
        for (int r = 0; r < k; ++r) cp[size_t(c) * nq + u * k + r] = ((k - 1) * j + u) * np1 + (k - 1) * i + r;
    }
}

void build_level(int N, int k, double nu, bool with_patches, int nthreads, HostLevel& L, bool element_data,
                 int cell) {
  if (cell == 2) {
    if (element_data) throw std::runtime_error("BDM: no element data (matrix-full patches only)");
    build_level_bdm(N, k, nu, with_patches, nthreads, L);
    return;
  }
  if (k < 2 || k > 6) throw std::runtime_error("order k must be in 2..6");
  const bool quadc = cell == 1;
  L.N = N;
  L.k = k;
  L.cell = cell;
  L.nv1 = k * N + 1;
  L.np1 = (k - 1) * N + 1;
  L.n_u = 2 * L.nv1 * L.nv1;
  L.n_p = L.np1 * L.np1;
  L.ndof = L.n_u + L.n_p;
  const int nv1 = L.nv1, np1 = L.np1, n_u = L.n_u;
  const double h = 1.0 / N;
  // triangles: lower cells (index < N^2) and upper cells have their own element matrices; squares
  // all share one
  const int nb = quadc ? (k + 1) * (k + 1) : (k + 1) * (k + 2) / 2;
  const int nq = quadc ? k * k : k * (k + 1) / 2, nvl = 2 * nb;
  const Element EL = quadc ? make_quad_element(k, h, nu) : make_element(k, kLower, h, nu);
  const Element EU = quadc ? EL : make_element(k, kUpper, h, nu);
  const int ncell = quadc ? N * N : 2 * N * N;
  const int nlow = quadc ? ncell : N * N;
  L.ncell_lower = nlow;

  // local -> global node maps
  std::vector<int> cv, cp;
  if (quadc)
    cell_maps_quad(N, k, cv, cp);
  else
    cell_maps(N, k, cv, cp);
  // Dirichlet flags
  L.dir.assign(L.ndof, 0);
  for (int b = 0; b < nv1; ++b)
    for (int a = 0; a < nv1; ++a)
      if (a == 0 || b == 0 || a == nv1 - 1 || b == nv1 - 1) {
        L.dir[2 * (b * nv1 + a)] = 1;
        L.dir[2 * (b * nv1 + a) + 1] = 1;
      }
  // node -> (cell, local) incidence, cells ascending
  auto incidence = [&](int nnode, int per, const std::vector<int>& map, std::vector<int>& ptr,
                       std::vector<int>& ent) {
    ptr.assign(nnode + 1, 0);
    for (int c = 0; c < ncell; ++c)
      for (int a = 0; a < per; ++a) ptr[map[size_t(c) * per + a] + 1]++;
    for (int i = 0; i < nnode; ++i) ptr[i + 1] += ptr[i];
    ent.assign(ptr[nnode], 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int c = 0; c < ncell; ++c)
      for (int a = 0; a < per; ++a) ent[fill[map[size_t(c) * per + a]]++] = c * per + a;
  };
  std::vector<int> vptr, vent, pptr, pent;
  incidence(nv1 * nv1, nb, cv, vptr, vent);
  incidence(np1 * np1, nq, cp, pptr, pent);

  // row patterns: union of the DoFs of the incident cells; Dirichlet rows keep only the diagonal,
  // Dirichlet columns are dropped (they are zero)
  const auto& dir = L.dir;
  auto row_cells = [&](int row, std::vector<int>& out) {
    out.clear();
    if (row < n_u) {
      int node = row / 2;
      for (int e = vptr[node]; e < vptr[node + 1]; ++e) out.push_back(vent[e]);  // c*nb + a
    } else {
      int node = row - n_u;
      for (int e = pptr[node]; e < pptr[node + 1]; ++e) out.push_back(pent[e]);  // c*nq + p
    }
  };
  std::vector<int> rowlen(L.ndof, 0);
  std::vector<std::vector<int>> pattern(L.ndof);
  parallel_for(L.ndof, nthreads, [&](int lo, int hi) {
    std::vector<int> inc, cols;
    for (int row = lo; row < hi; ++row) {
      cols.clear();
      if (dir[row]) {
        cols.push_back(row);
      } else {
        row_cells(row, inc);
        const int per = row < n_u ? nb : nq;
        for (int e : inc) {
          int c = e / per;
          for (int b = 0; b < nb; ++b)
            for (int d = 0; d < 2; ++d) {
              int g = 2 * cv[size_t(c) * nb + b] + d;
              if (!dir[g]) cols.push_back(g);
            }
          if (row < n_u)
            for (int p = 0; p < nq; ++p) cols.push_back(n_u + cp[size_t(c) * nq + p]);
        }
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      }
      pattern[row] = cols;
      rowlen[row] = int(cols.size());
    }
  });
  HostCsr& A = L.A;
  A.nrows = A.ncols = L.ndof;
  A.ptr.assign(L.ndof + 1, 0);
  for (int i = 0; i < L.ndof; ++i) A.ptr[i + 1] = A.ptr[i] + rowlen[i];
  A.col.resize(A.ptr.back());
  A.val.assign(A.ptr.back(), 0.0);
  parallel_for(L.ndof, nthreads, [&](int lo, int hi) {
    std::vector<int> inc;
    for (int row = lo; row < hi; ++row) {
      int* col = A.col.data() + A.ptr[row];
      double* val = A.val.data() + A.ptr[row];
      const auto& pat = pattern[row];
      std::copy(pat.begin(), pat.end(), col);
      if (dir[row]) {
        val[0] = 1.0;
        continue;
      }
      const int len = int(pat.size());
      auto add = [&](int g, double v) {
        int pos = int(std::lower_bound(col, col + len, g) - col);
        val[pos] += v;
      };
      row_cells(row, inc);
      if (row < n_u) {
        const int comp = row & 1;
        for (int e : inc) {
          int c = e / nb, a = e % nb;
          const Element& E = c < nlow ? EL : EU;
          const int la = 2 * a + comp;
          for (int b = 0; b < nb; ++b)
            for (int d = 0; d < 2; ++d) {
              int g = 2 * cv[size_t(c) * nb + b] + d;
              if (!dir[g]) add(g, E.A[size_t(la) * nvl + 2 * b + d]);
            }
          for (int p = 0; p < nq; ++p) add(n_u + cp[size_t(c) * nq + p], E.B[size_t(p) * nvl + la]);
        }
      } else {
        for (int e : inc) {
          int c = e / nq, p = e % nq;
          const Element& E = c < nlow ? EL : EU;
          for (int b = 0; b < nb; ++b)
            for (int d = 0; d < 2; ++d) {
              int g = 2 * cv[size_t(c) * nb + b] + d;
              if (!dir[g]) add(g, E.B[size_t(p) * nvl + 2 * b + d]);
            }
        }
      }
    }
  });
  pattern.clear();
  pattern.shrink_to_fit();

  if (!with_patches) return;
  // ---------------- Vanka patches (Sec. 3.1): one per entity carrying P_{k-1} DoFs ----------------
  auto lower = [&](int i, int j) { return j * N + i; };
  auto upper = [&](int i, int j) { return N * N + j * N + i; };
  L.patch_ptr.assign(1, 0);
  L.patch_dofs.clear();
  L.patch_kind.clear();
  std::vector<int> dofs;
  auto emit = [&](int kind, const int* cl, int ncl, const std::vector<int>& pnodes) {
    dofs.clear();
    for (int t = 0; t < ncl; ++t) {
      int c = cl[t];
      for (int a = 0; a < nb; ++a)
        for (int d = 0; d < 2; ++d) {
          int g = 2 * cv[size_t(c) * nb + a] + d;
          if (!dir[g]) dofs.push_back(g);
        }
    }
    for (int pn : pnodes) dofs.push_back(n_u + pn);
    std::sort(dofs.begin(), dofs.end());
    dofs.erase(std::unique(dofs.begin(), dofs.end()), dofs.end());
    L.patch_dofs.insert(L.patch_dofs.end(), dofs.begin(), dofs.end());
    L.patch_ptr.push_back(int(L.patch_dofs.size()));
    L.patch_kind.push_back(int8_t(kind));
  };
  const int k1 = k - 1;
  std::vector<int> pn;
  int cl[6];
  if (quadc) {
    // squares (Case 2): vertex patches (star = the up-to-four cells around the vertex), then for k >= 3
    // horizontal edges, vertical edges (the one or two adjacent cells; the k - 2 edge pressures) and
    // cells (the (k - 2)^2 interior pressures); each family y outer, x inner
    auto sq = [&](int i, int j) { return j * N + i; };
    for (int j = 0; j <= N; ++j)
      for (int i = 0; i <= N; ++i) {
        int n = 0;
        if (i > 0 && j > 0) cl[n++] = sq(i - 1, j - 1);
        if (i < N && j > 0) cl[n++] = sq(i, j - 1);
        if (i > 0 && j < N) cl[n++] = sq(i - 1, j);
        if (i < N && j < N) cl[n++] = sq(i, j);
        pn.assign(1, (k1 * j) * np1 + k1 * i);
        emit(0, cl, n, pn);
      }
    if (k >= 3) {
      for (int j = 0; j <= N; ++j)
        for (int i = 0; i < N; ++i) {
          int n = 0;
          if (j > 0) cl[n++] = sq(i, j - 1);
          if (j < N) cl[n++] = sq(i, j);
          pn.clear();
          for (int t = 1; t <= k - 2; ++t) pn.push_back((k1 * j) * np1 + k1 * i + t);
          emit(1, cl, n, pn);
        }
      for (int j = 0; j < N; ++j)
        for (int i = 0; i <= N; ++i) {
          int n = 0;
          if (i > 0) cl[n++] = sq(i - 1, j);
          if (i < N) cl[n++] = sq(i, j);
          pn.clear();
          for (int t = 1; t <= k - 2; ++t) pn.push_back((k1 * j + t) * np1 + k1 * i);
          emit(1, cl, n, pn);
        }
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          cl[0] = sq(i, j);
          pn.clear();
          for (int u = 1; u <= k - 2; ++u)
            for (int r = 1; r <= k - 2; ++r) pn.push_back((k1 * j + u) * np1 + k1 * i + r);
          emit(2, cl, 1, pn);
        }
    }
  } else {
  // vertices: star = the up-to-six incident cells
  for (int j = 0; j <= N; ++j)
    for (int i = 0; i <= N; ++i) {
      int n = 0;
      if (i < N && j < N) cl[n++] = lower(i, j);          // as v0
      if (i > 0 && j < N) cl[n++] = lower(i - 1, j);      // as v1
      if (i < N && j > 0) cl[n++] = lower(i, j - 1);      // as v2
      if (i > 0 && j < N) cl[n++] = upper(i - 1, j);      // as v0
      if (i > 0 && j > 0) cl[n++] = upper(i - 1, j - 1);  // as v1
      if (i < N && j > 0) cl[n++] = upper(i, j - 1);      // as v2
      pn.assign(1, (k1 * j) * np1 + k1 * i);
      emit(0, cl, n, pn);
    }
  if (k >= 3) {
    auto edge_nodes = [&](int ax, int ay, int dx, int dy) {
      pn.clear();
      for (int t = 1; t <= k - 2; ++t) pn.push_back((k1 * ay + t * dy) * np1 + k1 * ax + t * dx);
    };
    for (int j = 0; j <= N; ++j)  // horizontal (i,j)-(i+1,j)
      for (int i = 0; i < N; ++i) {
        int n = 0;
        if (j < N) cl[n++] = lower(i, j);
        if (j > 0) cl[n++] = upper(i, j - 1);
        edge_nodes(i, j, 1, 0);
        emit(1, cl, n, pn);
      }
    for (int j = 0; j < N; ++j)  // vertical (i,j)-(i,j+1)
      for (int i = 0; i <= N; ++i) {
        int n = 0;
        if (i < N) cl[n++] = lower(i, j);
        if (i > 0) cl[n++] = upper(i - 1, j);
        edge_nodes(i, j, 0, 1);
        emit(1, cl, n, pn);
      }
    for (int j = 0; j < N; ++j)  // diagonal (i+1,j)-(i,j+1)
      for (int i = 0; i < N; ++i) {
        cl[0] = lower(i, j);
        cl[1] = upper(i, j);
        edge_nodes(i + 1, j, -1, 1);
        emit(1, cl, 2, pn);
      }
  }
  if (k >= 4) {
    for (int up = 0; up < 2; ++up)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          const CellShape& s = up ? kUpper : kLower;
          int x0 = up ? i + 1 : i, y0 = j;
          pn.clear();
          for (int t = 1; t <= k - 3; ++t)
            for (int u = 1; u + t <= k - 2; ++u)
              pn.push_back((k1 * y0 + u * s.e1y + t * s.e2y) * np1 + k1 * x0 + u * s.e1x + t * s.e2x);
          cl[0] = up ? upper(i, j) : lower(i, j);
          emit(2, cl, 1, pn);
        }
  }
  }  // triangles
  if (!element_data) return;
  // ---- element data of the matrix-free patch assembly -------------------------------------------
  const int nloc = nvl + nq;
  L.nloc = nloc;
  L.cell_dofs.resize(size_t(ncell) * nloc);
  for (int c = 0; c < ncell; ++c) {
    int* cd = L.cell_dofs.data() + size_t(c) * nloc;
    for (int a = 0; a < nb; ++a)
      for (int d = 0; d < 2; ++d) cd[2 * a + d] = 2 * cv[size_t(c) * nb + a] + d;
    for (int p = 0; p < nq; ++p) cd[nvl + p] = n_u + cp[size_t(c) * nq + p];
  }
  L.kel.assign(size_t(2) * nloc * nloc, 0.0);
  for (int sh = 0; sh < 2; ++sh) {
    const Element& E = sh == 0 ? EL : EU;
    double* K = L.kel.data() + size_t(sh) * nloc * nloc;
    for (int a = 0; a < nvl; ++a)
      for (int b = 0; b < nvl; ++b) K[size_t(a) * nloc + b] = E.A[size_t(a) * nvl + b];
    for (int p = 0; p < nq; ++p)
      for (int a = 0; a < nvl; ++a) {
        K[size_t(nvl + p) * nloc + a] = E.B[size_t(p) * nvl + a];
        K[size_t(a) * nloc + nvl + p] = E.B[size_t(p) * nvl + a];
      }
  }
  // cells of each patch's assembly: every cell containing one of the patch's DoFs, ascending
  const int np = int(L.patch_ptr.size()) - 1;
  std::vector<std::vector<int>> pc(np);
  parallel_for(np, nthreads, [&](int lo, int hi) {
    std::vector<int> cs;
    for (int p = lo; p < hi; ++p) {
      cs.clear();
      for (int e = L.patch_ptr[p]; e < L.patch_ptr[p + 1]; ++e) {
        const int g = L.patch_dofs[e];
        if (g < n_u) {
          const int node = g / 2;
          for (int t = vptr[node]; t < vptr[node + 1]; ++t) cs.push_back(vent[t] / nb);
        } else {
          const int node = g - n_u;
          for (int t = pptr[node]; t < pptr[node + 1]; ++t) cs.push_back(pent[t] / nq);
        }
      }
      std::sort(cs.begin(), cs.end());
      cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
      pc[p] = cs;
    }
  });
  L.patch_cell_ptr.assign(np + 1, 0);
  for (int p = 0; p < np; ++p) L.patch_cell_ptr[p + 1] = L.patch_cell_ptr[p] + int(pc[p].size());
  L.patch_cells.resize(L.patch_cell_ptr.back());
  for (int p = 0; p < np; ++p) std::copy(pc[p].begin(), pc[p].end(), L.patch_cells.begin() + L.patch_cell_ptr[p]);
}

void build_transfer(const HostLevel& c, HostLevel& f) {
  // P = diag(P^V, P^Q): each fine node is located in a coarse cell; coarse basis functions are
  // evaluated there exactly: barycentric coordinates are m_i / (2 deg) with integer m_i, so
  // phi_alpha = prod_i prod_{j < alpha_i} (m_i - 2j) / (2 (j + 1)), an exact ratio of integers.
  // Squares: the basis is a tensor product, so P^V and P^Q are tensor products of the 1-D
  // interpolations l_s(m / (2 deg)) = prod_{j != s} (m - 2 j) / (2 (s - j)), also exact ratios.
  if (f.N != 2 * c.N || f.k != c.k || f.cell != c.cell) throw std::runtime_error("transfer: levels not nested");
  if (f.cell == 2) {
    build_transfer_bdm(c, f);
    return;
  }
  const int Nc = c.N;
  struct Trip {
    int r, c;
    double v;
  };
  std::vector<Trip> t;
  auto block_quad = [&](int deg, int nf1, int nc1, int offf, int offc, int stride) {
    const int two = 2 * deg;
    std::vector<std::vector<std::pair<int, double>>> w1(nf1);   // 1-D weights of fine node a
    for (int a = 0; a < nf1; ++a) {
      const int i = std::min(a / two, Nc - 1), m = a - two * i;
      for (int s2 = 0; s2 <= deg; ++s2) {
        int64_t num = 1, den = 1;
        for (int j = 0; j <= deg; ++j)
          if (j != s2) {
            num *= (m - 2 * j);
            den *= 2 * (s2 - j);
          }
        if (num != 0) w1[a].push_back({deg * i + s2, double(num) / double(den)});
      }
    }
    for (int b = 0; b < nf1; ++b)
      for (int a = 0; a < nf1; ++a)
        for (const auto& wy : w1[b])
          for (const auto& wx : w1[a]) {
            const double v = wx.second * wy.second;
            const int cn = wy.first * nc1 + wx.first, fn = b * nf1 + a;
            for (int d = 0; d < stride; ++d) t.push_back({offf + stride * fn + d, offc + stride * cn + d, v});
          }
  };
  auto block = [&](int deg, int nf1, int nc1, int offf, int offc, int stride) {
    if (f.cell == 1) {
      block_quad(deg, nf1, nc1, offf, offc, stride);
      return;
    }
    const auto al = node_indices(deg);
    const int two = 2 * deg;
    for (int b = 0; b < nf1; ++b)
      for (int a = 0; a < nf1; ++a) {
        int i = std::min(a / two, Nc - 1), j = std::min(b / two, Nc - 1);
        int fx = a - two * i, fy = b - two * j;
        int m[3], x0, y0;
        const CellShape* s;
        if (fx + fy <= two) {
          m[0] = two - fx - fy; m[1] = fx; m[2] = fy; x0 = i; y0 = j; s = &kLower;
        } else {
          m[2] = two - fx; m[1] = fx + fy - two; m[0] = two - fy; x0 = i + 1; y0 = j; s = &kUpper;
        }
        for (const auto& alpha : al) {
          int64_t num = 1, den = 1;
          for (int q = 0; q < 3; ++q)
            for (int jj = 0; jj < alpha[q]; ++jj) {
              num *= (m[q] - 2 * jj);
              den *= 2 * (jj + 1);
            }
          if (num == 0) continue;
          const double v = double(num) / double(den);
          int ca = deg * x0 + alpha[1] * s->e1x + alpha[2] * s->e2x;
          int cb = deg * y0 + alpha[1] * s->e1y + alpha[2] * s->e2y;
          int cn = cb * nc1 + ca, fn = b * nf1 + a;
          for (int d = 0; d < stride; ++d) t.push_back({offf + stride * fn + d, offc + stride * cn + d, v});
        }
      }
  };
  block(f.k, f.nv1, c.nv1, 0, 0, 2);
  block(f.k - 1, f.np1, c.np1, f.n_u, c.n_u, 1);
  std::stable_sort(t.begin(), t.end(), [](const Trip& x, const Trip& y) {
    return x.r != y.r ? x.r < y.r : x.c < y.c;
  });
  HostCsr& P = f.P;
  P.nrows = f.ndof;
  P.ncols = c.ndof;
  P.ptr.assign(P.nrows + 1, 0);
  P.col.resize(t.size());
  P.val.resize(t.size());
  for (size_t e = 0; e < t.size(); ++e) {
    P.ptr[t[e].r + 1]++;
    P.col[e] = t[e].c;
    P.val[e] = t[e].v;
  }
  for (int i = 0; i < P.nrows; ++i) P.ptr[i + 1] += P.ptr[i];
  // R = P^T (counting transpose; columns come out ascending)
  HostCsr& R = f.R;
  R.nrows = c.ndof;
  R.ncols = f.ndof;
  R.ptr.assign(R.nrows + 1, 0);
  for (int cc : P.col) R.ptr[cc + 1]++;
  for (int i = 0; i < R.nrows; ++i) R.ptr[i + 1] += R.ptr[i];
  R.col.resize(P.col.size());
  R.val.resize(P.col.size());
  std::vector<int> fill(R.ptr.begin(), R.ptr.end() - 1);
  for (int r = 0; r < P.nrows; ++r)
    for (int e = P.ptr[r]; e < P.ptr[r + 1]; ++e) {
      int pos = fill[P.col[e]]++;
      R.col[pos] = r;
      R.val[pos] = P.val[e];
    }
}

double splitmix_uniform_pm1(uint64_t seed, uint64_t i) {
  // SplitMix64 (Steele, Lea, Flood 2014): state_i = seed + (i+1) * golden gamma, then the mix.
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return 2.0 * (double(z >> 11) * 0x1.0p-53) - 1.0;
}

}  // namespace vk

namespace vk {

// Cell -> node maps of the structured mesh: velocity P_k nodes (cv, ncell x nb) and pressure P_{k-1}
// nodes (cp, ncell x nq) in the element's local order (the order of build_level's assembly).
void cell_maps(int N, int k, std::vector<int>& cv, std::vector<int>& cp) {
  const auto av = node_indices(k), aq = node_indices(k - 1);
  const int nb = int(av.size()), nq = int(aq.size()), nv1 = k * N + 1, np1 = (k - 1) * N + 1;
  Cells cells{N};
  const int ncell = cells.count();
  cv.resize(size_t(ncell) * nb);
  cp.resize(size_t(ncell) * nq);
  for (int c = 0; c < ncell; ++c) {
    int x0, y0;
    const CellShape* s;
    cells.vertex0(c, x0, y0, s);
    for (int a = 0; a < nb; ++a)
      cv[size_t(c) * nb + a] = (k * y0 + av[a][1] * s->e1y + av[a][2] * s->e2y) * nv1 +
                               k * x0 + av[a][1] * s->e1x + av[a][2] * s->e2x;
    for (int p = 0; p < nq; ++p)
      cp[size_t(c) * nq + p] = ((k - 1) * y0 + aq[p][1] * s->e1y + aq[p][2] * s->e2y) * np1 +
                               (k - 1) * x0 + aq[p][1] * s->e1x + aq[p][2] * s->e2x;
  }
}

// Collapsed (Duffy) Gauss-Legendre rule with q points per direction on the reference triangle and the
// P_k / P_{k-1} basis at its points: xi = u, eta = v (1 - u), weight w_u w_v (1 - u).
void reference_tables(int k, int q, std::vector<double>& xi, std::vector<double>& eta, std::vector<double>& w,
                      std::vector<double>& phi, std::vector<double>& dxi, std::vector<double>& deta,
                      std::vector<double>& psi) {
  const auto av = node_indices(k), aq = node_indices(k - 1);
  const int nb = int(av.size()), nq = int(aq.size()), Q = q * q;
  std::vector<double> gx, gw;
  gauss_legendre01(q, gx, gw);
  xi.resize(Q);
  eta.resize(Q);
  w.resize(Q);
  phi.resize(size_t(Q) * nb);
  dxi.resize(size_t(Q) * nb);
  deta.resize(size_t(Q) * nb);
  psi.resize(size_t(Q) * nq);
  for (int iu = 0; iu < q; ++iu)
    for (int iv = 0; iv < q; ++iv) {
      const int t = iu * q + iv;
      xi[t] = gx[iu];
      eta[t] = gx[iv] * (1.0 - gx[iu]);
      w[t] = gw[iu] * gw[iv] * (1.0 - gx[iu]);
      eval_basis(k, av, xi[t], eta[t], &phi[size_t(t) * nb], &dxi[size_t(t) * nb], &deta[size_t(t) * nb]);
      eval_basis(k - 1, aq, xi[t], eta[t], &psi[size_t(t) * nq], nullptr, nullptr);
    }
}

// Right-hand side of the manufactured problem (Eq. model_problem): u = (sin(pi x) cos(pi y),
// -cos(pi x) sin(pi y)), p = 0, so f = -div(2 nu eps(u)) + grad p = 2 pi^2 nu u.  The load <f, v> is
// integrated with the collapsed rule of k + 5 points per direction; the velocity's Dirichlet data g (its
// nodal interpolant on the boundary) is lifted: b_F = F_F - K_FB g, b_B = g, with K the element
// matrices before boundary conditions.
void manufactured_rhs(const HostLevel& L, double nu, std::vector<double>& b) {
  const int N = L.N, k = L.k, nv1 = L.nv1, n_u = L.n_u;
  const double h = 1.0 / N, pi = M_PI;
  std::vector<int> cv, cp;
  cell_maps(N, k, cv, cp);
  const int nb = (k + 1) * (k + 2) / 2, nq = k * (k + 1) / 2, nvl = 2 * nb;
  std::vector<double> xi, eta, w, phi, dxi, deta, psi;
  reference_tables(k, k + 5, xi, eta, w, phi, dxi, deta, psi);
  const int Q = int(w.size());
  const Element EL = make_element(k, kLower, h, nu), EU = make_element(k, kUpper, h, nu);
  Cells cells{N};
  b.assign(L.ndof, 0.0);
  std::vector<double> g(L.ndof, 0.0);
  for (int node = 0; node < nv1 * nv1; ++node)
    if (L.dir[2 * node]) {
      const double X = double(node % nv1) / (k * N), Y = double(node / nv1) / (k * N);
      g[2 * node] = std::sin(pi * X) * std::cos(pi * Y);
      g[2 * node + 1] = -std::cos(pi * X) * std::sin(pi * Y);
    }
  for (int c = 0; c < cells.count(); ++c) {
    int x0, y0;
    const CellShape* s;
    cells.vertex0(c, x0, y0, s);
    const double J00 = h * s->e1x, J01 = h * s->e2x, J10 = h * s->e1y, J11 = h * s->e2y;
    const double adet = std::fabs(J00 * J11 - J01 * J10);
    const int* nodes = &cv[size_t(c) * nb];
    for (int t = 0; t < Q; ++t) {
      const double X = h * x0 + J00 * xi[t] + J01 * eta[t], Y = h * y0 + J10 * xi[t] + J11 * eta[t];
      const double f1 = 2 * pi * pi * nu * std::sin(pi * X) * std::cos(pi * Y);
      const double f2 = -2 * pi * pi * nu * std::cos(pi * X) * std::sin(pi * Y);
      const double wt = w[t] * adet;
      for (int a = 0; a < nb; ++a) {
        b[2 * nodes[a]] += wt * f1 * phi[size_t(t) * nb + a];
        b[2 * nodes[a] + 1] += wt * f2 * phi[size_t(t) * nb + a];
      }
    }
    // lifting: subtract K_e g_e from every row of the element
    const Element& E = c < N * N ? EL : EU;
    double ge[64];
    bool any = false;
    for (int a = 0; a < nb; ++a)
      for (int d = 0; d < 2; ++d) {
        ge[2 * a + d] = g[2 * nodes[a] + d];
        any = any || ge[2 * a + d] != 0.0;
      }
    if (!any) continue;
    for (int la = 0; la < nvl; ++la) {
      double acc = 0.0;
      for (int lb = 0; lb < nvl; ++lb) acc += E.A[size_t(la) * nvl + lb] * ge[lb];
      b[2 * nodes[la / 2] + (la & 1)] -= acc;
    }
    for (int p = 0; p < nq; ++p) {
      double acc = 0.0;
      for (int lb = 0; lb < nvl; ++lb) acc += E.B[size_t(p) * nvl + lb] * ge[lb];
      b[n_u + cp[size_t(c) * nq + p]] -= acc;
    }
  }
  for (int i = 0; i < n_u; ++i)
    if (L.dir[i]) b[i] = g[i];
}

}  // namespace vk

namespace vk {

// Tensor Gauss-Legendre rule of q points per direction on the unit reference square and the Q_k /
// Q_{k-1} basis at its points (local node (s, t) -> index t (k+1) + s; pressure (r, u) -> u k + r).
void reference_tables_quad(int k, int q, std::vector<double>& xi, std::vector<double>& eta, std::vector<double>& w,
                           std::vector<double>& phi, std::vector<double>& dxi, std::vector<double>& deta,
                           std::vector<double>& psi) {
  const int n1 = k + 1, nb = n1 * n1, nq = k * k, Q = q * q;
  std::vector<double> gx, gw;
  gauss_legendre01(q, gx, gw);
  xi.resize(Q);
  eta.resize(Q);
  w.resize(Q);
  phi.resize(size_t(Q) * nb);
  dxi.resize(size_t(Q) * nb);
  deta.resize(size_t(Q) * nb);
  psi.resize(size_t(Q) * nq);
  std::vector<double> lx(n1), dx(n1), ly(n1), dy(n1), mx(k), my(k);
  for (int iy = 0; iy < q; ++iy)
    for (int ix = 0; ix < q; ++ix) {
      const int t = iy * q + ix;
      xi[t] = gx[ix];
      eta[t] = gx[iy];
      w[t] = gw[ix] * gw[iy];
      lagrange_1d(k, gx[ix], lx.data(), dx.data());
      lagrange_1d(k, gx[iy], ly.data(), dy.data());
      lagrange_1d(k - 1, gx[ix], mx.data(), nullptr);
      lagrange_1d(k - 1, gx[iy], my.data(), nullptr);
      for (int b = 0; b < n1; ++b)
        for (int a = 0; a < n1; ++a) {
          phi[size_t(t) * nb + b * n1 + a] = lx[a] * ly[b];
          dxi[size_t(t) * nb + b * n1 + a] = dx[a] * ly[b];
          deta[size_t(t) * nb + b * n1 + a] = lx[a] * dy[b];
        }
      for (int u = 0; u < k; ++u)
        for (int r = 0; r < k; ++r) psi[size_t(t) * nq + u * k + r] = mx[r] * my[u];
    }
}

// The manufactured right-hand side (Eq. model_problem) for Q_k / Q_{k-1} on the N x N squares: tensor
// Gauss-Legendre rule of k + 5 points per direction, boundary data lifted as for the triangles.
void manufactured_rhs_quad(const HostLevel& L, double nu, std::vector<double>& b) {
  const int N = L.N, k = L.k, nv1 = L.nv1, n_u = L.n_u;
  const double h = 1.0 / N, pi = M_PI;
  std::vector<int> cv, cp;
  cell_maps_quad(N, k, cv, cp);
  const int nb = (k + 1) * (k + 1), nq = k * k, nvl = 2 * nb;
  std::vector<double> xi, eta, w, phi, dxi, deta, psi;
  reference_tables_quad(k, k + 5, xi, eta, w, phi, dxi, deta, psi);
  const int Q = int(w.size());
  const Element E = make_quad_element(k, h, nu);
  b.assign(L.ndof, 0.0);
  std::vector<double> g(L.ndof, 0.0);
  for (int node = 0; node < nv1 * nv1; ++node)
    if (L.dir[2 * node]) {
      const double X = double(node % nv1) / (k * N), Y = double(node / nv1) / (k * N);
      g[2 * node] = std::sin(pi * X) * std::cos(pi * Y);
      g[2 * node + 1] = -std::cos(pi * X) * std::sin(pi * Y);
    }
  for (int c = 0; c < N * N; ++c) {
    const int i = c % N, j = c / N;
    const int* nodes = &cv[size_t(c) * nb];
    for (int t = 0; t < Q; ++t) {
      const double X = h * (i + xi[t]), Y = h * (j + eta[t]);
      const double f1 = 2 * pi * pi * nu * std::sin(pi * X) * std::cos(pi * Y);
      const double f2 = -2 * pi * pi * nu * std::cos(pi * X) * std::sin(pi * Y);
      const double wt = w[t] * h * h;
      for (int a = 0; a < nb; ++a) {
        b[2 * nodes[a]] += wt * f1 * phi[size_t(t) * nb + a];
        b[2 * nodes[a] + 1] += wt * f2 * phi[size_t(t) * nb + a];
      }
    }
    double ge[64];
    bool any = false;
    for (int a = 0; a < nb; ++a)
      for (int d = 0; d < 2; ++d) {
        ge[2 * a + d] = g[2 * nodes[a] + d];
        any = any || ge[2 * a + d] != 0.0;
      }
    if (!any) continue;
    for (int la = 0; la < nvl; ++la) {
      double acc = 0.0;
      for (int lb = 0; lb < nvl; ++lb) acc += E.A[size_t(la) * nvl + lb] * ge[lb];
      b[2 * nodes[la / 2] + (la & 1)] -= acc;
    }
    for (int p = 0; p < nq; ++p) {
      double acc = 0.0;
      for (int lb = 0; lb < nvl; ++lb) acc += E.B[size_t(p) * nvl + lb] * ge[lb];
      b[n_u + cp[size_t(c) * nq + p]] -= acc;
    }
  }
  for (int i = 0; i < n_u; ++i)
    if (L.dir[i]) b[i] = g[i];
}

}  // namespace vk
