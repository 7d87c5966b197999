// Internal declarations of the Vanka multigrid library (host setup structures, kernel launchers).
// Not part of the public C ABI; see include/vk.h for that.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace vk {

// ------------------------------------------------------------------------------------------------
// Host-side sparse matrix (CSR, int32 indices, FP64 values).
struct HostCsr {
  int nrows = 0, ncols = 0;
  std::vector<int> ptr, col;
  std::vector<double> val;
  int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

// One mesh level of the Taylor-Hood (P_k, P_{k-1}) discretization on the structured triangle mesh.
struct HostLevel {
  int N = 0, k = 0;
  int cell = 0;             // 0: triangles (P_k, P_{k-1}); 1: squares (Q_k, Q_{k-1}); 2: (BDM_k, dP_{k-1})
  int ncell_lower = 0;      // cells below this index use the first element matrix (all squares do)
  int nv1 = 0, np1 = 0;     // lattice sizes per side: k*N+1 (velocity), (k-1)*N+1 (pressure)
  int n_u = 0, n_p = 0, ndof = 0;
  HostCsr A;                // saddle-point matrix with Dirichlet identity rows / zero columns
  HostCsr P, R;             // prolongation from the next coarser level and R = P^T (empty on level 0)
  std::vector<uint8_t> dir; // 1 at Dirichlet velocity DoFs
  // Vanka patches (empty on the coarsest level): DoFs of patch p are dofs[ptr[p] .. ptr[p+1]).
  std::vector<int> patch_ptr, patch_dofs;
  std::vector<int8_t> patch_kind;  // 0 vertex, 1 edge, 2 cell
  // Element data for assembling patch matrices from element matrices (matrix-free patches; built only
  // on request): the element DoFs of every cell in element-local order (velocity 2a + c, then the
  // pressure nodes), the element matrix [[A_e, B_e^T], [B_e, 0]] of the lower and of the upper cell
  // shape (nloc x nloc each, row-major), and per patch the cells containing any of its DoFs (ascending).
  int nloc = 0;
  std::vector<int> cell_dofs;
  std::vector<double> kel;
  std::vector<int> patch_cell_ptr, patch_cells;
};

// host_fem.cpp
void build_level(int N, int k, double nu, bool with_patches, int nthreads, HostLevel& L, bool element_data = false,
                 int cell = 0);
void build_transfer(const HostLevel& coarse, HostLevel& fine);
// Element matrices of one cell shape, for tests and the manufactured load (row-major).
void element_matrices(int k, int e1x, int e1y, int e2x, int e2y, double h, double nu,
                      std::vector<double>& Aloc, std::vector<double>& Bloc);
void gauss_legendre01(int q, std::vector<double>& x, std::vector<double>& w);

void cell_maps(int N, int k, std::vector<int>& cv, std::vector<int>& cp);
void cell_maps_quad(int N, int k, std::vector<int>& cv, std::vector<int>& cp);
void reference_tables(int k, int q, std::vector<double>& xi, std::vector<double>& eta, std::vector<double>& w,
                      std::vector<double>& phi, std::vector<double>& dxi, std::vector<double>& deta,
                      std::vector<double>& psi);
void manufactured_rhs(const HostLevel& L, double nu, std::vector<double>& b);
void reference_tables_quad(int k, int q, std::vector<double>& xi, std::vector<double>& eta, std::vector<double>& w,
                           std::vector<double>& phi, std::vector<double>& dxi, std::vector<double>& deta,
                           std::vector<double>& psi);
void manufactured_rhs_quad(const HostLevel& L, double nu, std::vector<double>& b);

// host_bdm.cpp: (BDM_k, dP_{k-1}) with the interior-penalty form on the triangle mesh (Case 3).
void build_level_bdm(int N, int k, double nu, bool with_patches, int nthreads, HostLevel& L);
void build_transfer_bdm(const HostLevel& coarse, HostLevel& fine);
void manufactured_rhs_bdm(const HostLevel& L, double nu, std::vector<double>& b);
void bdm_dof_coords(const HostLevel& L, double* xy, int8_t* kind);
void bdm_error_data(const HostLevel& L, int q, std::vector<int>& cv, std::vector<double>& sg, std::vector<int>& cp,
                    std::vector<double>& xi, std::vector<double>& eta, std::vector<double>& w,
                    std::vector<double>& val, std::vector<double>& grad, std::vector<double>& psi);

// host_eig.cpp: eigenvalues of a small real upper-Hessenberg matrix (row-major m x m).
int hessenberg_eigenvalues(int m, const double* H, double* re, double* im);

// SplitMix64 counter-based uniform on [-1, 1): value i of stream `seed`.
double splitmix_uniform_pm1(uint64_t seed, uint64_t i);

}  // namespace vk
