"""Taylor-Hood (P_k, P_{k-1}) discretization of the Stokes problem on a structured triangle mesh.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows the paper:
* Stokes strong form and no-slip Dirichlet data: Eqs. (Stokes1), (StokesDivFree), (StokesDirichletNoSlip).
* Weak form, a(u, v) = 2 nu int eps(u):eps(v) and b(v, p) = -int (div v) p: Eqs. (VariationalStokesa/b).
* Saddle-point block matrix [[A, B^T], [B, 0]] (Sec. 3) and nested hierarchy by uniform refinement.
* Coarsest grid: squares "cut from top left to bottom right" into two triangles (Sec. 4).
* Canonical transfers: P = diag(P^V, P^Q) interpolates the natural embedding, R = P^T (Sec. 3).
* Manufactured solution u = (sin(pi x) cos(pi y), -cos(pi x) sin(pi y)), p = 0 (Eq. model_problem).
* Error measures: relative H^1 velocity error, L^2 pressure error after removing the mean (Sec. 4.4).

Readings where the paper is silent:
* node placement: equispaced Lagrange nodes, so P_k nodes form the lattice (kN+1)^2, x fastest;
* DoF order: velocity node-major (2*node + component), then the P_{k-1} pressure lattice;
* viscosity: nu = 1 by default (a parameter);
* Dirichlet velocity DoFs stay in the system with an identity row and a zeroed column;
* quadrature: exact for the bilinear forms (exact rational integration here).
"""
from fractions import Fraction

import numpy as np
import scipy.sparse as sp

from . import exact


class Mesh:
    """N x N squares of the unit square; square (i, j) = [i, i+1] x [j, j+1] (units of h = 1/N).

    The diagonal runs from the top-left corner (i, j+1) to the bottom-right corner (i+1, j) (Sec. 4),
    giving the lower-left triangle (i,j), (i+1,j), (i,j+1) and the upper-right triangle
    (i+1,j), (i+1,j+1), (i,j+1), both counter-clockwise.  Cells are listed lower triangles first
    (j outer, i inner), then upper triangles.  Vertex (i, j) has id j*(N+1) + i.
    """

    def __init__(self, N):
        self.N = N
        lower = [((i, j), (i + 1, j), (i, j + 1)) for j in range(N) for i in range(N)]
        upper = [((i + 1, j), (i + 1, j + 1), (i, j + 1)) for j in range(N) for i in range(N)]
        self.cells = lower + upper

    def vid(self, v):
        return v[1] * (self.N + 1) + v[0]


def _cell_geometry(cell):
    """Affine map x = v0 + J xi (J in units of h) as exact rationals: J, J^{-T}, |det J|."""
    (x0, y0), (x1, y1), (x2, y2) = cell
    J = [[Fraction(x1 - x0), Fraction(x2 - x0)], [Fraction(y1 - y0), Fraction(y2 - y0)]]
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0]
    Jinv = [[J[1][1] / det, -J[0][1] / det], [-J[1][0] / det, J[0][0] / det]]
    JinvT = [[Jinv[0][0], Jinv[1][0]], [Jinv[0][1], Jinv[1][1]]]
    return J, JinvT, abs(det)


_ELEM_CACHE = {}


def element_matrices(k, cell):
    """Exact element matrices for one cell shape (they depend only on v1-v0, v2-v0).

    Returns (A_loc, Bq_loc) as Fraction nested lists:
      A_loc[2a+c][2b+d] = int_T eps(phi_a e_c) : eps(phi_b e_d) * 2   (i.e. a(.,.)/nu)
                        = delta_cd grad phi_a . grad phi_b + d_d phi_a d_c phi_b
      Bq_loc[q][2a+c]   = -(1/h) int_T psi_q d_c phi_a      (multiply by h to get b(.,.))
    For the exact integrals: int_T d_i phi_a d_j phi_b dx = |det J| sum_mn (J^-T)_im (J^-T)_jn G_mn,
    which does not depend on h in 2D; the b(.,.) integral scales with h.
    """
    (x0, y0), (x1, y1), (x2, y2) = cell
    key = (k, x1 - x0, y1 - y0, x2 - x0, y2 - y0)
    if key in _ELEM_CACHE:
        return _ELEM_CACHE[key]
    _, JT, adet = _cell_geometry(cell)
    G = exact.grad_grad(k)
    K = exact.pressure_div(k)
    nb = len(exact.basis(k))
    nq = len(exact.basis(k - 1))
    S = [[[[adet * sum(JT[i][m] * JT[j][n] * G[m][n][a][b] for m in (0, 1) for n in (0, 1))
            for b in range(nb)] for a in range(nb)] for j in (0, 1)] for i in (0, 1)]
    A = [[Fraction(0)] * (2 * nb) for _ in range(2 * nb)]
    for a in range(nb):
        for c in (0, 1):
            for b in range(nb):
                for d in (0, 1):
                    v = S[d][c][a][b]
                    if c == d:
                        v += S[0][0][a][b] + S[1][1][a][b]
                    A[2 * a + c][2 * b + d] = v
    Bq = [[-adet * sum(JT[c][m] * K[m][q][a] for m in (0, 1)) for a in range(nb) for c in (0, 1)]
          for q in range(nq)]
    _ELEM_CACHE[key] = (A, Bq)
    return A, Bq


class Space:
    """P_k velocity / P_{k-1} pressure DoF layout on one mesh level.

    Velocity node (a, b) of the lattice (kN+1)^2 sits at (a/(kN), b/(kN)); its DoFs are 2*node + c.
    Pressure node (a, b) of the lattice ((k-1)N+1)^2 has DoF 2*(kN+1)^2 + b*((k-1)N+1) + a.
    """

    def __init__(self, N, k):
        assert k >= 2
        self.N, self.k = N, k
        self.mesh = Mesh(N)
        self.nv1 = k * N + 1
        self.np1 = (k - 1) * N + 1
        self.n_u = 2 * self.nv1 ** 2
        self.n_p = self.np1 ** 2
        self.ndof = self.n_u + self.n_p
        self.ref_v = exact.lattice_nodes(k)
        self.ref_p = exact.lattice_nodes(k - 1)

    def cell_vnodes(self, cell):
        """Global velocity node ids of the cell's local P_k nodes, in exact.lattice_nodes order."""
        (x0, y0), (x1, y1), (x2, y2) = cell
        k, n1 = self.k, self.nv1
        out = []
        for s, t in self.ref_v:
            a = k * x0 + s * (x1 - x0) + t * (x2 - x0)
            b = k * y0 + s * (y1 - y0) + t * (y2 - y0)
            out.append(b * n1 + a)
        return out

    def cell_pnodes(self, cell):
        (x0, y0), (x1, y1), (x2, y2) = cell
        k1, n1 = self.k - 1, self.np1
        out = []
        for s, t in self.ref_p:
            a = k1 * x0 + s * (x1 - x0) + t * (x2 - x0)
            b = k1 * y0 + s * (y1 - y0) + t * (y2 - y0)
            out.append(b * n1 + a)
        return out

    def cell_vdofs(self, cell):
        return [2 * g + c for g in self.cell_vnodes(cell) for c in (0, 1)]

    def cell_pdofs(self, cell):
        return [self.n_u + g for g in self.cell_pnodes(cell)]

    def vnode_xy(self):
        a = np.arange(self.nv1 ** 2) % self.nv1
        b = np.arange(self.nv1 ** 2) // self.nv1
        return a / (self.k * self.N), b / (self.k * self.N)

    def pnode_xy(self):
        a = np.arange(self.np1 ** 2) % self.np1
        b = np.arange(self.np1 ** 2) // self.np1
        return a / ((self.k - 1) * self.N), b / ((self.k - 1) * self.N)

    def dirichlet_mask(self):
        """True at velocity DoFs whose node lies on the boundary of the unit square."""
        a = np.arange(self.nv1 ** 2) % self.nv1
        b = np.arange(self.nv1 ** 2) // self.nv1
        bnd = (a == 0) | (b == 0) | (a == self.nv1 - 1) | (b == self.nv1 - 1)
        mask = np.zeros(self.ndof, dtype=bool)
        mask[0:self.n_u:2] = bnd
        mask[1:self.n_u:2] = bnd
        return mask

    def nullspace(self):
        """z = (0_u, 1_p): constant pressure, the kernel of the Dirichlet system (p in L^2_0, Sec. 2)."""
        z = np.zeros(self.ndof)
        z[self.n_u:] = 1.0
        return z


def assemble_full(space, nu=1.0):
    """Global block matrix [[A, B^T], [B, 0]] before boundary conditions (Sec. 3), CSR, FP64.

    A and B come from the exact element matrices; B^T is the transpose of the same integrals, so the
    matrix is exactly symmetric.  The sparsity pattern is the element connectivity.  Cells of the
    same shape share one element matrix, so the sum over cells is done one shape at a time."""
    h = Fraction(1, space.N)
    groups = {}
    for cell in space.mesh.cells:
        (x0, y0), (x1, y1), (x2, y2) = cell
        groups.setdefault((x1 - x0, y1 - y0, x2 - x0, y2 - y0), []).append(cell)
    rows, cols, vals = [], [], []
    for cells in groups.values():
        A, Bq = element_matrices(space.k, cells[0])
        Af = nu * np.array([[float(v) for v in row] for row in A])
        Bf = np.array([[float(v * h) for v in row] for row in Bq])
        vd = np.array([space.cell_vdofs(c) for c in cells])      # (ncell, 2nb)
        pd = np.array([space.cell_pdofs(c) for c in cells])      # (ncell, nq)
        nc, nv = vd.shape
        nq = pd.shape[1]
        rows.append(np.repeat(vd, nv, axis=1).ravel())
        cols.append(np.tile(vd, (1, nv)).ravel())
        vals.append(np.tile(Af.ravel(), nc))
        br = np.repeat(pd, nv, axis=1).ravel()
        bc = np.tile(vd, (1, nq)).ravel()
        bv = np.tile(Bf.ravel(), nc)
        rows += [br, bc]
        cols += [bc, br]
        vals += [bv, bv]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    K = sp.coo_matrix((vals, (rows, cols)), shape=(space.ndof, space.ndof)).tocsr()
    K.sum_duplicates()
    K.sort_indices()
    return K


def apply_dirichlet(K, mask):
    """Identity rows and zero columns at the Dirichlet velocity DoFs (reading of Eq. StokesDirichletNoSlip)."""
    free = sp.diags((~mask).astype(float))
    A = (free @ K @ free + sp.diags(mask.astype(float))).tocsr()
    A.sort_indices()
    return A


def prolongation(coarse, fine):
    """Canonical prolongation P = diag(P^V, P^Q) from level N to 2N (Sec. 3, grid transfers).

    Each fine node is located in a coarse cell and every coarse basis function of that cell is
    evaluated there in exact rational arithmetic, so P^V (per velocity component) and P^Q (P_{k-1})
    are the matrices of the natural embeddings.  Entries that are exactly zero are not stored."""
    assert fine.N == 2 * coarse.N and fine.k == coarse.k
    k, Nc = coarse.k, coarse.N
    rows, cols, vals = [], [], []

    def locate(X, Y):
        i = min(int(X), Nc - 1)
        j = min(int(Y), Nc - 1)
        fx, fy = X - i, Y - j
        if fx + fy <= 1:
            cell = ((i, j), (i + 1, j), (i, j + 1))
        else:
            cell = ((i + 1, j), (i + 1, j + 1), (i, j + 1))
        (x0, y0), (x1, y1), (x2, y2) = cell
        # solve v0 + J xi = (X, Y) exactly
        J, _, _ = _cell_geometry(cell)
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0]
        dx, dy = X - x0, Y - y0
        xi = (J[1][1] * dx - J[0][1] * dy) / det
        eta = (-J[1][0] * dx + J[0][0] * dy) / det
        return cell, xi, eta

    for comp_block, deg, n_f1, n_c1, off_f, off_c, stride in (
            ("V", k, fine.nv1, coarse.nv1, 0, 0, 2), ("Q", k - 1, fine.np1, coarse.np1, fine.n_u, coarse.n_u, 1)):
        basis = exact.basis(deg)
        ref = exact.lattice_nodes(deg)
        cache = {}
        for b in range(n_f1):
            for a in range(n_f1):
                X = Fraction(a, 2 * deg)
                Y = Fraction(b, 2 * deg)
                cell, xi, eta = locate(X, Y)
                (x0, y0), (x1, y1), (x2, y2) = cell
                shape = (x1 - x0, y1 - y0, x2 - x0, y2 - y0, xi, eta)
                if shape not in cache:
                    cache[shape] = [(loc, exact.evaluate(basis[loc], xi, eta)) for loc in range(len(ref))]
                for loc, val in cache[shape]:
                    if val == 0:
                        continue
                    s, t = ref[loc]
                    ca = deg * x0 + s * (x1 - x0) + t * (x2 - x0)
                    cb = deg * y0 + s * (y1 - y0) + t * (y2 - y0)
                    cnode = cb * n_c1 + ca
                    fnode = b * n_f1 + a
                    for c in range(stride):
                        rows.append(off_f + stride * fnode + c)
                        cols.append(off_c + stride * cnode + c)
                        vals.append(float(val))
    P = sp.coo_matrix((vals, (rows, cols)), shape=(fine.ndof, coarse.ndof)).tocsr()
    P.sort_indices()
    return P


# ---------------------------------------------------------------------------------------------
# Manufactured solution (Eq. model_problem), load vector, lifting and error norms (Sec. 4, 4.4)
# ---------------------------------------------------------------------------------------------

def u_exact(x, y):
    return np.sin(np.pi * x) * np.cos(np.pi * y), -np.cos(np.pi * x) * np.sin(np.pi * y)


def grad_u_exact(x, y):
    """((du1/dx, du1/dy), (du2/dx, du2/dy))."""
    pi = np.pi
    return ((pi * np.cos(pi * x) * np.cos(pi * y), -pi * np.sin(pi * x) * np.sin(pi * y)),
            (pi * np.sin(pi * x) * np.sin(pi * y), -pi * np.cos(pi * x) * np.cos(pi * y)))


def f_exact(x, y, nu=1.0):
    """f = -div(2 nu eps(u)) + grad p = -nu Laplace(u) = 2 pi^2 nu u, since div u = 0 and p = 0."""
    u1, u2 = u_exact(x, y)
    return 2 * np.pi ** 2 * nu * u1, 2 * np.pi ** 2 * nu * u2


def ref_quadrature(q):
    """Collapsed (Duffy) Gauss-Legendre rule on the reference triangle, exact to degree 2q-2.

    x = s, y = t (1 - s), dx dy = (1 - s) ds dt on [0,1]^2."""
    g, w = np.polynomial.legendre.leggauss(q)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    S, T = np.meshgrid(g, g, indexing="ij")
    WS, WT = np.meshgrid(w, w, indexing="ij")
    x = S.ravel()
    y = (T * (1 - S)).ravel()
    wt = (WS * WT * (1 - S)).ravel()
    return x, y, wt


def _basis_at(deg, x, y):
    """Float values and reference gradients of the P_deg basis at reference points."""
    mons, C = exact.monomial_coeff_matrix(deg)
    V = np.stack([x ** p * y ** q for p, q in mons], axis=1)
    Dx = np.stack([p * x ** max(p - 1, 0) * y ** q if p > 0 else 0 * x for p, q in mons], axis=1)
    Dy = np.stack([q * x ** p * y ** max(q - 1, 0) if q > 0 else 0 * x for p, q in mons], axis=1)
    return V @ C, Dx @ C, Dy @ C


def _cell_float_geometry(cell, h):
    (x0, y0), (x1, y1), (x2, y2) = cell
    J = h * np.array([[x1 - x0, x2 - x0], [y1 - y0, y2 - y0]], dtype=float)
    return np.array([x0 * h, y0 * h]), J


def load_vector(space, nu=1.0, qdeg=None):
    """<f, v> for every velocity test function (Eq. VariationalStokes1), with f of the manufactured
    solution; pressure rows are zero.  Quadrature exact to degree >= 2k + 6."""
    q = qdeg or (space.k + 5)
    xr, yr, wr = ref_quadrature(q)
    phi, _, _ = _basis_at(space.k, xr, yr)
    h = 1.0 / space.N
    F = np.zeros(space.ndof)
    for cell in space.mesh.cells:
        v0, J = _cell_float_geometry(cell, h)
        X = v0[0] + J[0, 0] * xr + J[0, 1] * yr
        Y = v0[1] + J[1, 0] * xr + J[1, 1] * yr
        f1, f2 = f_exact(X, Y, nu)
        w = wr * abs(np.linalg.det(J))
        vd = space.cell_vdofs(cell)
        for a in range(phi.shape[1]):
            F[vd[2 * a]] += np.sum(w * f1 * phi[:, a])
            F[vd[2 * a + 1]] += np.sum(w * f2 * phi[:, a])
    return F


def manufactured_rhs(space, K, nu=1.0):
    """Algebraic right-hand side with the Dirichlet data lifted (reading of Eq. StokesDirichletNoSlip):
    b_F = F_F - K_FB g, b_B = g, with g the nodal interpolant of the exact velocity on the boundary."""
    mask = space.dirichlet_mask()
    X, Y = space.vnode_xy()
    u1, u2 = u_exact(X, Y)
    gfull = np.zeros(space.ndof)
    gfull[0:space.n_u:2] = u1
    gfull[1:space.n_u:2] = u2
    g = np.where(mask, gfull, 0.0)
    F = load_vector(space, nu)
    b = F - K @ g
    b[mask] = g[mask]
    return b


def errors(space, x, nu=1.0, qdeg=None):
    """(relative H^1 velocity error, relative L^2 velocity error, L^2 pressure error) against
    Eq. (model_problem); the pressure is orthogonalised against constants in L^2 first (Sec. 4.4)."""
    q = qdeg or (space.k + 6)
    xr, yr, wr = ref_quadrature(q)
    phi, dphx, dphy = _basis_at(space.k, xr, yr)
    psi, _, _ = _basis_at(space.k - 1, xr, yr)
    h = 1.0 / space.N
    e_l2 = e_h1 = n_l2 = n_h1 = 0.0
    p_int = p_sq = 0.0
    area = 0.0
    for cell in space.mesh.cells:
        v0, J = _cell_float_geometry(cell, h)
        JinvT = np.linalg.inv(J).T
        X = v0[0] + J[0, 0] * xr + J[0, 1] * yr
        Y = v0[1] + J[1, 0] * xr + J[1, 1] * yr
        w = wr * abs(np.linalg.det(J))
        vd = space.cell_vdofs(cell)
        pd = space.cell_pdofs(cell)
        ux = x[vd[0::2]]
        uy = x[vd[1::2]]
        gx = JinvT[0, 0] * dphx + JinvT[0, 1] * dphy
        gy = JinvT[1, 0] * dphx + JinvT[1, 1] * dphy
        uh1, uh2 = phi @ ux, phi @ uy
        G = ((gx @ ux, gy @ ux), (gx @ uy, gy @ uy))
        u1, u2 = u_exact(X, Y)
        Ge = grad_u_exact(X, Y)
        e_l2 += np.sum(w * ((uh1 - u1) ** 2 + (uh2 - u2) ** 2))
        n_l2 += np.sum(w * (u1 ** 2 + u2 ** 2))
        for i in (0, 1):
            for j in (0, 1):
                e_h1 += np.sum(w * (G[i][j] - Ge[i][j]) ** 2)
                n_h1 += np.sum(w * Ge[i][j] ** 2)
        ph = psi @ x[pd]
        p_int += np.sum(w * ph)
        p_sq += np.sum(w * ph ** 2)
        area += np.sum(w)
    mean = p_int / area
    p_err = np.sqrt(max(p_sq - 2 * mean * p_int + mean ** 2 * area, 0.0))
    h1_rel = np.sqrt((e_l2 + e_h1) / (n_l2 + n_h1))
    l2_rel = np.sqrt(e_l2 / n_l2)
    return h1_rel, l2_rel, p_err
