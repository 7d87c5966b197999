"""Taylor-Hood (Q_k, Q_{k-1}) discretization on the structured quadrilateral mesh (Case 2 of Sec. 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows the paper:
* Case 2 of Sec. 3: continuous Q_k velocity and continuous Q_{k-1} pressure on quadrilaterals, k >= 2,
  the same weak form as the triangles (Eqs. VariationalStokesa/b), the same block matrix (Sec. 3).
* Nested meshes by uniform refinement (Sec. 3); the unit square cut into N x N squares (Sec. 4).
* Canonical transfers: interpolation of the natural embedding, R = P^T (Sec. 3).
* Composite Vanka patches of Sec. 3.1 for quadrilaterals: one patch per vertex (the vertex pressure,
  velocity on the closure of the vertex star, the up-to-four cells around it); for k >= 3 one patch per
  edge (its k - 2 pressures, velocity on the one or two adjacent cells) and one per cell (its (k - 2)^2
  interior pressures, velocity on the cell).
* Manufactured solution (Eq. model_problem) and the error measures of Sec. 4.4.

Readings where the paper is silent (the same as for the triangles):
* equispaced Lagrange nodes, so the Q_k nodes are the (kN+1)^2 lattice and the DoF layout is the one of
  the triangles (velocity node-major 2*node + component, then the Q_{k-1} pressure lattice);
* Dirichlet velocity DoFs stay in the system as identity rows with zeroed columns;
* patches exclude Dirichlet DoFs; patch order: vertices, horizontal edges, vertical edges, cells, each
  lexicographic (y outer, x inner); DoFs ascending within a patch.

Exactness: the 1-D Lagrange bases are exact rationals; every 2-D integral of the forms is a product of
exact 1-D integrals (int_0^1 x^n = 1 / (n + 1)), so every element matrix and transfer entry is exact.
"""
from fractions import Fraction

import numpy as np
import scipy.sparse as sp


# ---------------------------------------------------------------------------- 1-D exact polynomials
def _pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _pder(a):
    return [a[i] * i for i in range(1, len(a))] or [Fraction(0)]


def _pint01(a):
    return sum(c / (i + 1) for i, c in enumerate(a))


def _peval(a, x):
    return sum(c * x ** i for i, c in enumerate(a))


def lagrange_1d(deg):
    """Exact 1-D Lagrange basis on the nodes i/deg of [0, 1]: coefficient lists (ascending powers)."""
    nodes = [Fraction(i, deg) for i in range(deg + 1)]
    out = []
    for i, xi in enumerate(nodes):
        poly = [Fraction(1)]
        for j, xj in enumerate(nodes):
            if j != i:
                poly = _pmul(poly, [-xj / (xi - xj), 1 / (xi - xj)])
        out.append(poly)
    return out


def _gram(f, g):
    return [[_pint01(_pmul(a, b)) for b in g] for a in f]


_ELEM = {}


def element_matrices(k):
    """Exact element matrices of the unit reference square for Q_k / Q_{k-1}.

    Local velocity node (s, t), s, t = 0..k, has index t*(k+1) + s and basis l_s(x) l_t(y); local DoF
    2a + c is component c of node a.  Returns (A_loc, Bq_loc):
      A_loc[2a+c][2b+d] = delta_cd grad phi_a . grad phi_b + d_d phi_a d_c phi_b   (= a(.,.) / nu, 2 eps:eps)
      Bq_loc[q][2a+c]   = -int psi_q d_c phi_a                                        (multiply by h)
    The gradient integrals of a square of side h do not depend on h; the divergence integral scales by h."""
    if k in _ELEM:
        return _ELEM[k]
    L, Lp = lagrange_1d(k), lagrange_1d(k - 1)
    dL = [_pder(p) for p in L]
    M, D = _gram(L, L), _gram(dL, dL)
    C = _gram(dL, L)            # C[i][j] = int l_i' l_j
    E = _gram(dL, Lp)           # int l_i' m_r
    F = _gram(L, Lp)            # int l_i m_r
    n1 = k + 1
    nodes = [(s, t) for t in range(n1) for s in range(n1)]
    nb = len(nodes)

    def G(m, n, a, b):          # int d_m phi_a d_n phi_b
        (sa, ta), (sb, tb) = nodes[a], nodes[b]
        if m == 0 and n == 0:
            return D[sa][sb] * M[ta][tb]
        if m == 1 and n == 1:
            return M[sa][sb] * D[ta][tb]
        if m == 0 and n == 1:
            return C[sa][sb] * C[tb][ta]
        return C[sb][sa] * C[ta][tb]

    A = [[Fraction(0)] * (2 * nb) for _ in range(2 * nb)]
    for a in range(nb):
        for c in (0, 1):
            for b in range(nb):
                for d in (0, 1):
                    v = G(d, c, a, b)
                    if c == d:
                        v += G(0, 0, a, b) + G(1, 1, a, b)
                    A[2 * a + c][2 * b + d] = v
    pn = [(r, u) for u in range(k) for r in range(k)]
    Bq = [[Fraction(0)] * (2 * nb) for _ in range(len(pn))]
    for q, (r, u) in enumerate(pn):
        for a, (s, t) in enumerate(nodes):
            Bq[q][2 * a] = -E[s][r] * F[t][u]
            Bq[q][2 * a + 1] = -F[s][r] * E[t][u]
    _ELEM[k] = (A, Bq)
    return A, Bq


# ---------------------------------------------------------------------------- space
class QSpace:
    """Q_k velocity / Q_{k-1} pressure on the N x N squares of the unit square.

    Cell (i, j) = [i, i+1] x [j, j+1] in units of h = 1/N, listed j outer, i inner.  Velocity node (a, b) of
    the (kN+1)^2 lattice sits at (a/(kN), b/(kN)) with DoFs 2*node + c, node = b*(kN+1) + a; pressure node
    (a, b) of the ((k-1)N+1)^2 lattice has DoF 2*(kN+1)^2 + b*((k-1)N+1) + a."""

    cell_type = "quad"

    def __init__(self, N, k):
        assert k >= 2
        self.N, self.k = N, k
        self.cells = [(i, j) for j in range(N) for i in range(N)]
        self.nv1 = k * N + 1
        self.np1 = (k - 1) * N + 1
        self.n_u = 2 * self.nv1 ** 2
        self.n_p = self.np1 ** 2
        self.ndof = self.n_u + self.n_p

    def cell_vnodes(self, cell):
        i, j = cell
        k, n1 = self.k, self.nv1
        return [(k * j + t) * n1 + k * i + s for t in range(k + 1) for s in range(k + 1)]

    def cell_pnodes(self, cell):
        i, j = cell
        k1, n1 = self.k - 1, self.np1
        return [(k1 * j + u) * n1 + k1 * i + r for u in range(k1 + 1) for r in range(k1 + 1)]

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
        a = np.arange(self.nv1 ** 2) % self.nv1
        b = np.arange(self.nv1 ** 2) // self.nv1
        bnd = (a == 0) | (b == 0) | (a == self.nv1 - 1) | (b == self.nv1 - 1)
        mask = np.zeros(self.ndof, dtype=bool)
        mask[0:self.n_u:2] = bnd
        mask[1:self.n_u:2] = bnd
        return mask

    def nullspace(self):
        z = np.zeros(self.ndof)
        z[self.n_u:] = 1.0
        return z


def assemble_full(space, nu=1.0):
    """Global block matrix [[A, B^T], [B, 0]] before boundary conditions (Sec. 3), CSR, FP64; every cell
    is the same square, so one exact element matrix serves all of them."""
    A, Bq = element_matrices(space.k)
    h = Fraction(1, space.N)
    Af = nu * np.array([[float(v) for v in row] for row in A])
    Bf = np.array([[float(v * h) for v in row] for row in Bq])
    vd = np.array([space.cell_vdofs(c) for c in space.cells])
    pd = np.array([space.cell_pdofs(c) for c in space.cells])
    nc, nv = vd.shape
    nq = pd.shape[1]
    rows = [np.repeat(vd, nv, axis=1).ravel()]
    cols = [np.tile(vd, (1, nv)).ravel()]
    vals = [np.tile(Af.ravel(), nc)]
    br = np.repeat(pd, nv, axis=1).ravel()
    bc = np.tile(vd, (1, nq)).ravel()
    bv = np.tile(Bf.ravel(), nc)
    rows += [br, bc]
    cols += [bc, br]
    vals += [bv, bv]
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(space.ndof, space.ndof)).tocsr()
    K.sum_duplicates()
    K.sort_indices()
    return K


def _prolong_1d(deg, Nc):
    """Exact 1-D interpolation from the coarse nodes a/(deg Nc) to the fine nodes a/(2 deg Nc)."""
    L = lagrange_1d(deg)
    nf, nc = 2 * deg * Nc + 1, deg * Nc + 1
    out = []
    for a in range(nf):
        X = Fraction(a, 2 * deg) * 1          # in units of the coarse cell size
        i = min(int(X), Nc - 1)
        xi = X - i
        row = {}
        for s in range(deg + 1):
            v = _peval(L[s], xi)
            if v != 0:
                row[deg * i + s] = v
        out.append(row)
    assert all(c < nc for r in out for c in r)
    return out


def prolongation(coarse, fine):
    """P = diag(P^V, P^Q) from level N to 2N: tensor products of the exact 1-D interpolations, per
    velocity component for P^V; entries that are exactly zero are not stored."""
    assert fine.N == 2 * coarse.N and fine.k == coarse.k
    rows, cols, vals = [], [], []
    for deg, n_f1, n_c1, off_f, off_c, stride in ((coarse.k, fine.nv1, coarse.nv1, 0, 0, 2),
                                                  (coarse.k - 1, fine.np1, coarse.np1, fine.n_u, coarse.n_u, 1)):
        P1 = _prolong_1d(deg, coarse.N)
        for b in range(n_f1):
            for a in range(n_f1):
                for cb, wb in P1[b].items():
                    for ca, wa in P1[a].items():
                        for c in range(stride):
                            rows.append(off_f + stride * (b * n_f1 + a) + c)
                            cols.append(off_c + stride * (cb * n_c1 + ca) + c)
                            vals.append(float(wa * wb))
    P = sp.coo_matrix((vals, (rows, cols)), shape=(fine.ndof, coarse.ndof)).tocsr()
    P.sort_indices()
    return P


# ---------------------------------------------------------------------------- patches (Sec. 3.1)
def _entity_of(X, Y):
    """The mesh entity (in units of h) whose interior contains the point: ('vertex', (i, j)),
    ('hedge', (i, j)) for (i,j)-(i+1,j), ('vedge', (i, j)) for (i,j)-(i,j+1), or ('cell', (i, j))."""
    xi, yi = X.denominator == 1, Y.denominator == 1
    i, j = int(X), int(Y)          # floor for non-negative values
    if xi and yi:
        return ("vertex", (i, j))
    if yi:
        return ("hedge", (i, j))
    if xi:
        return ("vedge", (i, j))
    return ("cell", (i, j))


def _cells_of(kind, e, N):
    """Cells (i, j) whose closure contains the entity."""
    i, j = e
    if kind == "vertex":
        cand = [(i - 1, j - 1), (i, j - 1), (i - 1, j), (i, j)]
    elif kind == "hedge":
        cand = [(i, j - 1), (i, j)]
    elif kind == "vedge":
        cand = [(i - 1, j), (i, j)]
    else:
        cand = [(i, j)]
    return [(a, b) for a, b in cand if 0 <= a < N and 0 <= b < N]


def build_patches(space):
    """List of (kind, entity, dofs): one patch per entity carrying Q_{k-1} pressure DoFs, holding all of
    them and the free velocity DoFs of every cell whose closure contains the entity."""
    k, N = space.k, space.N
    mask = space.dirichlet_mask()
    groups = {}
    for b in range(space.np1):
        for a in range(space.np1):
            X, Y = Fraction(a, k - 1), Fraction(b, k - 1)     # units of h
            ent = _entity_of(X, Y)
            groups.setdefault(ent, []).append(space.n_u + b * space.np1 + a)
    order = {"vertex": 0, "hedge": 1, "vedge": 2, "cell": 3}
    out = []
    for (kind, e), pdofs in sorted(groups.items(), key=lambda it: (order[it[0][0]], it[0][1][1], it[0][1][0])):
        vel = set()
        for c in _cells_of(kind, e, N):
            vel.update(d for d in space.cell_vdofs(c) if not mask[d])
        dofs = np.array(sorted(vel) + sorted(pdofs), dtype=np.int64)
        out.append(({"vertex": "vertex", "hedge": "edge", "vedge": "edge", "cell": "cell"}[kind], (kind, e), dofs))
    return out


def interior_patch_size(k, kind):
    """Closed-form size of an interior patch: the closure of the vertex star is 2 x 2 cells ((2k+1)^2
    nodes), of an edge star 2 cells ((k+1)(2k+1) nodes), of a cell (k+1)^2 nodes; Q_{k-1} has one
    pressure per vertex, k - 2 per edge and (k - 2)^2 per cell."""
    if kind == "vertex":
        return 2 * (2 * k + 1) ** 2 + 1
    if kind == "edge":
        return 2 * (k + 1) * (2 * k + 1) + (k - 2)
    if kind == "cell":
        return 2 * (k + 1) ** 2 + (k - 2) ** 2
    raise ValueError(kind)


# ---------------------------------------------------------------------------- manufactured problem
def _gauss01(q):
    g, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (g + 1.0), 0.5 * w


def _basis_1d_float(deg, x):
    L = lagrange_1d(deg)
    V = np.stack([sum(float(c) * x ** i for i, c in enumerate(p)) for p in L], axis=1)
    dL = [_pder(p) for p in L]
    D = np.stack([sum(float(c) * x ** i for i, c in enumerate(p)) for p in dL], axis=1)
    return V, D


def load_vector(space, nu=1.0, q=None):
    """<f, v> with f of Eq. (model_problem), tensor Gauss-Legendre rule of q = k + 5 points per direction."""
    from .fem import f_exact
    k, N = space.k, space.N
    q = q or (k + 5)
    x, w = _gauss01(q)
    V, _ = _basis_1d_float(k, x)
    h = 1.0 / N
    F = np.zeros(space.ndof)
    for cell in space.cells:
        i, j = cell
        X = h * (i + x)[None, :]                 # [iy, ix]
        Y = h * (j + x)[:, None]
        f1, f2 = f_exact(X + 0 * Y, Y + 0 * X, nu)
        W = (w[:, None] * w[None, :]) * h * h
        vn = space.cell_vnodes(cell)
        for a, g in enumerate(vn):
            s, t = a % (k + 1), a // (k + 1)
            phi = V[:, t][:, None] * V[:, s][None, :]
            F[2 * g] += np.sum(W * f1 * phi)
            F[2 * g + 1] += np.sum(W * f2 * phi)
    return F


def manufactured_rhs(space, K, nu=1.0):
    """b_F = F_F - K_FB g, b_B = g with g the nodal interpolant of the exact velocity on the boundary."""
    from .fem import u_exact
    mask = space.dirichlet_mask()
    X, Y = space.vnode_xy()
    u1, u2 = u_exact(X, Y)
    g = np.zeros(space.ndof)
    g[0:space.n_u:2] = u1
    g[1:space.n_u:2] = u2
    g = np.where(mask, g, 0.0)
    b = load_vector(space, nu) - K @ g
    b[mask] = g[mask]
    return b


def errors(space, x, q=None):
    """(relative H^1 velocity error, relative L^2 velocity error, L^2 pressure error with the mean
    removed) against Eq. (model_problem), tensor Gauss-Legendre rule of k + 6 points per direction."""
    from .fem import u_exact, grad_u_exact
    k, N = space.k, space.N
    q = q or (k + 6)
    xg, w = _gauss01(q)
    V, D = _basis_1d_float(k, xg)
    Vp, _ = _basis_1d_float(k - 1, xg)
    h = 1.0 / N
    W = (w[:, None] * w[None, :]) * h * h
    e_l2 = n_l2 = e_h1 = n_h1 = p_int = p_sq = area = 0.0
    for cell in space.cells:
        i, j = cell
        X = h * (i + xg)[None, :] + 0 * xg[:, None]
        Y = h * (j + xg)[:, None] + 0 * xg[None, :]
        vn, pn = space.cell_vnodes(cell), space.cell_pnodes(cell)
        u = [np.zeros_like(X), np.zeros_like(X)]
        G = [[np.zeros_like(X), np.zeros_like(X)], [np.zeros_like(X), np.zeros_like(X)]]
        for a, g in enumerate(vn):
            s, t = a % (k + 1), a // (k + 1)
            phi = V[:, t][:, None] * V[:, s][None, :]
            dx = V[:, t][:, None] * D[:, s][None, :] / h
            dy = D[:, t][:, None] * V[:, s][None, :] / h
            for c in (0, 1):
                xv = x[2 * g + c]
                u[c] += xv * phi
                G[c][0] += xv * dx
                G[c][1] += xv * dy
        ph = np.zeros_like(X)
        for a, g in enumerate(pn):
            r, t = a % k, a // k
            ph += x[space.n_u + g] * (Vp[:, t][:, None] * Vp[:, r][None, :])
        ue = u_exact(X, Y)
        Ge = grad_u_exact(X, Y)
        e_l2 += np.sum(W * ((u[0] - ue[0]) ** 2 + (u[1] - ue[1]) ** 2))
        n_l2 += np.sum(W * (ue[0] ** 2 + ue[1] ** 2))
        for c in (0, 1):
            for d in (0, 1):
                e_h1 += np.sum(W * (G[c][d] - Ge[c][d]) ** 2)
                n_h1 += np.sum(W * Ge[c][d] ** 2)
        p_int += np.sum(W * ph)
        p_sq += np.sum(W * ph ** 2)
        area += np.sum(W)
    mean = p_int / area
    p_err = np.sqrt(max(p_sq - 2 * mean * p_int + mean ** 2 * area, 0.0))
    return np.sqrt((e_l2 + e_h1) / (n_l2 + n_h1)), np.sqrt(e_l2 / n_l2), p_err
