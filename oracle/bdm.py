"""H(div)-L^2 discretization (BDM_k, dP_{k-1}) with the interior-penalty form (Case 3 of Sec. 3, Sec. 2.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows the paper:
* BDM_k(T) = vector P_k on each triangle with the normal component continuous across edges (Sec. 2.1);
  pressures in the discontinuous P_{k-1}, mean zero.
* The no-flux condition u . n = 0 is imposed strongly (Eq. StokesBCforDGFEM1); the tangential
  normal-stress condition (Eq. StokesBCforDGFEM2) is natural, so the form only sums over interior edges.
* a_h(u, v) = 2 nu [ sum_T int_T eps(u):eps(v) - sum_e int_e {eps(u)}:[[v]]^t - sum_e int_e [[u]]^t:{eps(v)} ]
             + 2 nu alpha sum_e h_e^{-1} int_e [[u]]^t:[[v]]^t           (Eq. DiscontBilinearForm)
  with [[v]] = v1 (.) n1 + v2 (.) n2, v (.) n = (v n^T + n v^T) / 2, {t} = (t1 + t2) / 2, and the
  tangential part [[v]]^t = [[(v . t) t]]; b(v, q) = -int (div v) q (Eq. VariationalStokesb).
* Extended cell Vanka patches (Sec. 3.1): for each cell, its pressure DoFs and the velocity DoFs of the
  cell and of its (up to three) edge neighbours.
* Nested spaces under uniform refinement; canonical transfers interpolate the natural embedding (Sec. 3).

Readings where the paper is silent:
* DoFs of BDM_k on a cell: the normal flux v(x_j) . rot(x_b - x_a) at the k + 1 points
  x_j = x_a + (j + 1)/(k + 2) (x_b - x_a) of each edge (a, b) (rot(x, y) = (y, -x), so rot(x_b - x_a) is
  the normal scaled by the edge length), and the moments int v . q for q in Nedelec's first-kind space
  of degree k - 1 (P_{k-2}^2 plus (-y, x) times homogeneous P_{k-2}), with the q orthogonalised in
  L^2 of the reference cell and scaled to norms in [1, 2) by powers of two; global edge DoFs use the edge
  oriented from its lower to its higher vertex id, and a cell whose local edge runs the other way sees
  them with the opposite sign at mirrored points.  The contravariant Piola map v = J v_ref / det J
  carries the reference basis to every cell; with the scaled normal the edge DoFs are Piola invariant.
  (Moments against the raw monomials give a badly scaled basis: diagonal entries from 1 to 2e7 at
  k = 3 and FGMRES counts, which minimise the Euclidean residual of the DoF vector, of 70 to 160 where
  the orthogonalised moments give 30 to 36 at every k and mesh.)
* penalty alpha = (k + 1)(k + 2) (the paper only asks for "sufficiently large"): twice the k-dependence
  (k + 1)(k + 2) / 2 of the trace inverse inequality on triangles; on this mesh family a_h stops being
  coercive just below (k + 1)(k + 2) / 2 (k = 2: between 5 and 6; k = 3: between 10 and 12; k = 4:
  between 16 and 20), and a much larger alpha (10 k^2) doubles the iteration counts.
* DoF order: edge DoFs (edges horizontal, vertical, diagonal, each lexicographic; j ascending), then the
  interior DoFs of each cell (cells lower then upper), then the pressure DoFs cell by cell (equispaced
  P_{k-1} Lagrange nodes, discontinuous).  Dirichlet DoFs: the edge DoFs of boundary edges (u . n = 0).
* patches exclude Dirichlet DoFs; cells in canonical order (lower, then upper triangles, lexicographic).

Exactness: reference bases and transfers are exact rationals; element and edge integrals are evaluated
in FP64 (the diagonal edge's unit normal is irrational) with Gauss rules exact for the polynomial degrees.
"""
from fractions import Fraction
from functools import lru_cache

import numpy as np
import scipy.sparse as sp

from . import exact

# ---------------------------------------------------------------------------- reference element
_VERTS = [(Fraction(0), Fraction(0)), (Fraction(1), Fraction(0)), (Fraction(0), Fraction(1))]
_EDGES = [(1, 2), (0, 2), (0, 1)]     # local edge i is opposite local vertex i, traversed a -> b


def _rot(v):
    return (v[1], -v[0])


def _mono_vec(k):
    """Vector monomials of P_k^2: (component, p, q)."""
    return [(c, p, q) for c in (0, 1) for q in range(k + 1) for p in range(k + 1 - q)]


def _ned_monomial(k):
    """Nedelec's first-kind space of degree k - 1 spanned by monomial pairs: P_{k-2}^2 (x then y component
    for each monomial, q outer), then (-y, x) times the homogeneous monomials of degree k - 2."""
    out = []
    for q in range(k - 1):
        for p in range(k - 1 - q):
            out.append(({(p, q): Fraction(1)}, {}))
            out.append(({}, {(p, q): Fraction(1)}))
    d = k - 2
    if d >= 0:
        for q in range(d + 1):
            p = d - q
            # (-y, x) x^p y^q
            out.append(({(p, q + 1): Fraction(-1)}, {(p + 1, q): Fraction(1)}))
    return out


def _ned_inner(a, b):
    """L^2 inner product over the reference triangle of two polynomial pairs (exact)."""
    tot = Fraction(0)
    for c in (0, 1):
        for (p, q), u in a[c].items():
            for (r, s), v in b[c].items():
                tot += u * v * exact.integrate_ref({(p + r, q + s): 1})
    return tot


@lru_cache(maxsize=None)
def _ned_space_cached(k):
    out, norms = [], []
    for f in _ned_monomial(k):
        e = [dict(f[0]), dict(f[1])]
        for g, gg in zip(out, norms):
            c = _ned_inner(e, g) / gg
            for comp in (0, 1):
                for pq, u in g[comp].items():
                    v = e[comp].get(pq, 0) - c * u
                    if v == 0:
                        e[comp].pop(pq, None)
                    else:
                        e[comp][pq] = v
        out.append(e)
        norms.append(_ned_inner(e, e))
    scaled = []
    for e, n2 in zip(out, norms):
        t = n2.numerator.bit_length() - n2.denominator.bit_length()   # floor(log2 n2) is t or t - 1
        if Fraction(2) ** t > n2:
            t -= 1
        s = Fraction(2) ** (-(t // 2))                                 # s^2 n2 in [1, 4)
        scaled.append(({pq: s * u for pq, u in e[0].items()}, {pq: s * u for pq, u in e[1].items()}))
    return tuple(scaled)


def _ned_space(k):
    """Test functions of the interior moments: the monomial pairs of _ned_monomial orthogonalised in
    L^2 of the reference triangle (Gram-Schmidt in that order, exact) and each scaled by the power of
    two 2^-floor(floor(log2 |q|^2) / 2), so that its norm lies in [1, 2)."""
    return list(_ned_space_cached(k))


@lru_cache(maxsize=None)
def reference_basis(k):
    """Reference BDM_k basis as pairs of polynomial dicts (x-component, y-component), dual to the local
    DoFs: edge e (a, b), point j = 0..k at index e*(k+1) + j, then the interior moments."""
    monos = _mono_vec(k)
    funcs = []
    for (a, b) in _EDGES:
        va, vb = _VERTS[a], _VERTS[b]
        nu = _rot((vb[0] - va[0], vb[1] - va[1]))
        for j in range(k + 1):
            t = Fraction(j + 1, k + 2)
            x = va[0] + t * (vb[0] - va[0])
            y = va[1] + t * (vb[1] - va[1])
            funcs.append(("pt", x, y, nu))
    for q in _ned_space(k):
        funcs.append(("mom", q))
    n = len(monos)
    assert len(funcs) == n == (k + 1) * (k + 2)
    V = [[Fraction(0)] * n for _ in range(n)]
    for i, f in enumerate(funcs):
        for m, (c, p, q) in enumerate(monos):
            if f[0] == "pt":
                _, x, y, nu = f
                V[i][m] = (x ** p) * (y ** q) * nu[c]
            else:
                qq = f[1][c]
                V[i][m] = sum(coef * exact.integrate_ref({(p + pp, q + qq_): 1}) for (pp, qq_), coef in qq.items())
    eye = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    C = exact._solve_exact(V, eye)       # V C = I: column i = coefficients of basis function i
    basis = []
    for i in range(n):
        bx, by = {}, {}
        for m, (c, p, q) in enumerate(monos):
            if C[m][i] != 0:
                (bx if c == 0 else by)[(p, q)] = C[m][i]
        basis.append((bx, by))
    return tuple(basis)


def _eval(poly, x, y):
    return sum(c * x ** p * y ** q for (p, q), c in poly.items())


def _deriv(poly, var):
    return exact.deriv(poly, var)


# ---------------------------------------------------------------------------- mesh and DoFs
class BDMSpace:
    """BDM_k velocity / dP_{k-1} pressure on the structured triangle mesh (cells as in fem.Mesh)."""

    cell_type = "tri"

    def __init__(self, N, k):
        assert k >= 1
        self.N, self.k = N, k
        N1 = N + 1
        lower = [((i, j), (i + 1, j), (i, j + 1)) for j in range(N) for i in range(N)]
        upper = [((i + 1, j), (i + 1, j + 1), (i, j + 1)) for j in range(N) for i in range(N)]
        self.cells = lower + upper
        vid = lambda v: v[1] * N1 + v[0]
        edges = [((i, j), (i + 1, j)) for j in range(N + 1) for i in range(N)]          # horizontal
        edges += [((i, j), (i, j + 1)) for j in range(N) for i in range(N + 1)]         # vertical
        edges += [((i + 1, j), (i, j + 1)) for j in range(N) for i in range(N)]         # diagonal
        self.edges = [tuple(sorted(e, key=vid)) for e in edges]   # oriented lower id -> higher id
        self.edge_id = {e: n for n, e in enumerate(self.edges)}
        self.vid = vid
        ne, nc = len(self.edges), len(self.cells)
        self.n_edge = ne * (k + 1)
        self.n_int = nc * (k + 1) * (k - 1)
        self.n_u = self.n_edge + self.n_int
        self.nq = k * (k + 1) // 2
        self.n_p = nc * self.nq
        self.ndof = self.n_u + self.n_p

    def cell_dofs(self, c):
        """(global velocity DoFs, signs) in local order, and global pressure DoFs of cell c."""
        k = self.k
        cell = self.cells[c]
        dofs, signs = [], []
        for (a, b) in _EDGES:
            ga, gb = cell[a], cell[b]
            e = self.edge_id[tuple(sorted((ga, gb), key=self.vid))]
            same = self.vid(ga) < self.vid(gb)
            for j in range(k + 1):
                jj = j if same else k - j
                dofs.append(e * (k + 1) + jj)
                signs.append(1.0 if same else -1.0)
        ni = (k + 1) * (k - 1)
        for m in range(ni):
            dofs.append(self.n_edge + c * ni + m)
            signs.append(1.0)
        pd = [self.n_u + c * self.nq + m for m in range(self.nq)]
        return dofs, signs, pd

    def dirichlet_mask(self):
        mask = np.zeros(self.ndof, dtype=bool)
        k, N = self.k, self.N
        for n, (va, vb) in enumerate(self.edges):
            on = (va[0] == vb[0] and va[0] in (0, N)) or (va[1] == vb[1] and va[1] in (0, N))
            if on:
                mask[n * (k + 1):(n + 1) * (k + 1)] = True
        return mask

    def nullspace(self):
        z = np.zeros(self.ndof)
        z[self.n_u:] = 1.0
        return z

    def geometry(self, c, h):
        """Affine map x = x0 + J xhat of cell c (physical units)."""
        (x0, y0), (x1, y1), (x2, y2) = self.cells[c]
        J = h * np.array([[x1 - x0, x2 - x0], [y1 - y0, y2 - y0]], dtype=float)
        return h * np.array([x0, y0], dtype=float), J


# ---------------------------------------------------------------------------- float evaluation
def _gauss01(q):
    g, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (g + 1.0), 0.5 * w


def _tri_rule(q):
    gx, gw = _gauss01(q)
    S, T = np.meshgrid(gx, gx, indexing="ij")
    WS, WT = np.meshgrid(gw, gw, indexing="ij")
    return S.ravel(), (T * (1 - S)).ravel(), (WS * WT * (1 - S)).ravel()


@lru_cache(maxsize=None)
def _ref_eval(k, pts_key):
    """Values and reference gradients of the reference basis at points (tuple of (x, y))."""
    B = reference_basis(k)
    pts = np.array(pts_key, dtype=float).reshape(-1, 2)
    x, y = pts[:, 0], pts[:, 1]
    nb = len(B)
    val = np.zeros((len(x), nb, 2))
    grad = np.zeros((len(x), nb, 2, 2))      # grad[., ., c, d] = d_d vhat_c
    for i, comps in enumerate(B):
        for c in (0, 1):
            poly = {pq: float(v) for pq, v in comps[c].items()}
            val[:, i, c] = sum(v * x ** p * y ** q for (p, q), v in poly.items()) if poly else 0.0
            for d in (0, 1):
                dp = {pq: float(v) for pq, v in _deriv(comps[c], d).items()}
                grad[:, i, c, d] = sum(v * x ** p * y ** q for (p, q), v in dp.items()) if dp else 0.0
    return val, grad


def _piola(J, val, grad):
    """Physical values J v / det J and gradients J (grad vhat) J^{-1} / det J."""
    det = np.linalg.det(J)
    Ji = np.linalg.inv(J)
    v = np.einsum("cd,xid->xic", J, val) / det
    g = np.einsum("ca,xiab,bd->xicd", J, grad, Ji) / det
    return v, g


def penalty(k):
    return float((k + 1) * (k + 2))


def assemble_full(space, nu=1.0):
    """[[A, B^T], [B, 0]] before the no-flux condition (FP64): cell terms, interior-edge terms of Eq.
    (DiscontBilinearForm), divergence form."""
    k, N = space.k, space.N
    h = 1.0 / N
    alpha = penalty(k)
    xs, ys, ws = _tri_rule(k + 2)
    pts = tuple(zip(xs.tolist(), ys.tolist()))
    val, grad = _ref_eval(k, pts)
    psi = _pressure_basis_at(k, xs, ys)
    rows, cols, vals = [], [], []
    cellinfo = []
    for c in range(len(space.cells)):
        x0, J = space.geometry(c, h)
        v, g = _piola(J, val, grad)
        w = ws * abs(np.linalg.det(J))
        dofs, signs, pd = space.cell_dofs(c)
        sg = np.array(signs)
        eps = 0.5 * (g + np.swapaxes(g, 2, 3))
        Ae = 2 * nu * np.einsum("x,xicd,xjcd->ij", w, eps, eps)
        div = g[:, :, 0, 0] + g[:, :, 1, 1]
        Be = -np.einsum("x,xq,xi->qi", w, psi, div)
        Ae = 0.5 * (Ae + Ae.T)                   # symmetric form: remove summation-order asymmetry
        Ae = sg[:, None] * Ae * sg[None, :]
        Be = Be * sg[None, :]
        for a, da in enumerate(dofs):
            for b, db in enumerate(dofs):
                rows.append(da); cols.append(db); vals.append(Ae[a, b])
        for q, dq in enumerate(pd):
            for b, db in enumerate(dofs):
                rows += [dq, db]; cols += [db, dq]; vals += [Be[q, b], Be[q, b]]
        cellinfo.append((x0, J, dofs, sg))
    # interior edges
    cells_of_edge = {}
    for c, cell in enumerate(space.cells):
        for (a, b) in _EDGES:
            e = space.edge_id[tuple(sorted((cell[a], cell[b]), key=space.vid))]
            cells_of_edge.setdefault(e, []).append(c)
    ge, gw = _gauss01(k + 1)
    for e, cs in cells_of_edge.items():
        if len(cs) != 2:
            continue
        va, vb = [np.array(p, dtype=float) * h for p in space.edges[e]]
        tau = vb - va
        he = np.linalg.norm(tau)
        t = tau / he
        X = va[None, :] + ge[:, None] * tau[None, :]
        W = gw * he
        side = []
        for c in cs:
            x0, J, dofs, sg = cellinfo[c]
            ref = np.linalg.solve(J, (X - x0[None, :]).T).T
            vv, gg = _ref_eval(k, tuple(map(tuple, ref.tolist())))
            v, g = _piola(J, vv, gg)
            v = v * sg[None, :, None]
            g = g * sg[None, :, None, None]
            centroid = x0 + J @ np.array([1 / 3, 1 / 3])
            n = np.array([t[1], -t[0]])
            if np.dot(n, centroid - va) > 0:
                n = -n                         # outward from this cell
            side.append((dofs, v, g, n))
        (d1, v1, g1, n1), (d2, v2, g2, n2) = side
        # tangential jump jt(w) = (w1 - w2) . t (times t (.) n1) and the average of eps : (t (.) n1)
        jt1 = np.einsum("xic,c->xi", v1, t)
        jt2 = -np.einsum("xic,c->xi", v2, t)
        e1 = 0.5 * (g1 + np.swapaxes(g1, 2, 3))
        e2 = 0.5 * (g2 + np.swapaxes(g2, 2, 3))
        tn = 0.5 * (np.outer(t, n1) + np.outer(n1, t))
        av1 = 0.5 * np.einsum("xicd,cd->xi", e1, tn)
        av2 = 0.5 * np.einsum("xicd,cd->xi", e2, tn)
        dofs = list(d1) + list(d2)
        JT = np.concatenate([jt1, jt2], axis=1)
        AV = np.concatenate([av1, av2], axis=1)
        # [[u]]^t : [[v]]^t = jt(u) jt(v) (t (.) n):(t (.) n) = jt(u) jt(v) / 2
        Ee = 2 * nu * (-np.einsum("x,xi,xj->ij", W, AV, JT) - np.einsum("x,xi,xj->ij", W, JT, AV)) \
            + 2 * nu * alpha / he * 0.5 * np.einsum("x,xi,xj->ij", W, JT, JT)
        Ee = 0.5 * (Ee + Ee.T)
        for a, da in enumerate(dofs):
            for b, db in enumerate(dofs):
                rows.append(da); cols.append(db); vals.append(Ee[a, b])
    K = sp.coo_matrix((vals, (rows, cols)), shape=(space.ndof, space.ndof)).tocsr()
    K.sum_duplicates()
    K = ((K + K.T) * 0.5).tocsr()       # the form is symmetric; duplicates were summed in different orders
    K.sort_indices()
    return K


def _pressure_basis_at(k, xs, ys):
    """dP_{k-1} Lagrange basis (equispaced nodes, exact.lattice_nodes order) at reference points."""
    B = exact.basis(k - 1)
    return np.stack([sum(float(c) * xs ** p * ys ** q for (p, q), c in f.items()) for f in B], axis=1)


# ---------------------------------------------------------------------------- transfers
def _cell_of_point(space, X, Y):
    """Cell containing the point (units of h; exact rationals): lower / upper triangle of its square."""
    N = space.N
    i = min(int(X), N - 1)
    j = min(int(Y), N - 1)
    fx, fy = X - i, Y - j
    return j * N + i if fx + fy <= 1 else N * N + j * N + i


def _coarse_value(space, c, X, Y):
    """Exact values of the Piola-mapped reference basis of cell c at the point (units of h)."""
    cell = space.cells[c]
    (x0, y0), (x1, y1), (x2, y2) = cell
    J = [[Fraction(x1 - x0), Fraction(x2 - x0)], [Fraction(y1 - y0), Fraction(y2 - y0)]]
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0]
    dx, dy = X - x0, Y - y0
    xh = (J[1][1] * dx - J[0][1] * dy) / det
    yh = (-J[1][0] * dx + J[0][0] * dy) / det
    out = []
    for bx, by in reference_basis(space.k):
        vx, vy = _eval(bx, xh, yh), _eval(by, xh, yh)
        # Piola in units of h: the factor h of J cancels against 1 / det (h^2) up to 1/h, common to
        # every function of the level; the fine functionals below carry the matching h
        out.append(((J[0][0] * vx + J[0][1] * vy) / det, (J[1][0] * vx + J[1][1] * vy) / det))
    return out


def prolongation(coarse, fine):
    """P: fine DoFs of every coarse basis function (exact rationals; Sec. 3, natural embedding)."""
    assert fine.N == 2 * coarse.N and fine.k == coarse.k
    k = coarse.k
    rows, cols, vals = [], [], []

    def coarse_field(Xc, Yc, c=None):
        """Coarse basis values at a point given in coarse units: list of (global coarse DoF, sign,
        (vx, vy)); c fixes the coarse cell (needed on coarse edges, where tangential parts jump)."""
        if c is None:
            c = _cell_of_point(coarse, Xc, Yc)
        dofs, signs, _ = coarse.cell_dofs(c)
        vs = _coarse_value(coarse, c, Xc, Yc)
        # the signs as exact integers: a float sign would turn the moment sums below into float sums
        return [(d, int(s), v) for d, s, v in zip(dofs, signs, vs)]

    # fine edge DoFs: normal flux at the fine edge points; fine units are half the coarse ones, and the
    # Piola factor 1/h doubles on the fine level while rot(x_b - x_a) halves: both in coarse units below
    for n, (va, vb) in enumerate(fine.edges):
        nu_c = (Fraction(vb[1] - va[1], 2), -Fraction(vb[0] - va[0], 2))   # rot of the edge in coarse units
        for j in range(k + 1):
            t = Fraction(j + 1, k + 2)
            Xc = (va[0] + t * (vb[0] - va[0])) / 2
            Yc = (va[1] + t * (vb[1] - va[1])) / 2
            for d, s, (vx, vy) in coarse_field(Xc, Yc):
                val = s * (vx * nu_c[0] + vy * nu_c[1])
                if val != 0:
                    rows.append(n * (k + 1) + j); cols.append(d); vals.append(float(val))
    # fine interior DoFs: reference moments of the pulled-back coarse function on each fine cell
    ned = _ned_space(k)
    ni = (k + 1) * (k - 1)
    if ni:
        # exact Gauss-free evaluation: the pulled-back coarse function is a polynomial on the fine
        # reference cell; integrate it against each Nedelec function by sampling at the lattice of
        # degree 2k and fitting exactly (interpolation in P_{2k} is exact for these products)
        deg = 2 * k
        nodes = exact.lattice_nodes(deg)
        mons = exact.monomials(deg)
        Vm = [[Fraction(s, deg) ** p * Fraction(t, deg) ** q for (p, q) in mons] for (s, t) in nodes]
        intm = [exact.integrate_ref({pq: 1}) for pq in mons]
        # weights w_node such that sum_node w f(node) = int_T f for every f in P_{2k}
        wts = exact._solve_exact([list(r) for r in zip(*Vm)], [[v] for v in intm])
        wts = [r[0] for r in wts]
        for c, cell in enumerate(fine.cells):
            (x0, y0), (x1, y1), (x2, y2) = cell
            Jf = [[Fraction(x1 - x0), Fraction(x2 - x0)], [Fraction(y1 - y0), Fraction(y2 - y0)]]
            cc = _cell_of_point(coarse, Fraction(x0 + x1 + x2, 6), Fraction(y0 + y1 + y2, 6))
            acc = {}
            for (s, t), wgt in zip(nodes, wts):
                xh, yh = Fraction(s, deg), Fraction(t, deg)
                X = x0 + Jf[0][0] * xh + Jf[0][1] * yh
                Y = y0 + Jf[1][0] * xh + Jf[1][1] * yh
                for d, sg, (vx, vy) in coarse_field(Fraction(X, 2), Fraction(Y, 2), cc):
                    # pull back to the fine reference cell: vhat = det J_f J_f^{-1} v (units: the coarse
                    # Piola factor in coarse units times 1/2 per fine unit)
                    ux = (Jf[1][1] * vx - Jf[0][1] * vy) / 2
                    uy = (-Jf[1][0] * vx + Jf[0][0] * vy) / 2
                    for m, (qx, qy) in enumerate(ned):
                        contrib = wgt * sg * (ux * _eval(qx, xh, yh) + uy * _eval(qy, xh, yh))
                        if contrib != 0:
                            key = (m, d)
                            acc[key] = acc.get(key, 0) + contrib
            for (m, d), v in acc.items():
                if v != 0:
                    rows.append(fine.n_edge + c * ni + m); cols.append(d); vals.append(float(v))
    # pressure: dP_{k-1} Lagrange values of the coarse pressure at the fine nodes
    Bq = exact.basis(k - 1)
    pn = exact.lattice_nodes(k - 1)
    for c, cell in enumerate(fine.cells):
        (x0, y0), (x1, y1), (x2, y2) = cell
        _, _, pdf = fine.cell_dofs(c)
        for m, (s, t) in enumerate(pn):
            if k == 1:
                xh = yh = Fraction(1, 3)
            else:
                xh, yh = Fraction(s, k - 1), Fraction(t, k - 1)
            X = x0 + (x1 - x0) * xh + (x2 - x0) * yh
            Y = y0 + (y1 - y0) * xh + (y2 - y0) * yh
            cc = _cell_of_point(coarse, Fraction(x0 + x1 + x2, 6), Fraction(y0 + y1 + y2, 6))
            (a0, b0), (a1, b1), (a2, b2) = coarse.cells[cc]
            Jc = [[Fraction(a1 - a0), Fraction(a2 - a0)], [Fraction(b1 - b0), Fraction(b2 - b0)]]
            det = Jc[0][0] * Jc[1][1] - Jc[0][1] * Jc[1][0]
            dx, dy = Fraction(X, 2) - a0, Fraction(Y, 2) - b0
            xc = (Jc[1][1] * dx - Jc[0][1] * dy) / det
            yc = (-Jc[1][0] * dx + Jc[0][0] * dy) / det
            _, _, pdc = coarse.cell_dofs(cc)
            for mm, f in enumerate(Bq):
                v = _eval(f, xc, yc)
                if v != 0:
                    rows.append(pdf[m]); cols.append(pdc[mm]); vals.append(float(v))
    P = sp.coo_matrix((vals, (rows, cols)), shape=(fine.ndof, coarse.ndof)).tocsr()
    P.sum_duplicates()
    P.sort_indices()
    return P


# ---------------------------------------------------------------------------- patches (Sec. 3.1)
def build_patches(space):
    """Extended cell patches: ('cell', c, dofs) with the pressure DoFs of cell c and the free velocity
    DoFs of c and of its edge neighbours, ascending."""
    mask = space.dirichlet_mask()
    cells_of_edge = {}
    for c, cell in enumerate(space.cells):
        for (a, b) in _EDGES:
            e = space.edge_id[tuple(sorted((cell[a], cell[b]), key=space.vid))]
            cells_of_edge.setdefault(e, []).append(c)
    out = []
    for c, cell in enumerate(space.cells):
        nbrs = {c}
        for (a, b) in _EDGES:
            e = space.edge_id[tuple(sorted((cell[a], cell[b]), key=space.vid))]
            nbrs.update(cells_of_edge[e])
        vel = set()
        for d in sorted(nbrs):
            dofs, _, _ = space.cell_dofs(d)
            vel.update(x for x in dofs if not mask[x])
        _, _, pd = space.cell_dofs(c)
        out.append(("cell", c, np.array(sorted(vel) + list(pd), dtype=np.int64)))
    return out


def interior_patch_size(k):
    """Cell and its three neighbours: 4 (k+1)(k+2) velocity DoFs less 3 (k+1) shared, plus P_{k-1}."""
    return 4 * (k + 1) * (k + 2) - 3 * (k + 1) + k * (k + 1) // 2


# ---------------------------------------------------------------------------- fields and errors
def evaluate(space, x, c, pts_ref):
    """Velocity (values, gradients) of the global vector x on cell c at reference points (n, 2)."""
    h = 1.0 / space.N
    x0, J = space.geometry(c, h)
    val, grad = _ref_eval(space.k, tuple(map(tuple, np.asarray(pts_ref, dtype=float).tolist())))
    v, g = _piola(J, val, grad)
    dofs, signs, _ = space.cell_dofs(c)
    coef = x[dofs] * np.array(signs)
    return np.einsum("xic,i->xc", v, coef), np.einsum("xicd,i->xcd", g, coef)


def interpolate(space, fu, fp=None):
    """Global DoFs of a velocity field fu(X, Y) -> (u1, u2) (physical coordinates): normal fluxes at the
    edge points, reference moments of the pulled-back field; pressure fp(X, Y) at the dP_{k-1} nodes."""
    k, N = space.k, space.N
    h = 1.0 / N
    out = np.zeros(space.ndof)
    for n, (va, vb) in enumerate(space.edges):
        A, B = np.array(va, float) * h, np.array(vb, float) * h
        nu = np.array([B[1] - A[1], -(B[0] - A[0])])
        for j in range(k + 1):
            t = (j + 1) / (k + 2)
            P = A + t * (B - A)
            u1, u2 = fu(P[0], P[1])
            out[n * (k + 1) + j] = u1 * nu[0] + u2 * nu[1]
    ned = _ned_space(k)
    ni = (k + 1) * (k - 1)
    xs, ys, ws = _tri_rule(k + 2)
    for c in range(len(space.cells)):
        x0, J = space.geometry(c, h)
        X = x0[0] + J[0, 0] * xs + J[0, 1] * ys
        Y = x0[1] + J[1, 0] * xs + J[1, 1] * ys
        u1, u2 = fu(X, Y)
        uh = np.linalg.det(J) * np.linalg.solve(J, np.stack([u1 + 0 * xs, u2 + 0 * xs]))   # pull back
        for m, (qx, qy) in enumerate(ned):
            qxv = sum(float(cf) * xs ** a * ys ** b for (a, b), cf in qx.items()) if qx else 0 * xs
            qyv = sum(float(cf) * xs ** a * ys ** b for (a, b), cf in qy.items()) if qy else 0 * xs
            out[space.n_edge + c * ni + m] = np.sum(ws * (uh[0] * qxv + uh[1] * qyv))
        if fp is not None:
            _, _, pd = space.cell_dofs(c)
            nodes = exact.lattice_nodes(k - 1)
            for m, (s_, t_) in enumerate(nodes):
                xh, yh = (s_ / (k - 1), t_ / (k - 1)) if k > 1 else (1 / 3, 1 / 3)
                out[pd[m]] = fp(x0[0] + J[0, 0] * xh + J[0, 1] * yh, x0[1] + J[1, 0] * xh + J[1, 1] * yh)
    return out


def load_vector(space, nu=1.0, q=None):
    """<f, v> with f = 2 pi^2 nu u of Eq. (model_problem) (p = 0), collapsed rule of k + 5 points."""
    from .fem import f_exact
    k, N = space.k, space.N
    h = 1.0 / N
    xs, ys, ws = _tri_rule(q or (k + 5))
    val, grad = _ref_eval(k, tuple(zip(xs.tolist(), ys.tolist())))
    F = np.zeros(space.ndof)
    for c in range(len(space.cells)):
        x0, J = space.geometry(c, h)
        v, _ = _piola(J, val, grad)
        X = x0[0] + J[0, 0] * xs + J[0, 1] * ys
        Y = x0[1] + J[1, 0] * xs + J[1, 1] * ys
        f1, f2 = f_exact(X, Y, nu)
        w = ws * abs(np.linalg.det(J))
        dofs, signs, _ = space.cell_dofs(c)
        F[dofs] += np.array(signs) * np.einsum("x,xi->i", w, v[:, :, 0] * f1[:, None] + v[:, :, 1] * f2[:, None])
    return F


def errors(space, x, q=None):
    """(relative broken H^1 velocity error, relative L^2 velocity error, L^2 pressure error with the
    mean removed) against Eq. (model_problem)."""
    from .fem import u_exact, grad_u_exact
    k, N = space.k, space.N
    h = 1.0 / N
    xs, ys, ws = _tri_rule(q or (k + 6))
    pts = np.stack([xs, ys], axis=1)
    psi = _pressure_basis_at(k, xs, ys)
    e_l2 = n_l2 = e_h1 = n_h1 = p_int = p_sq = area = 0.0
    for c in range(len(space.cells)):
        x0, J = space.geometry(c, h)
        u, g = evaluate(space, x, c, pts)
        X = x0[0] + J[0, 0] * xs + J[0, 1] * ys
        Y = x0[1] + J[1, 0] * xs + J[1, 1] * ys
        w = ws * abs(np.linalg.det(J))
        ue = u_exact(X, Y)
        Ge = grad_u_exact(X, Y)
        e_l2 += np.sum(w * ((u[:, 0] - ue[0]) ** 2 + (u[:, 1] - ue[1]) ** 2))
        n_l2 += np.sum(w * (ue[0] ** 2 + ue[1] ** 2))
        for a in (0, 1):
            for b in (0, 1):
                e_h1 += np.sum(w * (g[:, a, b] - Ge[a][b]) ** 2)
                n_h1 += np.sum(w * Ge[a][b] ** 2)
        _, _, pd = space.cell_dofs(c)
        ph = psi @ x[pd]
        p_int += np.sum(w * ph)
        p_sq += np.sum(w * ph ** 2)
        area += np.sum(w)
    mean = p_int / area
    return (np.sqrt((e_l2 + e_h1) / (n_l2 + n_h1)), np.sqrt(e_l2 / n_l2),
            np.sqrt(max(p_sq - 2 * mean * p_int + mean ** 2 * area, 0.0)))
