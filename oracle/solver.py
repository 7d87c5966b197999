"""Additive Vanka relaxation, Chebyshev smoothing, V-cycle and FGMRES (Sec. 3, Algorithm 1, Sec. 4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Plain FP64 NumPy/SciPy restatement of the method, step by step:

* ``vanka_apply``: Algorithm 1 (additive subspace correction) as a preconditioner:
      M^{-1} r = sum_i R_i^T W_i A_i^{-1} R_i r   on the free DoFs,  identity on Dirichlet DoFs,
  with A_i = script-A[idx_i, idx_i] gathered from the assembled matrix ("matrix-full", Sec. 3.1 last
  paragraph) and solved by LU with partial pivoting.  Reading: W_i = I (a plain sum); the optional
  "multiplicity" weights scale each DoF by 1 / (number of patches that contain it).
* ``chebyshev``: Chebyshev acceleration of the additive smoother on the interval
  [lambda/4, 1.1 lambda] (Sec. 3, "Relaxation"); three-term recurrence of Saad, "Iterative Methods
  for Sparse Linear Systems", Algorithm 12.1, applied to the preconditioned operator.
* ``estimate_lambda``: the "standard GMRES estimation" read as 10 Arnoldi steps on M^{-1} A from a
  seeded SplitMix64 start vector (Dirichlet entries zeroed, projected off the constant pressure);
  lambda is the largest real part of the Ritz values.
* ``vcycle``: multiplicative V(nu, nu) cycle, canonical transfers, R = P^T (Sec. 3); the coarse
  Dirichlet entries of a restricted residual are zeroed; the coarsest level is solved directly with the
  bordered system [[A_c, z], [z^T, 0]] (reading: the paper does not name its coarse solver).
* ``fgmres``: right-preconditioned, unrestarted FGMRES (Sec. 3: chosen for its stored preconditioned
  vectors), zero initial guess, stop when the Givens residual estimate falls below rtol * ||b||
  (Sec. 4: relative reduction 1e10, at most 100 iterations).  Orthogonalisation: modified Gram-Schmidt.
  The pressure nullspace is handled by projecting b and every preconditioned vector off z.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import bdm, fem, patches as patches_mod, quad, splitmix

CHEB_LO = 0.25
CHEB_HI = 1.1
EIG_STEPS = 10
EIG_SEED = 0x5EED


def project(space, v):
    """Euclidean projection off the nullspace z = (0_u, 1_p): subtract the pressure mean."""
    w = v.copy()
    w[space.n_u:] -= w[space.n_u:].mean()
    return w


class Level:
    def __init__(self, space, A, mask, patch_list, weights="plain"):
        self.space = space
        self.A = A
        self.mask = mask
        self.patches = patch_list
        self.lam = None
        self.P = None       # prolongation from the next coarser level
        self.R = None
        if patch_list is None:
            return
        dofs = [p[2] for p in patch_list]
        self.slot_dofs = np.concatenate(dofs)
        self.slot_ptr = np.concatenate([[0], np.cumsum([len(d) for d in dofs])])
        Ad = A.tocsr()
        self.blocks = [Ad[d][:, d].toarray() for d in dofs]
        if weights == "plain":
            self.weight = np.ones(space.ndof)
        elif weights == "multiplicity":
            cnt = np.bincount(self.slot_dofs, minlength=space.ndof).astype(float)
            self.weight = np.where(cnt > 0, 1.0 / np.maximum(cnt, 1), 1.0)
        else:
            raise ValueError(weights)
        # group patches of equal size for batched LAPACK solves; results are placed back in
        # canonical patch order before the scatter-add
        self.groups = {}
        for i, d in enumerate(dofs):
            self.groups.setdefault(len(d), []).append(i)
        self.group_data = {}
        for n, ids in self.groups.items():
            self.group_data[n] = (np.array(ids), np.stack([self.blocks[i] for i in ids]),
                                  np.stack([dofs[i] for i in ids]))


def patch_solves(level, r):
    """delta_i = A_i^{-1} r[idx_i] for every patch (Algorithm 1, local problems); LU with partial
    pivoting (LAPACK gesv).  Returns the concatenation of the delta_i in canonical patch order."""
    out = np.empty(len(level.slot_dofs))
    for n, (ids, blocks, idx) in level.group_data.items():
        sol = np.linalg.solve(blocks, r[idx][..., None])[..., 0]
        for row, pid in enumerate(ids):
            out[level.slot_ptr[pid]:level.slot_ptr[pid + 1]] = sol[row]
    return out


def vanka_apply(level, r):
    """Additive Vanka preconditioner M^{-1} r (Algorithm 1 with the weights of ``Level``).

    Contributions to a DoF are summed in ascending patch order starting from zero; Dirichlet DoFs
    receive r itself (identity rows)."""
    delta = patch_solves(level, r)
    z = np.zeros_like(r)
    np.add.at(z, level.slot_dofs, delta * level.weight[level.slot_dofs])
    z[level.mask] = r[level.mask]
    return z


def chebyshev(A_apply, Minv, b, x, lam, nu, lo=CHEB_LO, hi=CHEB_HI):
    """nu steps of Chebyshev acceleration of the preconditioned iteration on [lo*lam, hi*lam].

    x = None means a zero initial guess, so the first residual is b (no SpMV)."""
    emax, emin = hi * lam, lo * lam
    theta = 0.5 * (emax + emin)
    delta = 0.5 * (emax - emin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b.copy() if x is None else b - A_apply(x)
    d = Minv(r) / theta
    x = d.copy() if x is None else x + d
    for _ in range(1, nu):
        r = b - A_apply(x)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * Minv(r)
        x = x + d
        rho = rho_new
    return x


def arnoldi_ritz(op, v0, steps=EIG_STEPS):
    """Ritz values of ``op`` from ``steps`` Arnoldi steps (modified Gram-Schmidt) started at v0.

    Stops early on breakdown, read as ||w after orthogonalisation|| <= 1e-12 ||op(v_j)|| (the Krylov
    space became invariant to working precision)."""
    n = len(v0)
    V = np.zeros((steps + 1, n))
    H = np.zeros((steps + 1, steps))
    V[0] = v0 / np.linalg.norm(v0)
    m = steps
    for j in range(steps):
        w = op(V[j])
        wnorm = np.linalg.norm(w)
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-12 * wnorm:
            m = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    return np.linalg.eigvals(H[:m, :m])


def eig_start_vector(level_index, space, mask, seed=EIG_SEED):
    v = splitmix.uniform_pm1(seed + level_index, space.ndof)
    v[mask] = 0.0
    return project(space, v)


def estimate_lambda(level, level_index, seed=EIG_SEED, steps=EIG_STEPS):
    """Largest real part of the Ritz values of M^{-1} A on one level (Sec. 3, "Relaxation")."""
    v0 = eig_start_vector(level_index, level.space, level.mask, seed)
    ritz = arnoldi_ritz(lambda v: vanka_apply(level, level.A @ v), v0, steps)
    return float(np.max(ritz.real))


class Hierarchy:
    """Levels 0 (coarsest, N_coarse) ... L-1 (finest, N_coarse * 2^(L-1)) for one order k.

    cell = "tri": Taylor-Hood (P_k, P_{k-1}) on triangles (Case 1 of Sec. 3); cell = "quad":
    (Q_k, Q_{k-1}) on quadrilaterals (Case 2); cell = "bdm": (BDM_k, dP_{k-1}) with the interior-penalty
    form and extended cell patches (Case 3); the same relaxation, cycle and Krylov method for all."""

    def __init__(self, N_coarse, nlevels, k, nu=1.0, sweeps=1, weights="plain", lambdas=None,
                 eig_seed=EIG_SEED, cell="tri"):
        self.k, self.nu_visc, self.sweeps, self.cell = k, nu, sweeps, cell
        disc = {"tri": (fem.Space, fem.assemble_full, patches_mod.build_patches, fem.prolongation),
                "quad": (quad.QSpace, quad.assemble_full, quad.build_patches, quad.prolongation),
                "bdm": (bdm.BDMSpace, bdm.assemble_full, bdm.build_patches, bdm.prolongation)}[cell]
        make_space, assemble, build_patches, prolong = disc
        self.levels = []
        for l in range(nlevels):
            space = make_space(N_coarse * 2 ** l, k)
            K = assemble(space, nu)
            mask = space.dirichlet_mask()
            A = fem.apply_dirichlet(K, mask)
            plist = build_patches(space) if l > 0 else None
            lev = Level(space, A, mask, plist, weights)
            lev.K = K
            if l > 0:
                lev.P = prolong(self.levels[l - 1].space, space)
                lev.R = lev.P.T.tocsr()
            self.levels.append(lev)
        c = self.levels[0]
        n = c.space.ndof
        z = c.space.nullspace()
        Bd = np.zeros((n + 1, n + 1))
        Bd[:n, :n] = c.A.toarray()
        Bd[:n, n] = z
        Bd[n, :n] = z
        self.coarse_lu = sla.lu_factor(Bd)
        for l in range(1, nlevels):
            lev = self.levels[l]
            lev.lam = (lambdas[l] if lambdas is not None else estimate_lambda(lev, l, eig_seed))

    @property
    def finest(self):
        return self.levels[-1]

    def coarse_solve(self, b):
        """Bordered solve [[A_c, z], [z^T, 0]] [x; mu] = [b; 0]: x is the solution orthogonal to z."""
        n = len(b)
        rhs = np.concatenate([b, [0.0]])
        return sla.lu_solve(self.coarse_lu, rhs)[:n]

    def smooth(self, l, b, x):
        lev = self.levels[l]
        return chebyshev(lambda v: lev.A @ v, lambda r: vanka_apply(lev, r), b, x, lev.lam, self.sweeps)

    def vcycle(self, b, l=None):
        """Multiplicative V(nu, nu) cycle on level l (default finest) with zero initial guess."""
        if l is None:
            l = len(self.levels) - 1
        if l == 0:
            return self.coarse_solve(b)
        lev = self.levels[l]
        x = self.smooth(l, b, None)
        r = b - lev.A @ x
        rc = lev.R @ r
        rc[self.levels[l - 1].mask] = 0.0
        ec = self.vcycle(rc, l - 1)
        x = x + lev.P @ ec
        return self.smooth(l, b, x)


class FGMRESResult:
    def __init__(self, x, iters, hist, true_res, converged):
        self.x, self.iters, self.hist, self.true_res, self.converged = x, iters, hist, true_res, converged


def fgmres(A_apply, prec, b, rtol, maxit, proj=lambda v: v, orth="mgs"):
    """Right-preconditioned unrestarted FGMRES with zero initial guess (Sec. 3, Sec. 4).

    The paper does not fix the orthogonalisation: orth = "mgs" (modified Gram-Schmidt, the default)
    or "cgs2" (classical Gram-Schmidt applied twice, each pass projecting against the whole basis
    with one set of inner products).  hist[0] = ||b||, hist[j] = Givens residual estimate after j
    iterations.  Stops at hist[j] <= rtol * hist[0] or after maxit iterations."""
    if orth not in ("mgs", "cgs2"):
        raise ValueError("orth must be 'mgs' or 'cgs2'")
    b = proj(b)
    beta = np.linalg.norm(b)
    n = len(b)
    if beta == 0.0:
        return FGMRESResult(np.zeros(n), 0, [0.0], 0.0, True)
    V = [b / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    hist = [beta]
    m = 0
    converged = False
    for j in range(maxit):
        z = proj(prec(V[j]))
        Z.append(z)
        w = A_apply(z)
        if orth == "mgs":
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
        else:
            Vj = np.array(V[:j + 1])
            for _ in range(2):
                h = Vj @ w
                w = w - Vj.T @ h
                H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = np.hypot(H[j, j], H[j + 1, j])
        cs[j] = H[j, j] / den
        sn[j] = H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        hist.append(abs(g[j + 1]))
        m = j + 1
        if abs(g[j + 1]) <= rtol * beta:
            converged = True
            break
    y = sla.solve_triangular(H[:m, :m], g[:m])
    x = np.zeros(n)
    for i in range(m):
        x = x + y[i] * Z[i]
    true_res = np.linalg.norm(b - A_apply(x))
    return FGMRESResult(x, m, hist, true_res, converged)


def solve(H, b, rtol=1e-8, maxit=100, orth="mgs"):
    """FGMRES preconditioned by one V-cycle on the finest level of hierarchy H."""
    fin = H.finest
    return fgmres(lambda v: fin.A @ v, H.vcycle, b, rtol, maxit, lambda v: project(fin.space, v), orth)


def direct_solve(A, z, b):
    """Sparse bordered solve [[A, z], [z^T, 0]] for reference solutions (SuperLU)."""
    n = A.shape[0]
    Bd = sp.bmat([[A, sp.csr_matrix(z[:, None])], [sp.csr_matrix(z[None, :]), None]]).tocsc()
    return spla.spsolve(Bd, np.concatenate([b, [0.0]]))[:n]
