"""GPU parity for (BDM_k, dP_{k-1}) with the interior-penalty form (Case 3 of Sec. 3, results of Sec. 4.3):
the same C ABI and kernels as the Taylor-Hood cases, with the library's H(div) discretization, transfers
and extended cell patches (Sec. 3.1) against the oracle's.

Tolerances: one Vanka application 1e-10 (stored Gauss-Jordan inverses against the oracle's LU solves),
residual 1e-13, V-cycle 1e-9; whole solves as for the quadrilaterals (check_solve: iteration count, the
1e-8 history target on the entries the method determines, 1e-10 solution target against the oracle run
with the same orthogonalisation); discretisation errors to 1e-10.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import bdm, fem, solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# k = 1 (19-DoF interior patches), 2 (42), 3 (74), 4 (115): coarsest 2 x 2, two or three levels;
# k = 5 on 1 x 1 -> 2 x 2 (patches of up to 141 DoFs, the fifth size class of the patch kernels)
CASES = [(2, 2, 1), (2, 3, 1), (2, 2, 2), (2, 3, 2), (2, 2, 3), (2, 2, 4), (1, 2, 5)]


@pytest.fixture(scope="module")
def vk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_14222_gb300 import build
    build.build()
    import paper_2409_14222_gb300 as vk
    return vk


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def pair(vk, case, nu=1.0):
    Nc, L, k = case
    return solver.Hierarchy(Nc, L, k, nu=nu, cell="bdm"), vk.Hierarchy(Nc, L, k, nu=nu, cell=vk.vk.VK_CELL_BDM)


@pytest.mark.parametrize("case", CASES)
def test_bdm_rows_match_the_oracle(vk, case):
    from test_gpu_quad import check_solve
    H, G = pair(vk, case)
    rng = np.random.default_rng(303)
    for l in range(1, case[1]):
        lev = H.levels[l]
        assert abs(G.lam(l) - lev.lam) <= 1e-10 * lev.lam
        r = rng.standard_normal(lev.space.ndof)
        z = torch.empty_like(dev(r))
        G.vanka(l, dev(r), z)
        got = host(z)
        assert rel(got, solver.vanka_apply(lev, r)) <= 1e-10
        assert np.array_equal(got[lev.mask], r[lev.mask])
        x = rng.standard_normal(lev.space.ndof)
        rr = torch.empty_like(z)
        G.residual(l, dev(r), dev(x), rr)
        assert rel(host(rr), r - lev.A @ x) <= 1e-13
    b = si.rhs_normal(H.finest.space.ndof, 0)
    xv = torch.empty_like(dev(b))
    G.vcycle(dev(b), xv)
    assert rel(host(xv), H.vcycle(b)) <= 1e-9
    x = torch.zeros_like(dev(b))
    out = G.solve(dev(b), x, rtol=1e-10)
    print(f"bdm {case}:", end=" ")
    check_solve(out, host(x), solver.solve(H, b, 1e-10, 100), solver.solve(H, b, 1e-10, 100, orth="cgs2"))


@pytest.mark.parametrize("case", [(5, 2, 2), (5, 2, 3), (5, 3, 1)])
def test_bdm_paper_coarse_grid_solves(vk, case):
    # the paper's 5 x 5 coarsest grid (Sec. 4): BDM2 and BDM3 on 10 x 10, BDM1 on 20 x 20, rtol 1e-10
    from test_gpu_quad import check_solve
    H, G = pair(vk, case)
    b = si.rhs_normal(H.finest.space.ndof, 2)
    x = torch.zeros_like(dev(b))
    out = G.solve(dev(b), x, rtol=1e-10)
    print(f"bdm {case}:", end=" ")
    check_solve(out, host(x), solver.solve(H, b, 1e-10, 100), solver.solve(H, b, 1e-10, 100, orth="cgs2"))
    # the iteration counts of Sec. 4.3 stay small and level-independent (h- and p-robust)
    assert out["iterations"] <= 40


@pytest.mark.parametrize("N,k", [(4, 1), (4, 2), (2, 3), (2, 4)])
def test_bdm_error_norms_equal_the_oracle(vk, N, k):
    # vk_errors (broken H^1 and L^2 velocity errors of the Piola-mapped field, L^2 pressure error after
    # removing the mean, on the device) against the oracle's bdm.errors on the same vectors
    s = bdm.BDMSpace(N, k)
    G = vk.Hierarchy(N, 1, k, cell=vk.vk.VK_CELL_BDM)
    K = bdm.assemble_full(s)
    mask = s.dirichlet_mask()
    A = fem.apply_dirichlet(K, mask)
    b = bdm.load_vector(s)
    b[mask] = 0.0
    assert np.linalg.norm(G.manufactured_rhs() - b) <= 1e-13 * np.linalg.norm(b)
    xd = solver.project(s, solver.direct_solve(A, s.nullspace(), solver.project(s, b)))
    rng = np.random.default_rng(82)
    for x in (xd, xd + 1e-3 * rng.standard_normal(len(xd))):
        got = G.errors(dev(x))
        want = bdm.errors(s, x)
        for g, w in zip(got, want):
            assert abs(g - w) <= 1e-10 * w, (got, want)


def test_bdm_manufactured_solve_converges_at_order_k(vk):
    # BDM2 on 5 x 5 -> 10 x 10 -> 20 x 20: solving the manufactured problem to 1e-12 through the whole
    # GPU path (setup, FGMRES, errors) gives errors falling like h^k in the velocity's broken H^1 norm and
    # the pressure (Sec. 4.4)
    errs = []
    for L in (2, 3):
        G = vk.Hierarchy(5, L, 2, cell=vk.vk.VK_CELL_BDM)
        b = dev(G.manufactured_rhs())
        x = torch.zeros_like(b)
        out = G.solve(b, x, rtol=1e-12)
        assert out["converged"]
        errs.append(G.errors(x))
    h1, pl2 = np.log2(errs[0][0] / errs[1][0]), np.log2(errs[0][2] / errs[1][2])
    print(f"BDM2 rates: H1 {h1:.2f}, pressure {pl2:.2f}")
    assert h1 > 1.8 and pl2 > 1.8
