"""GPU parity for Taylor-Hood (Q_k, Q_{k-1}) on quadrilaterals (Case 2 of Sec. 3, results of Sec. 4.2):
the same C ABI and kernels as the triangles with the quadrilateral element, transfers and composite
vertex / edge / cell patches (Sec. 3.1), against the oracle's quadrilateral discretization.

Tolerances as for the triangles: one Vanka application 1e-10 (stored Gauss-Jordan inverses against LU
solves), V-cycle 1e-9; whole solves as described in check_solve (the 1e-8 history and 1e-10 solution
targets where the method determines them).
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Q2 (vertex patches, 51 DoFs inside), Q3 (vertex / edge / cell, 99 / 57 / 33), Q4 (163 / 92 / 54: the
# vertex patches exceed 128 DoFs, the fifth size class of the patch kernels)
# (a 1 x 1 coarsest grid is not used: for k = 3 it has 8 free velocities against 9 pressures, so the
# coarse saddle-point system is singular beyond the constant pressure)
CASES = [(2, 2, 2), (2, 3, 2), (2, 2, 3), (2, 3, 3), (2, 2, 4)]


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


@pytest.mark.parametrize("case", CASES)
def test_quad_rows_match_the_oracle(vk, case):
    Nc, L, k = case
    H = solver.Hierarchy(Nc, L, k, cell="quad")
    G = vk.Hierarchy(Nc, L, k, cell=vk.vk.VK_CELL_QUAD)
    rng = np.random.default_rng(101)
    for l in range(1, L):
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
    check_solve(out, host(x), solver.solve(H, b, 1e-10, 100), solver.solve(H, b, 1e-10, 100, orth="cgs2"))


def check_solve(out, xg, ref, ref2):
    """A GPU solve against the oracle's MGS (ref) and CGS2 (ref2) runs.  The Q3 and Q4 Vanka cycles converge
    slowly (40 to 60 iterations) and some of their Givens estimates are ill-conditioned: the oracle's own
    two orthogonalisations differ there by up to 1e-6 of the initial residual, and on one full-size case
    they cross the tolerance one iteration apart.  So: the iteration count equals one of the oracle's; the
    history meets the 1e-8 target on the entries the method determines (where the oracle's two runs
    agree) when both runs take the same count; the iterate is within 1e-10 of the oracle run with the
    same orthogonalisation and count, else within twice the oracle's own MGS/CGS2 spread."""
    from test_gpu_schedule import check_history
    spread = rel(ref2.x, ref.x)
    print(f"{out['iterations']} iterations (oracle MGS {ref.iters}, CGS2 {ref2.iters}); x rel. dev "
          f"{rel(xg, ref2.x):.2e} from the oracle's CGS2 run, {rel(xg, ref.x):.2e} from its MGS run "
          f"(MGS/CGS2 spread {spread:.2e})")
    assert out["converged"] and out["iterations"] in (ref.iters, ref2.iters)
    if ref.iters == ref2.iters:
        check_history(out["history"], np.array(ref.hist), np.array(ref2.hist))
    if out["iterations"] == ref2.iters and rel(xg, ref2.x) <= 1e-10:
        return
    same = [r for r in (ref, ref2) if r.iters == out["iterations"]]
    assert min(rel(xg, r.x) for r in same) <= max(1e-10, 2 * spread)


@pytest.mark.parametrize("case", [(16, 3, 2), (8, 3, 3)])
def test_quad_full_size_solves(vk, case):
    # Q2/Q1 on 16 -> 64 (37,507 DoFs) and Q3/Q2 on 8 -> 32 (23,043 DoFs), rtol 1e-8, FP64
    Nc, L, k = case
    H = solver.Hierarchy(Nc, L, k, cell="quad")
    G = vk.Hierarchy(Nc, L, k, cell=vk.vk.VK_CELL_QUAD)
    b = si.rhs_normal(H.finest.space.ndof, 1)
    x = torch.zeros_like(dev(b))
    out = G.solve(dev(b), x, rtol=1e-8)
    print(f"quad {case}:", end=" ")
    check_solve(out, host(x), solver.solve(H, b, 1e-8, 100), solver.solve(H, b, 1e-8, 100, orth="cgs2"))
