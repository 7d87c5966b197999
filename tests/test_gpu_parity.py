"""GPU parity: every hot-path row through the C ABI against the oracle, element by element.

Tolerances (relative, norm-wise unless stated), derived from the arithmetic:
  * SpMV residual, restriction, prolongation: same products, FMA vs separate rounding -> 1e-13;
  * one Vanka application: patch solves by a stored Gauss-Jordan inverse (GPU) vs LU solves (oracle):
    the difference is bounded by cond(A_i) * eps per patch; patch condition numbers here are < 1e4 -> 1e-10;
  * coarse solve: stored bordered inverse vs LU, cond(coarse) ~ 1e5 -> 1e-9;
  * full FGMRES solve (the stated target): equal iteration counts, per-iteration residual estimates
    within 1e-8, solution within 1e-10.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import fem, solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


# (N_coarse, nlevels, k): config 1 (4 -> 8, P2), a 3-level P2 case, P3 and P4 composite patches
SMALL = [(4, 2, 2), (2, 3, 2), (2, 2, 3), (2, 2, 4), (2, 3, 3)]

_cache = {}


def pair(vk, case, inject=True, sweeps=1, prec=None):
    key = (case, inject, sweeps, prec)
    if key not in _cache:
        Nc, L, k = case
        okey = (case, sweeps)
        if okey not in _cache:
            _cache[okey] = solver.Hierarchy(Nc, L, k, sweeps=sweeps)
        H = _cache[okey]
        opts = vk.default_options(sweeps=sweeps)
        if prec is not None:
            opts.factor_prec = prec
        lams = [0.0] + [H.levels[l].lam for l in range(1, L)] if inject else None
        G = vk.Hierarchy(Nc, L, k, options=opts, lambdas=lams)
        _cache[key] = (H, G)
    return _cache[key]


@pytest.mark.parametrize("case", SMALL)
def test_lambda_estimate(vk, case):
    H, G = pair(vk, case, inject=False)
    for l in range(1, case[1]):
        assert abs(G.lam(l) - H.levels[l].lam) <= 1e-10 * H.levels[l].lam


@pytest.mark.parametrize("case", SMALL)
def test_residual(vk, case):
    H, G = pair(vk, case)
    rng = np.random.default_rng(11)
    for l, lev in enumerate(H.levels):
        n = lev.space.ndof
        b, x = rng.standard_normal(n), rng.standard_normal(n)
        r = torch.empty(n, dtype=torch.float64, device="cuda")
        G.residual(l, dev(b), dev(x), r)
        assert rel(host(r), b - lev.A @ x) <= 1e-13


@pytest.mark.parametrize("case", SMALL)
def test_vanka_application(vk, case):
    H, G = pair(vk, case)
    rng = np.random.default_rng(12)
    for l in range(1, case[1]):
        lev = H.levels[l]
        r = rng.standard_normal(lev.space.ndof)
        z = torch.empty_like(dev(r))
        G.vanka(l, dev(r), z)
        want = solver.vanka_apply(lev, r)
        got = host(z)
        print(f"vanka {case} level {l}: rel. dev {rel(got, want):.2e}")
        assert rel(got, want) <= 1e-10
        # Dirichlet DoFs are the identity, bit for bit
        assert np.array_equal(got[lev.mask], r[lev.mask])


@pytest.mark.parametrize("case", SMALL)
@pytest.mark.parametrize("zero_init", [True, False])
def test_chebyshev_smoothing(vk, case, zero_init):
    for sweeps in (1, 3):
        H, G = pair(vk, case, sweeps=sweeps)
        rng = np.random.default_rng(13)
        for l in range(1, case[1]):
            lev = H.levels[l]
            b, x0 = rng.standard_normal(lev.space.ndof), rng.standard_normal(lev.space.ndof)
            x = dev(x0)
            G.smooth(l, dev(b), x, zero_init)
            want = solver.chebyshev(lambda v: lev.A @ v, lambda rr: solver.vanka_apply(lev, rr), b,
                                    None if zero_init else x0, lev.lam, sweeps)
            assert rel(host(x), want) <= 1e-10


@pytest.mark.parametrize("case", SMALL)
def test_transfers(vk, case):
    H, G = pair(vk, case)
    rng = np.random.default_rng(14)
    for l in range(1, case[1]):
        f, c = H.levels[l], H.levels[l - 1]
        r = rng.standard_normal(f.space.ndof)
        rc = torch.empty(c.space.ndof, dtype=torch.float64, device="cuda")
        G.restrict(l, dev(r), rc)
        want = f.R @ r
        want[c.mask] = 0.0
        got = host(rc)
        assert rel(got, want) <= 1e-13
        assert np.all(got[c.mask] == 0.0)
        e, x0 = rng.standard_normal(c.space.ndof), rng.standard_normal(f.space.ndof)
        x = dev(x0)
        G.prolong(l, dev(e), x)
        assert rel(host(x), x0 + f.P @ e) <= 1e-13


@pytest.mark.parametrize("case", SMALL)
def test_coarse_solve(vk, case):
    H, G = pair(vk, case)
    c = H.levels[0]
    b = solver.project(c.space, np.random.default_rng(15).standard_normal(c.space.ndof))
    x = torch.empty_like(dev(b))
    G.coarse_solve(dev(b), x)
    print(f"coarse {case}: rel. dev {rel(host(x), H.coarse_solve(b)):.2e}")
    assert rel(host(x), H.coarse_solve(b)) <= 1e-9


@pytest.mark.parametrize("case", SMALL)
def test_vcycle(vk, case):
    for sweeps in (1, 2):
        H, G = pair(vk, case, sweeps=sweeps)
        b = np.random.default_rng(16).standard_normal(H.finest.space.ndof)
        x = torch.empty_like(dev(b))
        G.vcycle(dev(b), x)
        assert rel(host(x), H.vcycle(b)) <= 1e-9


def check_history(hist, want):
    """Residual histories: normalised by ||b|| (the relative-residual curve) they agree to 1e-8; entry by
    entry they agree to 1e-8 relative wherever the residual is still >= 1e-6 ||b||.  Below that, FP64
    Arnoldi rounding (about eps * ||b|| absolute) is the floor, so per-entry relative agreement there is
    limited by floating point, not by the method; the normalised check still covers those entries."""
    assert len(hist) == len(want)
    norm_dev = np.max(np.abs(hist - want)) / want[0]
    big = want >= 1e-6 * want[0]
    rel_dev = np.max(np.abs(hist - want)[big] / want[big])
    print(f"history: normalised max dev {norm_dev:.2e}, per-entry rel. dev (>=1e-6) {rel_dev:.2e}")
    assert norm_dev <= 1e-8, norm_dev
    assert rel_dev <= 1e-8, rel_dev


def _solve_parity(vk, H, G, b, rtol, maxit=100):
    x = torch.zeros_like(dev(b))
    out = G.solve(dev(b), x, rtol=rtol, maxit=maxit)
    ref = solver.solve(H, b, rtol, maxit)
    assert out["iterations"] == ref.iters, (out["iterations"], ref.iters)
    assert out["converged"] == ref.converged
    hist = out["history"]
    want = np.array(ref.hist)
    check_history(hist, want)
    print(f"solve: {out['iterations']} iterations, x rel. dev {rel(host(x), ref.x):.2e}")
    assert rel(host(x), ref.x) <= 1e-10
    # recomputing b - A x in FP64 carries about eps * ||b|| of rounding: compare with that floor
    assert abs(out["true_res"] - ref.true_res) <= 1e-11 * ref.hist[0]
    return out, ref


@pytest.mark.parametrize("case", SMALL)
def test_fgmres_solve_small(vk, case):
    # lambda estimated independently on both sides (no injection)
    H, G = pair(vk, case, inject=False)
    b = si.rhs_normal(H.finest.space.ndof, 0)
    out, ref = _solve_parity(vk, H, G, b, 1e-10)
    assert out["converged"] and out["true_res"] <= 1.01e-10 * out["res0"] * 10


def test_fgmres_solve_config1_sweeps(vk):
    for sweeps in (2, 3):
        H, G = pair(vk, (4, 2, 2), inject=False, sweeps=sweeps)
        _solve_parity(vk, H, G, si.rhs_normal(H.finest.space.ndof, 1), 1e-10)


@pytest.fixture(scope="module")
def config2(vk):
    # 16 -> 128, P2/P1, 4 levels: 148,739 DoFs on the finest level
    H = solver.Hierarchy(16, 4, 2)
    G = vk.Hierarchy(16, 4, 2)
    return H, G


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_fgmres_solve_config2_full_size(vk, config2, seed):
    H, G = config2
    for l in range(1, 4):
        assert abs(G.lam(l) - H.levels[l].lam) <= 1e-10 * H.levels[l].lam
    b = si.rhs_normal(H.finest.space.ndof, seed)
    out, ref = _solve_parity(vk, H, G, b, 1e-8)
    assert out["converged"]


def test_edge_cases(vk):
    H, G = pair(vk, (4, 2, 2), inject=False)
    n = H.finest.space.ndof
    # zero right-hand side: zero solution, no iteration
    x = torch.full((n,), 3.0, dtype=torch.float64, device="cuda")
    out = G.solve(torch.zeros(n, dtype=torch.float64, device="cuda"), x)
    assert out["iterations"] == 0 and out["converged"] and float(x.abs().max()) == 0.0
    # a right-hand side in the nullspace (constant pressure) projects to zero
    b = np.zeros(n)
    b[H.finest.space.n_u:] = 2.5
    out = G.solve(dev(b), x)
    assert out["iterations"] == 0 and float(x.abs().max()) == 0.0
    # maxit reached: status NOT_CONVERGED, iterate and history still match the oracle
    b = si.rhs_normal(n, 3)
    out = G.solve(dev(b), x, rtol=1e-14, maxit=3)
    ref = solver.solve(H, b, 1e-14, 3)
    assert out["status"] == vk.vk.VK_ERR_NOT_CONVERGED and out["iterations"] == 3 and not out["converged"]
    assert rel(host(x), ref.x) <= 1e-10
    check_history(out["history"], np.array(ref.hist))
    # non-finite right-hand side is reported
    bad = b.copy()
    bad[5] = np.nan
    with pytest.raises(vk.VkError) as e:
        G.solve(dev(bad), x)
    assert e.value.code == vk.vk.VK_ERR_NONFINITE
    # invalid arguments
    with pytest.raises(vk.VkError):
        G.solve(dev(b), x, maxit=0)
    with pytest.raises(vk.VkError):
        G.vanka(0, dev(b), x)


@pytest.mark.parametrize("case", [(4, 2, 2), (2, 3, 3)])
def test_graph_and_host_loop_paths_agree(vk, case):
    # the whole-solve CUDA graph (device-side loop) and the host-driven loop run the same kernels
    H, G = pair(vk, case, inject=False)
    Nc, L, k = case
    Gh = vk.Hierarchy(Nc, L, k, options=vk.default_options(use_graph=0))
    b = si.rhs_normal(H.finest.space.ndof, 21)
    xg, xh = torch.zeros_like(dev(b)), torch.zeros_like(dev(b))
    og = G.solve(dev(b), xg, rtol=1e-10)
    oh = Gh.solve(dev(b), xh, rtol=1e-10)
    assert og["iterations"] == oh["iterations"]
    assert np.allclose(og["history"], oh["history"], rtol=1e-14, atol=0)
    assert rel(host(xg), host(xh)) <= 1e-14
    # launches are counted the same way on both paths
    G.stats_reset()
    Gh.stats_reset()
    G.solve(dev(b), xg, rtol=1e-10)
    Gh.solve(dev(b), xh, rtol=1e-10)
    sg, sh = G.stats(), Gh.stats()
    assert sg["vcycles"] == sh["vcycles"] == og["iterations"]
    assert sg["launches"] > 0 and sh["launches"] > 0


def test_graph_with_and_without_programmatic_launch_agree(vk):
    # programmatic dependent launch only lets a kernel be scheduled early; each kernel waits for its
    # predecessor's completion before touching memory, so the solves are bit-identical
    H = solver.Hierarchy(2, 3, 2)
    G = vk.Hierarchy(2, 3, 2, options=vk.default_options(graph_pdl=1))
    G0 = vk.Hierarchy(2, 3, 2, options=vk.default_options(graph_pdl=0))
    b = si.rhs_normal(H.finest.space.ndof, 33)
    x1, x0 = torch.zeros_like(dev(b)), torch.zeros_like(dev(b))
    o1 = G.solve(dev(b), x1, rtol=1e-10)
    o0 = G0.solve(dev(b), x0, rtol=1e-10)
    assert G.stats()["graph_pdl"] == 1 and G0.stats()["graph_pdl"] == 0
    assert o1["iterations"] == o0["iterations"]
    assert np.array_equal(o1["history"], o0["history"])
    assert torch.equal(x1, x0)


def test_host_buffer_solve_equals_device_solve(vk):
    H, G = pair(vk, (2, 3, 2), inject=False)
    n = H.finest.space.ndof
    b = si.rhs_normal(n, 7)
    xd = torch.zeros_like(dev(b))
    out_d = G.solve(dev(b), xd, rtol=1e-10)
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    out_h = G.solve_host(bh.numpy(), xh.numpy(), rtol=1e-10)
    assert out_h["iterations"] == out_d["iterations"]
    assert np.array_equal(xh.numpy(), host(xd))


@pytest.mark.parametrize("case", [(4, 2, 2), (2, 3, 3), (2, 2, 4)])
def test_emulated_fp64_inverses_parity(vk, case):
    # FP32-pair inverses applied in FP32-pair arithmetic: ~48-bit products, so one Vanka application
    # agrees with the oracle's LU solves to ~1e-13 and whole solves keep the FP64 parity targets
    H, G = pair(vk, case, inject=False, prec=vk.VK_PREC_F64E)
    rng = np.random.default_rng(31)
    for l in range(1, case[1]):
        lev = H.levels[l]
        r = rng.standard_normal(lev.space.ndof)
        z = torch.empty_like(dev(r))
        G.vanka(l, dev(r), z)
        err = rel(host(z), solver.vanka_apply(lev, r))
        print(f"f64e vanka {case} level {l}: rel. dev {err:.2e}")
        assert err <= 1e-12
    _solve_parity(vk, H, G, si.rhs_normal(H.finest.space.ndof, 0), 1e-10)


def test_emulated_fp64_config2_full_size(vk, config2):
    H, _ = config2
    G = vk.Hierarchy(16, 4, 2, options=vk.default_options(factor_prec=vk.VK_PREC_F64E))
    out, ref = _solve_parity(vk, H, G, si.rhs_normal(H.finest.space.ndof, 0), 1e-8)
    assert out["converged"]


def test_fp32_factors_reach_tolerance(vk):
    H, G64 = pair(vk, (2, 3, 2), inject=False)
    _, G32 = pair(vk, (2, 3, 2), inject=False, prec=vk.VK_PREC_F32)
    b = si.rhs_normal(H.finest.space.ndof, 0)
    x32 = torch.zeros_like(dev(b))
    out32 = G32.solve(dev(b), x32, rtol=1e-8)
    ref = solver.solve(H, b, 1e-8, 100)
    assert out32["converged"] and out32["true_res"] <= 1e-8 * out32["res0"] * 1.5
    assert out32["iterations"] <= ref.iters + 3
    # solution error against the FP64 oracle at the same tolerance (reported; loose sanity bound)
    err = rel(host(x32), ref.x)
    print(f"FP32 inverses: {out32['iterations']} iterations (FP64 oracle {ref.iters}), rel. error {err:.2e}")
    assert err <= 1e-3


@pytest.fixture(scope="module")
def weighted(vk):
    # Algorithm 1 with the multiplicity weights (each DoF's summed correction divided by the number of
    # patches containing it), lambda estimated independently on both sides
    out = {}
    for case in [(4, 2, 2), (2, 3, 3), (2, 2, 4)]:
        Nc, L, k = case
        H = solver.Hierarchy(Nc, L, k, weights="multiplicity")
        G = vk.Hierarchy(Nc, L, k, options=vk.default_options(weights=vk.VK_WEIGHTS_MULTIPLICITY))
        out[case] = (H, G)
    return out


@pytest.mark.parametrize("case", [(4, 2, 2), (2, 3, 3), (2, 2, 4)])
def test_multiplicity_weights_parity(vk, weighted, case):
    H, G = weighted[case]
    for l in range(1, case[1]):
        assert abs(G.lam(l) - H.levels[l].lam) <= 1e-10 * H.levels[l].lam
    rng = np.random.default_rng(51)
    for l in range(1, case[1]):
        lev = H.levels[l]
        r = rng.standard_normal(lev.space.ndof)
        z = torch.empty_like(dev(r))
        G.vanka(l, dev(r), z)
        got = host(z)
        assert rel(got, solver.vanka_apply(lev, r)) <= 1e-10
        assert np.array_equal(got[lev.mask], r[lev.mask])
    b = rng.standard_normal(H.finest.space.ndof)
    x = torch.empty_like(dev(b))
    G.vcycle(dev(b), x)
    assert rel(host(x), H.vcycle(b)) <= 1e-9
    if case[2] == 2:
        _solve_parity(vk, H, G, si.rhs_normal(H.finest.space.ndof, 0), 1e-10)
        return
    # P3 / P4: some Givens estimates are ill-conditioned; the 1e-8 history target applies to the entries
    # the method determines (where the oracle's two orthogonalisations agree), as in the higher-order tests
    from test_gpu_schedule import check_history as check_determined
    bb = si.rhs_normal(H.finest.space.ndof, 0)
    xs = torch.zeros_like(dev(bb))
    out = G.solve(dev(bb), xs, rtol=1e-10)
    ref = solver.solve(H, bb, 1e-10, 100)
    ref2 = solver.solve(H, bb, 1e-10, 100, orth="cgs2")
    assert out["iterations"] == ref.iters == ref2.iters
    check_determined(out["history"], np.array(ref.hist), np.array(ref2.hist))
    assert rel(host(xs), ref2.x) <= 1e-10 and rel(host(xs), ref.x) <= max(1e-10, 2 * rel(ref2.x, ref.x))


def test_device_footprint_matches_prediction(vk):
    H, G = pair(vk, (2, 3, 3), inject=False)
    assert G.device_bytes() == vk.footprint(2, 3, 3)
    assert G.alloc.bytes() >= G.device_bytes()
