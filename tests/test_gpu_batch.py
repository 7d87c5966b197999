"""vk_solve_batch: 16 right-hand sides at once, FP32 V-cycle with BF16 / FP16 patch inverses on the
tensor cores, FP64 FGMRES per column.

Accuracy target (mixed precision): every column's true residual reaches rtol (FP64 outer iteration),
and the solution error against the FP64 oracle is reported; a column's result does not depend on the
other columns of the batch (bit for bit).  Both tensor-core instruction families are covered: tcgen05
(TMEM accumulators, TMA loads; the default) and warp-level mma.sync, which compute the same rounded
products and must agree to the FP32 accumulation order."""
import time

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


_h = {}


def batch_hierarchy(vk, key, prec, engine=0):
    if (key, prec, engine) not in _h:
        _h[(key, prec, engine)] = vk.Hierarchy(*key, options=vk.default_options(batch_prec=prec, batch_engine=engine))
    return _h[(key, prec, engine)]


ENGINES = {"tcgen05": 0, "mma_sync": 1}


@pytest.mark.parametrize("key", [(4, 2, 2), (2, 3, 3), (2, 2, 4), (4, 2, 4)])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
def test_batch_columns_converge_and_match_oracle(vk, key, prec, engine):
    p = vk.VK_BATCH_BF16 if prec == "bf16" else vk.VK_BATCH_FP16
    G = batch_hierarchy(vk, key, p, ENGINES[engine])
    n = G.ndof()
    B = si.rhs_batch(n, range(16)).T.copy()             # (16, n): row r = right-hand side r
    X = torch.zeros(16, n, dtype=torch.float64, device="cuda")
    out = G.solve_batch(torch.from_numpy(B).cuda(), X, rtol=1e-8, maxit=60)
    H = solver.Hierarchy(*key)
    Xh = X.cpu().numpy()
    errs = []
    for r in (0, 7, 15):
        assert out[r]["converged"], out[r]
        assert out[r]["true_res"] <= 1.5e-8 * out[r]["res0"]
        ref = solver.solve(H, B[r], 1e-10, 100)
        # both solve the projected system: the difference is bounded by the residuals' reach
        errs.append(np.linalg.norm(Xh[r] - ref.x) / np.linalg.norm(ref.x))
    print(f"batch {engine} {prec} {key}: iterations {[o['iterations'] for o in out]}, "
          f"error vs FP64 oracle {max(errs):.2e}")
    assert max(errs) <= 1e-5


@pytest.mark.parametrize("key", [(8, 3, 2), (4, 2, 3), (4, 2, 4)])
def test_tcgen05_and_mma_sync_engines_agree(vk, key):
    # same 16-bit operands, FP32 accumulation in a different order: V-cycles agree to ~1e-6, so the
    # FGMRES iteration counts agree within one and the solutions to the reach of rtol
    n = batch_hierarchy(vk, key, vk.VK_BATCH_BF16, 0).ndof()
    B = torch.from_numpy(si.rhs_batch(n, range(200, 216)).T.copy()).cuda()
    out, X = {}, {}
    for name, e in ENGINES.items():
        X[name] = torch.zeros(16, n, dtype=torch.float64, device="cuda")
        out[name] = batch_hierarchy(vk, key, vk.VK_BATCH_BF16, e).solve_batch(B, X[name], rtol=1e-8)
    for r in range(16):
        a, b = out["tcgen05"][r], out["mma_sync"][r]
        assert a["converged"] and b["converged"]
        assert abs(a["iterations"] - b["iterations"]) <= 1
        d = float(torch.linalg.vector_norm(X["tcgen05"][r] - X["mma_sync"][r]) / torch.linalg.vector_norm(X["mma_sync"][r]))
        assert d <= 1e-6, (r, d)


@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
def test_batch_column_is_independent_of_the_other_columns(vk, engine):
    G = batch_hierarchy(vk, (2, 3, 3), vk.VK_BATCH_BF16, ENGINES[engine])
    n = G.ndof()
    B = si.rhs_batch(n, range(100, 116)).T.copy()
    X = torch.zeros(16, n, dtype=torch.float64, device="cuda")
    full = G.solve_batch(torch.from_numpy(B).cuda(), X, rtol=1e-8)
    for r in (3, 12):
        x1 = torch.zeros(1, n, dtype=torch.float64, device="cuda")
        one = G.solve_batch(torch.from_numpy(B[r:r + 1].copy()).cuda(), x1, rtol=1e-8)
        assert one[0]["iterations"] == full[r]["iterations"]
        assert torch.equal(x1[0], X[r])


def test_batch_edge_cases(vk):
    G = batch_hierarchy(vk, (4, 2, 2), vk.VK_BATCH_BF16)
    n = G.ndof()
    B = np.zeros((3, n))
    B[1] = si.rhs_normal(n, 5)
    X = torch.full((3, n), 7.0, dtype=torch.float64, device="cuda")
    out = G.solve_batch(torch.from_numpy(B).cuda(), X, rtol=1e-8)
    assert out[0]["iterations"] == 0 and out[0]["converged"] and float(X[0].abs().max()) == 0.0
    assert out[1]["converged"]
    Hn = vk.Hierarchy(4, 2, 2)                           # built without batch support
    with pytest.raises(vk.VkError):
        Hn.solve_batch(torch.from_numpy(B).cuda(), X)
    with pytest.raises(vk.VkError):
        G.solve_batch(torch.zeros(17, n, dtype=torch.float64, device="cuda"),
                      torch.zeros(17, n, dtype=torch.float64, device="cuda"))


def test_batch_full_size_512_p2_residuals_on_oracle_matrix(vk):
    # the cfg4 workload: 32 -> 512 (5 levels), P2/P1, 16 right-hand sides; each returned column is
    # checked against the oracle's own assembled 512x512 matrix (a property that holds at any size)
    G = vk.Hierarchy(32, 5, 2, options=vk.default_options(batch_prec=vk.VK_BATCH_BF16))
    n = G.ndof()
    assert n == 2364419
    B = si.rhs_batch(n, range(16)).T.copy()
    X = torch.zeros(16, n, dtype=torch.float64, device="cuda")
    out = G.solve_batch(torch.from_numpy(B).cuda(), X, rtol=1e-8, maxit=60)
    assert all(o["converged"] for o in out)
    s = fem.Space(512, 2)
    A = fem.apply_dirichlet(fem.assemble_full(s), s.dirichlet_mask())
    Xh = X.cpu().numpy()
    for r in (0, 9):
        b = solver.project(s, B[r])
        res = np.linalg.norm(b - A @ Xh[r]) / np.linalg.norm(b)
        print(f"512^2 column {r}: {out[r]['iterations']} iterations, oracle-matrix residual {res:.2e}")
        assert res <= 1.5e-8
        assert abs(Xh[r][s.n_u:].sum()) <= 1e-8 * np.abs(Xh[r]).sum()


def test_tcgen05_bounded_wait_expires_and_recovers(vk):
    # failure detection without a fault: the test hook makes the first finest sweep announce one bulk
    # copy without issuing it; the producer's bounded wait expires, every role of that CTA stops, the
    # kernel drains and frees its tensor memory, and the call reports VK_ERR_TIMEOUT.  The context and
    # the hierarchy stay usable: the next call runs normally and converges.
    G = vk.Hierarchy(4, 2, 2, options=vk.default_options(batch_prec=vk.VK_BATCH_BF16,
                                                         batch_engine=vk.VK_ENGINE_TCGEN05, test_expire_wait=1))
    n = G.ndof()
    B = torch.from_numpy(si.rhs_batch(n, range(16)).T.copy()).cuda()
    X = torch.zeros(16, n, dtype=torch.float64, device="cuda")
    t0 = time.time()
    with pytest.raises(vk.VkError) as e:
        G.solve_batch(B, X, rtol=1e-8)
    assert e.value.code == vk.vk.VK_ERR_TIMEOUT
    assert time.time() - t0 < 60
    out = G.solve_batch(B, X, rtol=1e-8)
    assert all(o["converged"] for o in out)
    ref = batch_hierarchy(vk, (4, 2, 2), vk.VK_BATCH_BF16, ENGINES["tcgen05"])
    X2 = torch.zeros_like(X)
    ref.solve_batch(B, X2, rtol=1e-8)
    assert torch.equal(X, X2)
