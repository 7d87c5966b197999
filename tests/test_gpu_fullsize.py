"""Parity at the largest single-GPU size: Taylor-Hood P2/P1, 32x32 -> 512x512 (5 levels), 2,364,419
DoFs, in the launch configuration the benchmark times (whole-solve CUDA graph, autotuned patch-apply
shapes, SELL with one thread per row at this size, persistent apply grids).

The oracle's solve at this size takes tens of minutes, so its result is stored once by
tests/golden/make_golden.py (oracle only): eigenvalue estimates, iteration count, residual history and
every 37th solution entry with the norm of the whole solution.  The GPU solve must give the same
iteration count, a residual history within 1e-8 (normalised, and per entry above the FP64 floor),
eigenvalue estimates within 1e-10 and, on the stored entries, a solution within 1e-10 relative.

The mixed-precision 16-right-hand-side solve (BF16 patch inverses on the tensor cores, FP32 V-cycle,
FP64 FGMRES per column) reaches rtol on every column; its first column's error against the FP64
oracle solution is stated and bounded.
"""
import numpy as np
import pytest

import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEY = (32, 5, 2)


@pytest.fixture(scope="module")
def vk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_14222_gb300 import build
    build.build()
    import paper_2409_14222_gb300 as vk
    return vk


@pytest.fixture(scope="module")
def ref():
    from golden.make_golden import load
    r = load("p2_32to512")
    assert r is not None, "tests/golden/oracle_p2_32to512.npz is missing"
    return r


def sampled_rel(x, ref):
    idx, want = ref["x_idx"], ref["x_val"]
    return np.linalg.norm(x[idx] - want) / np.linalg.norm(want)


def test_fp64_solve_512_matches_the_oracle(vk, ref):
    G = vk.Hierarchy(*KEY)
    n = G.ndof()
    assert n == int(ref["ndof"]) == 2364419
    for l in range(1, KEY[1]):
        assert abs(G.lam(l) - ref["lambdas"][l]) <= 1e-10 * ref["lambdas"][l], l
    b = si.rhs_normal(n, int(ref["seed"]))
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = G.solve(torch.from_numpy(b).cuda(), x, rtol=float(ref["rtol"]))
    xh = x.cpu().numpy()
    want = ref["hist"]
    assert out["converged"] and out["iterations"] == int(ref["iterations"])
    hist = out["history"]
    norm_dev = np.max(np.abs(hist - want)) / want[0]
    big = want >= 1e-6 * want[0]
    ent_dev = np.max(np.abs(hist - want)[big] / want[big])
    err = sampled_rel(xh, ref)
    nrm = abs(np.linalg.norm(xh) - float(ref["x_norm"])) / float(ref["x_norm"])
    print(f"512x512 P2 FP64: {out['iterations']} iterations; history dev {norm_dev:.2e} normalised, "
          f"{ent_dev:.2e} per entry; x rel. dev {err:.2e} on {len(ref['x_idx'])} entries, norm {nrm:.2e}")
    assert norm_dev <= 1e-8 and ent_dev <= 1e-8
    assert err <= 1e-10 and nrm <= 1e-10
    assert abs(out["true_res"] - float(ref["true_res"])) <= 1e-11 * want[0]


def test_batched_bf16_solve_512_against_the_fp64_oracle(vk, ref):
    G = vk.Hierarchy(*KEY, options=vk.default_options(batch_prec=vk.VK_BATCH_BF16))
    n = G.ndof()
    B = torch.from_numpy(si.rhs_batch(n, range(16)).T.copy()).cuda()
    X = torch.zeros_like(B)
    outs = G.solve_batch(B, X, rtol=1e-8, maxit=60)
    for o in outs:
        assert o["converged"] and o["true_res"] <= 1.5e-8 * o["res0"]
    x0 = X[0].cpu().numpy()
    err = sampled_rel(x0, ref)
    print(f"512x512 16-RHS BF16 batch: iterations {[o['iterations'] for o in outs]}; column 0 rel. error vs "
          f"FP64 oracle {err:.2e}")
    assert err <= 1e-6
