"""Group solves (vk_group_*): independent solves of different mesh sizes, level counts and orders
advanced together, every stage of an FGMRES iteration one launch over all members.

* Each member's iteration count, residual history and solution are bit-identical to a vk_solve of the
  same right-hand side on the same hierarchy (host-driven loop), alone or in any mix, including
  members that join while others are half-way through their solve.
* The launches per group step do not grow with the number of members.
* The FP32-pair (symmetric tile) inverses give the same equality.
"""
import numpy as np
import pytest

import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (N_coarse, nlevels, k): P2 with 2 and 3 levels, P3 and P4 composite patches
KEYS = [(4, 2, 2), (8, 3, 2), (2, 3, 3), (2, 2, 4), (4, 3, 3)]


@pytest.fixture(scope="module")
def vk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_14222_gb300 import build
    build.build()
    import paper_2409_14222_gb300 as vk
    return vk


def _hier(vk, key, prec=0):
    return vk.Hierarchy(*key, options=vk.default_options(use_graph=0, factor_prec=prec))


def _reference(vk, G, b, rtol):
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    out = G.solve(torch.from_numpy(b).cuda(), x, rtol=rtol, maxit=100)
    torch.cuda.synchronize()
    return out, x.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 2])
def test_group_members_equal_single_solves_bit_for_bit(vk, prec):
    Gs = [_hier(vk, k, prec) for k in KEYS]
    bs = [si.rhs_normal(G.ndof(), 60 + i) for i, G in enumerate(Gs)]
    refs = [_reference(vk, G, b, 1e-10) for G, b in zip(Gs, bs)]
    grp = vk.Group(max_members=8)
    xs = [torch.zeros(G.ndof(), dtype=torch.float64, device="cuda") for G in Gs]
    bd = [torch.from_numpy(b).cuda() for b in bs]
    # three members from the start; the other two join after three iterations
    ms = [grp.add(Gs[i], bd[i], xs[i], rtol=1e-10) for i in range(3)]
    for _ in range(3):
        grp.step()
    ms += [grp.add(Gs[i], bd[i], xs[i], rtol=1e-10) for i in range(3, len(Gs))]
    grp.run()
    torch.cuda.synchronize()
    iters = []
    for i, m in enumerate(ms):
        out = grp.result(m)
        ref, xr = refs[i]
        assert out["iterations"] == ref["iterations"] and out["converged"] == ref["converged"], KEYS[i]
        assert np.array_equal(out["history"], ref["history"]), KEYS[i]
        assert np.array_equal(xs[i].cpu().numpy(), xr), KEYS[i]
        assert out["true_res"] == ref["true_res"]
        iters.append(out["iterations"])
    assert len(set(iters)) > 1      # members finished at different iterations
    grp.close()


def test_group_launches_per_step_do_not_grow_with_members(vk):
    keys = [(8, 3, 2), (4, 3, 3), (2, 3, 4), (4, 3, 2)]   # all three levels
    Gs = [_hier(vk, k) for k in keys]
    per_step = []
    for count in (1, len(keys)):
        grp = vk.Group(max_members=8)
        xs = [torch.zeros(G.ndof(), dtype=torch.float64, device="cuda") for G in Gs[:count]]
        bd = [torch.from_numpy(si.rhs_normal(G.ndof(), 7)).cuda() for G in Gs[:count]]
        ms = [grp.add(G, b, x, rtol=1e-14, maxit=6) for G, b, x in zip(Gs[:count], bd, xs)]
        l0 = grp.launches()
        grp.step()
        per_step.append(grp.launches() - l0)
        grp.run()
        for m in ms:
            grp.result(m)
        grp.close()
    assert per_step[0] == per_step[1], per_step


def test_group_refuses_misuse(vk):
    G = _hier(vk, (4, 2, 2))
    n = G.ndof()
    b = torch.from_numpy(si.rhs_normal(n, 1)).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    grp = vk.Group(max_members=1)
    m = grp.add(G, b, x, rtol=1e-10)
    with pytest.raises(vk.VkError):
        grp.add(_hier(vk, (4, 2, 2)), b, torch.zeros_like(x))   # group full
    with pytest.raises(vk.VkError):
        grp.result(m)                                            # still active
    grp.run()
    out = grp.result(m)
    assert out["converged"]
    grp2 = vk.Group(max_members=2)
    m2 = grp2.add(G, b, x, rtol=1e-10)
    with pytest.raises(vk.VkError):
        grp2.add(G, b, torch.zeros_like(x))                      # hierarchy already in a member
    grp2.run()
    grp2.result(m2)
    # a zero right-hand side finishes at once
    m3 = grp2.add(G, torch.zeros_like(b), x)
    assert grp2.step() == 0
    out = grp2.result(m3)
    assert out["iterations"] == 0 and out["converged"] and float(x.abs().max()) == 0.0
