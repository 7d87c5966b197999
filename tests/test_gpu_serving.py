"""Solve service (vk_server_*): continuous batching of mixed Stokes solves on one GPU.

Each result must be the same whether the request is solved alone or in a mix (every request runs the
same deterministic arithmetic on its own resident hierarchy): in the default group mode the admitted
requests of different sizes and orders share every launch of each FGMRES iteration and equal vk_solve's
host-driven loop bit for bit; in the stream mode each request is a vk_solve of its own.  Admission
must respect the memory budget by evicting idle hierarchies, and a request larger than the budget must
be refused."""
import numpy as np
import pytest

import synthetic_inputs as si

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


MIX = [(4, 2, 2), (2, 3, 2), (2, 2, 3), (2, 2, 4), (8, 2, 2), (4, 2, 3)]


def solo(vk, key, b, rtol, mode=0):
    # the group mode runs vk_solve's host-driven loop; the stream mode vk_solve's default graph path
    G = vk.Hierarchy(*key, options=vk.default_options(use_graph=1 if mode == vk.vk.VK_SERVE_STREAMS else 0))
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    out = G.solve(torch.from_numpy(b).cuda(), x, rtol=rtol)
    torch.cuda.synchronize()
    return x.cpu().numpy(), out


@pytest.mark.parametrize("mode", [0, 1])
def test_results_are_the_same_alone_and_in_the_mix(vk, mode):
    srv = vk.Server(slots=4, mode=mode)
    results = []
    st0 = None
    for rnd in (range(1), range(1, 3)):          # the second round finds every hierarchy resident
        reqs = []
        for rep in rnd:
            for i, key in enumerate(MIX):
                b = si.rhs_normal(vk.ndof_of(*key), 1000 * rep + i)
                reqs.append((key, b, srv.submit(*key, b, rtol=1e-9)))
        results += [(key, b) + srv.wait(t, timeout_ms=120000) for key, b, t in reqs]
        if st0 is None:
            st0 = srv.stats()
    st = srv.stats()
    assert st["completed"] == 3 * len(MIX) and st["failed"] == 0
    assert st["builds"] >= len(MIX)
    if mode == vk.vk.VK_SERVE_GROUP:
        # requests of different sizes and orders shared the launches of their iterations
        steps, members = st["group_steps"] - st0["group_steps"], st["member_steps"] - st0["member_steps"]
        print(f"group mode: {members / steps:.2f} requests per launch on average")
        assert steps > 0 and members > 1.5 * steps, (steps, members)
    for key, b, x, res in results:
        assert res["status"] == 0 and res["converged"]
        xs, out = solo(vk, key, b, 1e-9, mode)
        assert res["iterations"] == out["iterations"]
        assert np.array_equal(x, xs), key            # bit for bit: same kernels, same order
        assert res["latency_ms"] >= res["solve_ms"] > 0
    srv.close()


def test_admission_by_footprint_evicts_idle_hierarchies(vk):
    keys = [(4, 2, 2), (2, 2, 3), (2, 3, 2)]
    fps = [vk.footprint(*k) for k in keys]
    # room for the largest single hierarchy only: every change of key must evict
    srv = vk.Server(slots=1, memory_budget=max(fps) + 1)
    tickets = []
    for rep in range(2):
        for i, key in enumerate(keys):
            b = si.rhs_normal(vk.ndof_of(*key), 50 + 10 * rep + i)
            tickets.append((key, b, srv.submit(*key, b, rtol=1e-8)))
    for key, b, t in tickets:
        x, res = srv.wait(t, timeout_ms=120000)
        assert res["status"] == 0
        xs, _ = solo(vk, key, b, 1e-8)
        assert np.array_equal(x, xs)
    st = srv.stats()
    assert st["evictions"] >= len(tickets) - 1
    assert st["bytes_used"] <= st["memory_budget"]
    assert st["resident"] == 1
    srv.close()


def test_request_larger_than_budget_is_refused(vk):
    srv = vk.Server(slots=2, memory_budget=1 << 20)
    key = (4, 2, 2)
    t = srv.submit(*key, si.rhs_normal(vk.ndof_of(*key), 0))
    x, res = srv.wait(t, timeout_ms=60000)
    assert res["status"] == vk.vk.VK_ERR_NO_MEMORY
    srv.close()


def test_wait_timeout_then_result(vk):
    srv = vk.Server(slots=1)
    key = (16, 3, 2)
    t = srv.submit(*key, si.rhs_normal(vk.ndof_of(*key), 3))
    with pytest.raises(vk.VkError) as e:
        srv.wait(t, timeout_ms=0)
    assert e.value.code == vk.vk.VK_ERR_TIMEOUT
    x, res = srv.wait(t, timeout_ms=120000)
    assert res["status"] == 0 and res["setup_ms"] > 0
    srv.close()
