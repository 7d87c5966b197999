"""Solve service (vk_server_*): continuous batching of mixed Stokes solves on one GPU.

Each result must be the same whether the request is solved alone or in a concurrent mix (every solve
runs the same deterministic kernels on its own resident hierarchy), admission must respect the
memory budget by evicting idle hierarchies, and a request larger than the budget must be refused."""
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


def solo(vk, key, b, rtol):
    G = vk.Hierarchy(*key)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    out = G.solve(torch.from_numpy(b).cuda(), x, rtol=rtol)
    torch.cuda.synchronize()
    return x.cpu().numpy(), out


def test_results_are_the_same_alone_and_in_the_mix(vk):
    srv = vk.Server(slots=4)
    reqs = []
    for rep in range(3):
        for i, key in enumerate(MIX):
            b = si.rhs_normal(vk.ndof_of(*key), 1000 * rep + i)
            reqs.append((key, b, srv.submit(*key, b, rtol=1e-9)))
    results = [(key, b) + srv.wait(t, timeout_ms=120000) for key, b, t in reqs]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["builds"] >= len(MIX)
    for key, b, x, res in results:
        assert res["status"] == 0 and res["converged"]
        xs, out = solo(vk, key, b, 1e-9)
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
