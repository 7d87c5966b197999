"""Failure paths, injected on the host (nothing here faults, traps or hangs the GPU):

* a singular patch matrix (one row of the gathered copy of the matrix zeroed before upload) makes
  vk_setup return VK_ERR_SINGULAR naming that patch, and every device buffer is released;
* an allocator whose n-th call fails makes vk_setup return VK_ERR_NO_MEMORY with nothing leaked;
* the solve service: a queued request can be cancelled; hierarchies are shared only between requests
  with the same matrix (the viscosity is part of the key); a worker waiting for memory behind a build
  that fails is woken and finishes.
"""
import ctypes

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


class CountingAllocator:
    """vk_allocator over PyTorch tensors that fails its `fail_at`-th call (1-based; 0 = never)."""

    def __init__(self, vkmod, fail_at=0):
        self.calls = 0
        self.fail_at = fail_at
        self.live = {}

        def _alloc(ctx, nbytes, stream):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            self.live[t.data_ptr()] = t
            return t.data_ptr()

        def _release(ctx, ptr, stream):
            self.live.pop(ptr, None)

        self._a = vkmod.vk.ALLOC_FN(_alloc)
        self._r = vkmod.vk.RELEASE_FN(_release)
        self.struct = vkmod.vk.vk_allocator(None, self._a, self._r)


def _setup(vk, alloc, opts, key=(4, 2, 2)):
    prob = vk.vk.make_problem(*key)
    h = ctypes.c_void_p()
    rc = vk.lib().vk_setup(ctypes.byref(prob), ctypes.byref(opts), ctypes.byref(alloc.struct),
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("patch", [0, 7, 24])
def test_singular_patch_is_reported_with_its_id(vk, patch):
    a = CountingAllocator(vk)
    rc, h = _setup(vk, a, vk.default_options(test_singular_patch=patch))
    assert rc == vk.vk.VK_ERR_SINGULAR
    assert not h.value
    msg = vk.lib().vk_last_error().decode()
    assert f"patch {patch} " in msg and "level 1" in msg, msg
    assert a.calls > 0 and not a.live          # every buffer released on the error path
    # the same problem without the injected zero row sets up normally
    a2 = CountingAllocator(vk)
    rc, h = _setup(vk, a2, vk.default_options())
    assert rc == vk.vk.VK_OK
    vk.lib().vk_destroy(h)
    assert not a2.live


def test_allocator_failing_on_the_nth_call_leaks_nothing(vk):
    ok = CountingAllocator(vk)
    rc, h = _setup(vk, ok, vk.default_options(), key=(2, 3, 2))
    assert rc == vk.vk.VK_OK
    total = ok.calls
    vk.lib().vk_destroy(h)
    assert total > 10 and not ok.live
    for n in sorted({1, 2, total // 3, total // 2, total - 1, total}):
        a = CountingAllocator(vk, fail_at=n)
        rc, h = _setup(vk, a, vk.default_options(), key=(2, 3, 2))
        assert rc == vk.vk.VK_ERR_NO_MEMORY, (n, rc)
        assert not h.value and a.calls == n
        assert not a.live, (n, len(a.live))
    torch.cuda.synchronize()


def test_server_cancels_a_queued_request(vk):
    srv = vk.Server(slots=1)
    try:
        key = (8, 4, 2)   # 64 x 64: its setup keeps the single slot busy while the second waits
        n = vk.ndof_of(*key)
        t1 = srv.submit(*key, si.rhs_normal(n, 0))
        t2 = srv.submit(*key, si.rhs_normal(n, 1))
        srv.cancel(t2)
        x2, r2 = srv.wait(t2, timeout_ms=300000)
        assert r2["status"] == vk.vk.VK_ERR_CANCELLED and r2["iterations"] == 0
        x1, r1 = srv.wait(t1, timeout_ms=300000)
        assert r1["status"] == 0 and r1["converged"]
        with pytest.raises(vk.VkError):
            srv.cancel(t1)                         # finished: not cancellable
        st = srv.stats()
        assert st["completed"] == 2 and st["failed"] == 1
    finally:
        srv.close()


def test_server_keys_hierarchies_by_viscosity(vk):
    # two requests that differ only in nu: each must be solved with its own matrix
    key = (4, 2, 2)
    n = vk.ndof_of(*key)
    b = si.rhs_normal(n, 3)
    srv = vk.Server(slots=2)
    try:
        ta = srv.submit(*key, b, rtol=1e-10, nu=1.0)
        tb = srv.submit(*key, b, rtol=1e-10, nu=0.25)
        xa, ra = srv.wait(ta, timeout_ms=300000)
        xb, rb = srv.wait(tb, timeout_ms=300000)
        assert srv.stats()["builds"] == 2
    finally:
        srv.close()
    for nu, x in ((1.0, xa), (0.25, xb)):
        G = vk.Hierarchy(*key, nu=nu, options=vk.default_options(use_graph=0))   # the group mode's loop
        xd = torch.zeros(n, dtype=torch.float64, device="cuda")
        G.solve(torch.from_numpy(b).cuda(), xd, rtol=1e-10)
        torch.cuda.synchronize()
        assert np.array_equal(x, xd.cpu().numpy()), nu
    assert np.linalg.norm(xa - xb) > 0.1 * np.linalg.norm(xa)


def test_server_worker_waiting_behind_a_failed_build_finishes(vk):
    # every build fails (injected singular patch); the budget holds one reservation at a time, so the
    # second worker waits for memory until the first build's reservation is released
    opts = vk.default_options(test_singular_patch=0)
    fa, fb = vk.footprint(8, 3, 2), vk.footprint(8, 3, 3)
    srv = vk.Server(slots=2, options=opts, memory_budget=int(1.01 * max(fa, fb)))
    try:
        ta = srv.submit(8, 3, 2, si.rhs_normal(vk.ndof_of(8, 3, 2), 0))
        tb = srv.submit(8, 3, 3, si.rhs_normal(vk.ndof_of(8, 3, 3), 0))
        _, ra = srv.wait(ta, timeout_ms=120000)
        _, rb = srv.wait(tb, timeout_ms=120000)
        assert ra["status"] == vk.vk.VK_ERR_SINGULAR and rb["status"] == vk.vk.VK_ERR_SINGULAR
        assert srv.stats()["bytes_used"] == 0
    finally:
        srv.close()


def test_server_refuses_problems_vk_setup_would_refuse(vk):
    srv = vk.Server(slots=1)
    try:
        b = np.zeros(10)
        for p in (vk.vk.make_problem(8, 13, 2), vk.vk.make_problem(8, 3, 2, nu=-1.0),
                  vk.vk.make_problem(8, 3, 2, bc=3), vk.vk.make_problem(1 << 20, 2, 2)):
            r = vk.vk.vk_request(p, b.ctypes.data, 1e-8, 10)
            t = ctypes.c_uint64()
            assert vk.lib().vk_server_submit(srv.handle, ctypes.byref(r), ctypes.byref(t)) == vk.vk.VK_ERR_ARG
    finally:
        srv.close()
