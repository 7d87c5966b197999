"""vk_vanka_noalloc: the Vanka application that allocates nothing at call time (its corrections live in
a fixed device array inside the library), for callers that cannot allocate device memory where they
relax.  It must give what vk_vanka gives, call after call, and refuse levels too large for the array.

Collected last on purpose (file name), so a stop-at-first-failure run has run everything else first;
it also passes alone in a fresh process."""
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


@pytest.mark.parametrize("case", [(4, 2, 2), (2, 3, 3), (16, 4, 2)])
def test_noalloc_vanka_matches_vk_vanka_twice(vk, case):
    Nc, L, k = case
    G = vk.Hierarchy(Nc, L, k)
    for level in range(1, L):
        n = G.ndof(level)
        r = torch.from_numpy(si.rhs_normal(n, 100 + level)).cuda()
        z_ref = torch.empty_like(r)
        G.vanka(level, r, z_ref)
        for call in range(2):                      # two calls in a row share the fixed array
            z = torch.full_like(r, np.nan)
            G.vanka_noalloc(level, r, z)
            torch.cuda.synchronize()
            err = float(torch.linalg.vector_norm(z - z_ref) / torch.linalg.vector_norm(z_ref))
            assert err <= 1e-10, (case, level, call, err)


def test_noalloc_rejects_levels_beyond_the_array(vk):
    G = vk.Hierarchy(16, 3, 4)                     # 64x64 P4/P3: about 1.4 million patch slots
    info = G.level_info(2)
    assert info["nslots"] > 2 ** 20
    n = info["ndof"]
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(vk.VkError) as e:
        G.vanka_noalloc(2, r, z)
    assert e.value.code == vk.vk.VK_ERR_ARG and "at most" in str(e.value)
    G.vanka_noalloc(1, r[:G.ndof(1)].contiguous(), z[:G.ndof(1)].contiguous())   # the 32x32 level fits
