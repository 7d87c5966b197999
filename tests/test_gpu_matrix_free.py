"""Matrix-free (PCPATCH-style) patch matrices against matrix-full ones (Sec. 3.1, last paragraph).

VK_ASSEMBLY_MATRIX_FREE assembles each patch matrix from the element matrices of every cell containing
one of its DoFs, without the global matrix; VK_ASSEMBLY_MATRIX_FULL extracts it from the assembled CSR
matrix.  Both sum every entry over the same cells in the same order, so the patch matrices, their
inverses, each Vanka application and whole solves must be bit-identical (the paper reports essentially
identical iteration counts for the two implementations); the setup cost of each is reported.
"""
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


@pytest.mark.parametrize("case", [(4, 2, 2), (2, 3, 3), (2, 2, 4), (8, 3, 2)])
@pytest.mark.parametrize("prec", [0, 2])
def test_matrix_free_patches_equal_matrix_full_bit_for_bit(vk, case, prec):
    Nc, L, k = case
    full = vk.Hierarchy(Nc, L, k, options=vk.default_options(factor_prec=prec))
    free = vk.Hierarchy(Nc, L, k, options=vk.default_options(factor_prec=prec,
                                                             patch_assembly=vk.vk.VK_ASSEMBLY_MATRIX_FREE))
    rng = np.random.default_rng(71)
    for l in range(1, L):
        assert free.lam(l) == full.lam(l)
        n = full.ndof(l)
        r = torch.from_numpy(rng.standard_normal(n)).cuda()
        za, zb = torch.empty_like(r), torch.empty_like(r)
        full.vanka(l, r, za)
        free.vanka(l, r, zb)
        torch.cuda.synchronize()
        assert torch.equal(za, zb), (case, l)
    n = full.ndof()
    b = torch.from_numpy(si.rhs_normal(n, 3)).cuda()
    xa, xb = torch.zeros_like(b), torch.zeros_like(b)
    oa = full.solve(b, xa, rtol=1e-10)
    ob = free.solve(b, xb, rtol=1e-10)
    assert oa["iterations"] == ob["iterations"] and np.array_equal(oa["history"], ob["history"])
    assert torch.equal(xa, xb)
    sa, sb = full.stats(), free.stats()
    print(f"{case} prec {prec}: patch matrices + inverses at setup: matrix-full {sa['setup_factor_ms']:.3f} ms, "
          f"matrix-free {sb['setup_factor_ms']:.3f} ms")
    assert sa["setup_factor_ms"] > 0 and sb["setup_factor_ms"] > 0
