"""CPU tests of the C-ABI library: it builds, loads, exports every declared symbol, and its host-side
setup (assembly, transfers, patches, Dirichlet flags, eigenvalue helper) equals the oracle's."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import exact, fem, patches as opatches

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vk():
    from paper_2409_14222_gb300 import build
    build.build()
    import paper_2409_14222_gb300 as vk
    return vk


def test_every_declared_symbol_is_exported(vk):
    with open(os.path.join(ROOT, "include", "vk.h")) as f:
        hdr = f.read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(vk_\w+)\s*\(", hdr, re.M))
    assert declared == set(vk.SYMBOLS)
    L = vk.lib()
    for name in declared:
        assert hasattr(L, name), name


def _csr(vkmod, h, level, which):
    (nr, nc), ptr, col, val = h.export_csr(level, which)
    return sp.csr_matrix((val, col, ptr), shape=(nr, nc))


@pytest.mark.parametrize("Nc,L,k", [(4, 2, 2), (2, 3, 2), (2, 2, 3), (2, 2, 4), (1, 3, 3)])
def test_host_setup_equals_oracle(vk, Nc, L, k):
    h = vk.Hierarchy(Nc, L, k, nu=1.3, host_only=True)
    for l in range(L):
        s = fem.Space(Nc * 2 ** l, k)
        K = fem.assemble_full(s, 1.3)
        mask = s.dirichlet_mask()
        Ao = fem.apply_dirichlet(K, mask)
        A = _csr(vk, h, l, vk.VK_CSR_A)
        assert A.shape == Ao.shape
        assert abs(A - Ao).max() <= 1e-14 * abs(Ao).max()
        # columns sorted, Dirichlet rows are exactly identity rows
        (nr, nc), ptr, col, val = h.export_csr(l, vk.VK_CSR_A)
        assert all(np.all(np.diff(col[ptr[i]:ptr[i + 1]]) > 0) for i in range(nr))
        assert np.array_equal(h.export_dirichlet(l), mask)
        if l > 0:
            P = _csr(vk, h, l, vk.VK_CSR_P)
            Po = fem.prolongation(fem.Space(Nc * 2 ** (l - 1), k), s)
            assert abs(P - Po).max() == 0.0          # both exact rationals, correctly rounded
            R = _csr(vk, h, l, vk.VK_CSR_R)
            assert abs(R - Po.T).max() == 0.0
            ptr, dofs, kind = h.export_patches(l)
            op = opatches.build_patches(s)
            assert len(ptr) - 1 == len(op)
            for i, (knd, ent, d) in enumerate(op):
                assert np.array_equal(dofs[ptr[i]:ptr[i + 1]], d), (l, i)
                assert kind[i] == {"vertex": 0, "edge": 1, "cell": 2}[knd]


def test_hessenberg_eigenvalues_match_lapack(vk):
    rng = np.random.default_rng(0)
    for m in (1, 2, 3, 5, 10, 12):
        for trial in range(5):
            H = np.triu(rng.standard_normal((m, m)), -1)
            got = list(vk.hessenberg_eigenvalues(H))
            want = np.linalg.eigvals(H)
            tol = 1e-10 * max(1.0, np.abs(want).max())
            for w in want:                      # match each LAPACK eigenvalue to a distinct one of ours
                i = int(np.argmin([abs(g - w) for g in got]))
                assert abs(got.pop(i) - w) <= tol, (m, w)
    # symmetric tridiagonal: real spectrum
    T = np.diag(np.arange(1.0, 9.0)) + np.diag(np.ones(7), 1) + np.diag(np.ones(7), -1)
    got = np.sort(vk.hessenberg_eigenvalues(T).real)
    assert np.allclose(got, np.linalg.eigvalsh(T), atol=1e-12)


def test_footprint_and_sizes(vk):
    b = vk.footprint(16, 4, 2)
    assert b > 0
    h = vk.Hierarchy(16, 4, 2, host_only=True)
    info = h.level_info(3)
    assert info["ndof"] == 148739 and info["n_u"] == 132098
    assert info["npatch"] == 129 ** 2
    with pytest.raises(vk.VkError):
        vk.Hierarchy(4, 2, 5, host_only=True)
    with pytest.raises(vk.VkError):
        h.export_patches(0)


def test_host_only_hierarchy_refuses_device_calls(vk):
    import ctypes
    h = vk.Hierarchy(2, 2, 2, host_only=True)
    with pytest.raises(vk.VkError) as e:
        h.lam(1)
    assert e.value.code == vk.vk.VK_ERR_ARG


@pytest.mark.parametrize("key", [(8, 3, 2), (8, 3, 4), (4, 3, 3)])
def test_footprint_builds_every_device_layout_on_the_host(vk, key):
    # vk_footprint builds the SELL forms of A, P and R (with their column-range check) and the patch
    # plans without a device; P has more rows than columns, so its padding must point at column 0
    assert vk.footprint(*key) > 0


@pytest.mark.parametrize("Nc,L,k", [(4, 2, 2), (2, 2, 3), (2, 2, 4)])
def test_dof_counts_and_coordinates_equal_the_oracle_layout(vk, Nc, L, k):
    h = vk.Hierarchy(Nc, L, k, host_only=True)
    for l in range(L):
        s = fem.Space(Nc * 2 ** l, k)
        assert h.dof_counts(l) == (s.n_u, s.n_p)
        xy, kind = h.export_dof_coords(l)
        vx, vy = s.vnode_xy()
        px, py = s.pnode_xy()
        assert np.array_equal(xy[0:s.n_u:2, 0], vx) and np.array_equal(xy[1:s.n_u:2, 0], vx)
        assert np.array_equal(xy[0:s.n_u:2, 1], vy) and np.array_equal(xy[1:s.n_u:2, 1], vy)
        assert np.array_equal(xy[s.n_u:, 0], px) and np.array_equal(xy[s.n_u:, 1], py)
        assert np.array_equal(kind[:s.n_u], np.tile([0, 1], s.n_u // 2)) and np.all(kind[s.n_u:] == 2)
        # Dirichlet flags are exactly the velocity DoFs on the boundary of the unit square
        on_bnd = (xy[:, 0] == 0) | (xy[:, 1] == 0) | (xy[:, 0] == 1) | (xy[:, 1] == 1)
        assert np.array_equal(h.export_dirichlet(l), on_bnd & (kind < 2))


def test_default_options_are_the_documented_ones(vk):
    o = vk.default_options()
    assert (o.sweeps, o.weights, o.cheb_lo, o.cheb_hi, o.eig_steps) == (1, vk.VK_WEIGHTS_PLAIN, 0.25, 1.1, 10)
    assert o.factor_prec == vk.VK_PREC_F64 and o.use_graph == 1 and o.max_iterations == 100
    assert o.batch_prec == vk.VK_BATCH_NONE and o.batch_max_iterations == 60
    assert o.autotune == 1 and o.apply_schedule == -1 and o.batch_engine == vk.VK_ENGINE_TCGEN05
    assert o.test_expire_wait == 0 and o.spmv_warps == 48 and o.batch_coarse_fp32 == 0


def test_footprint_follows_the_options(vk):
    key = (8, 3, 2)
    f64 = vk.footprint(*key)
    f32 = vk.footprint(*key, options=vk.default_options(factor_prec=vk.VK_PREC_F32))
    f64e = vk.footprint(*key, options=vk.default_options(factor_prec=vk.VK_PREC_F64E))
    # P2 patches (<= 39 DoFs): FP32 and FP32-pair inverses keep only the upper 8x8 tiles of the
    # symmetric inverse; FP64 keeps the full warp-packed inverse
    assert f32 < f64e < f64
    # P4 patches (up to 123 DoFs) exceed the symmetric layout's bound: FP32 pairs are stored in full
    # and keep a split residual as well
    f64_p4 = vk.footprint(4, 2, 4)
    assert f64_p4 < vk.footprint(4, 2, 4, options=vk.default_options(factor_prec=vk.VK_PREC_F64E))
    batch = vk.footprint(*key, options=vk.default_options(batch_prec=vk.VK_BATCH_BF16))
    assert batch > f64
    # FP32 coarse copy (n_c + 1)^2 floats instead of two FP64 16-column coarse blocks
    nc = vk.ndof_of(8, 1, 2)
    coarse32 = vk.footprint(*key, options=vk.default_options(batch_prec=vk.VK_BATCH_BF16, batch_coarse_fp32=1))
    assert abs((coarse32 - batch) - (4 * (nc + 1) ** 2 - 2 * 16 * 8 * nc)) < 4096


@pytest.mark.parametrize("field,value", [("apply_schedule", 12), ("apply_schedule", -2), ("batch_engine", 2),
                                         ("spmv_warps", 0), ("test_expire_wait", 2), ("batch_coarse_fp32", 3),
                                         ("sweeps", 0), ("eig_steps", 65), ("factor_prec", 3)])
def test_invalid_options_are_refused(vk, field, value):
    with pytest.raises(vk.VkError) as e:
        vk.footprint(4, 2, 2, options=vk.default_options(**{field: value}))
    assert e.value.code == vk.vk.VK_ERR_ARG


def test_batch_basis_size_is_bounded(vk):
    with pytest.raises(vk.VkError):
        vk.footprint(4, 2, 2, options=vk.default_options(batch_prec=vk.VK_BATCH_BF16, batch_max_iterations=128))
    assert vk.footprint(4, 2, 2, options=vk.default_options(batch_prec=vk.VK_BATCH_BF16, batch_max_iterations=127)) > 0


def _check(vk, prob, opts=None):
    import ctypes
    o = opts if opts is not None else vk.default_options()
    return vk.lib().vk_check_problem(ctypes.byref(prob), ctypes.byref(o))


def test_problem_boundary_data_and_domain_are_checked(vk):
    # the method's problem: velocity Dirichlet data on the whole boundary of the unit square
    assert _check(vk, vk.vk.make_problem(4, 2, 2)) == vk.vk.VK_OK
    assert _check(vk, vk.vk.make_problem(4, 2, 2, domain=(0.0, 0.0, 0.0, 0.0))) == vk.vk.VK_OK
    bad = [vk.vk.make_problem(4, 2, 2, bc=1), vk.vk.make_problem(4, 2, 2, domain=(0.0, 2.0, 0.0, 2.0)),
           vk.vk.make_problem(4, 2, 2, domain=(-1.0, 0.0, 0.0, 1.0)), vk.vk.make_problem(4, 2, 2, nu=0.0),
           vk.vk.make_problem(4, 2, 2, nu=float("inf")), vk.vk.make_problem(4, 13, 2),
           vk.vk.make_problem(4, 2, 5), vk.vk.make_problem(4096, 2, 2)]
    for p in bad:
        assert _check(vk, p) == vk.vk.VK_ERR_ARG
    with pytest.raises(vk.VkError) as e:
        vk.footprint(4, 2, 2, options=vk.default_options(test_singular_patch=10 ** 6))
    assert e.value.code == vk.vk.VK_ERR_ARG
    assert vk.default_options().test_singular_patch == -1


def test_matrix_free_option_builds_element_data(vk):
    # the matrix-free patch assembly keeps each cell's element DoFs and each patch's cell list on the
    # device: a larger footprint, refused values rejected
    base = vk.footprint(8, 3, 2)
    mf = vk.footprint(8, 3, 2, options=vk.default_options(patch_assembly=vk.vk.VK_ASSEMBLY_MATRIX_FREE))
    assert mf > base
    with pytest.raises(vk.VkError):
        vk.footprint(8, 3, 2, options=vk.default_options(patch_assembly=2))


@pytest.mark.parametrize("N,k", [(4, 2), (8, 2), (4, 3), (2, 4)])
def test_manufactured_rhs_equals_the_oracle(vk, N, k):
    # load of Eq. (model_problem) with the Dirichlet data lifted: the library (Silvester basis, its own
    # Gauss-Legendre nodes) and the oracle (exact rational basis, NumPy's Gauss-Legendre) agree to
    # rounding
    h = vk.Hierarchy(N, 1, k, nu=1.0, host_only=True)
    s = fem.Space(N, k)
    want = fem.manufactured_rhs(s, fem.assemble_full(s, 1.0), 1.0)
    got = h.manufactured_rhs()
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)
    mask = s.dirichlet_mask()
    assert np.array_equal(got[mask] == 0.0, want[mask] == 0.0)


@pytest.mark.parametrize("Nc,L,k", [(2, 2, 2), (2, 3, 2), (2, 2, 3), (1, 3, 3), (2, 2, 4)])
def test_quad_host_setup_equals_oracle(vk, Nc, L, k):
    # Taylor-Hood Q_k / Q_{k-1} (Case 2 of Sec. 3): the library's element matrices (FP64 Gauss-Legendre),
    # assembly, tensor-product transfers and quadrilateral patches against the oracle's exact ones
    from oracle import quad
    h = vk.Hierarchy(Nc, L, k, nu=0.7, host_only=True, cell=vk.vk.VK_CELL_QUAD)
    for l in range(L):
        s = quad.QSpace(Nc * 2 ** l, k)
        Ao = fem.apply_dirichlet(quad.assemble_full(s, 0.7), s.dirichlet_mask())
        A = _csr(vk, h, l, vk.VK_CSR_A)
        assert A.shape == Ao.shape
        assert abs(A - Ao).max() <= 1e-14 * abs(Ao).max()
        assert np.array_equal(h.export_dirichlet(l), s.dirichlet_mask())
        if l > 0:
            Po = quad.prolongation(quad.QSpace(Nc * 2 ** (l - 1), k), s)
            assert abs(_csr(vk, h, l, vk.VK_CSR_P) - Po).max() == 0.0
            assert abs(_csr(vk, h, l, vk.VK_CSR_R) - Po.T).max() == 0.0
            ptr, dofs, kind = h.export_patches(l)
            op = quad.build_patches(s)
            assert len(ptr) - 1 == len(op)
            for i, (knd, ent, d) in enumerate(op):
                assert np.array_equal(dofs[ptr[i]:ptr[i + 1]], d), (l, i)
                assert kind[i] == {"vertex": 0, "edge": 1, "cell": 2}[knd]


def test_quad_order_bound(vk):
    with pytest.raises(vk.VkError):
        vk.Hierarchy(2, 2, 5, host_only=True, cell=vk.vk.VK_CELL_QUAD)
    with pytest.raises(vk.VkError):
        vk.Hierarchy(2, 2, 2, host_only=True, cell=3)


@pytest.mark.parametrize("N,k", [(4, 2), (2, 3)])
def test_quad_manufactured_rhs_equals_the_oracle(vk, N, k):
    from oracle import quad
    h = vk.Hierarchy(N, 1, k, host_only=True, cell=vk.vk.VK_CELL_QUAD)
    s = quad.QSpace(N, k)
    want = quad.manufactured_rhs(s, quad.assemble_full(s))
    assert np.linalg.norm(h.manufactured_rhs() - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("Nc,L,k", [(1, 3, 1), (2, 2, 1), (1, 3, 2), (2, 2, 2), (1, 2, 3), (2, 2, 4)])
def test_bdm_host_setup_equals_oracle(vk, Nc, L, k):
    # (BDM_k, dP_{k-1}) (Case 3 of Sec. 3): the library's FP64 reference basis (Vandermonde solve), cell
    # and interior-edge integrals, transfers and extended cell patches against the oracle's exact basis
    # and transfers; the assembled values agree to rounding (the reference basis is solved in
    # double-double: its Vandermonde matrix has condition 1e7 at k = 4)
    from oracle import bdm
    h = vk.Hierarchy(Nc, L, k, nu=0.7, host_only=True, cell=vk.vk.VK_CELL_BDM)
    for l in range(L):
        s = bdm.BDMSpace(Nc * 2 ** l, k)
        Ao = fem.apply_dirichlet(bdm.assemble_full(s, 0.7), s.dirichlet_mask())
        A = _csr(vk, h, l, vk.VK_CSR_A)
        assert A.shape == Ao.shape
        assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max(), (l, abs(A - Ao).max() / abs(Ao).max())
        assert abs(A - A.T).max() <= 1e-13 * abs(Ao).max()
        assert np.array_equal(h.export_dirichlet(l), s.dirichlet_mask())
        if l > 0:
            Po = bdm.prolongation(bdm.BDMSpace(Nc * 2 ** (l - 1), k), s)
            P = _csr(vk, h, l, vk.VK_CSR_P)
            # formed in double-double and rounded once: the oracle's exact rationals to the last bit
            # (the pressure rows in FP64 to a few units of the last place)
            assert P.nnz == Po.nnz and abs(P - Po).max() <= 1e-15 * abs(Po).max()
            assert abs(_csr(vk, h, l, vk.VK_CSR_R) - P.T).max() == 0.0
            ptr, dofs, kind = h.export_patches(l)
            op = bdm.build_patches(s)
            assert len(ptr) - 1 == len(op)
            for i, (knd, ent, d) in enumerate(op):
                assert np.array_equal(dofs[ptr[i]:ptr[i + 1]], d), (l, i)
                assert kind[i] == 2


def test_bdm_order_and_assembly_bounds(vk):
    for k in (0, 6):
        with pytest.raises(vk.VkError):
            vk.Hierarchy(2, 2, k, host_only=True, cell=vk.vk.VK_CELL_BDM)
    with pytest.raises(vk.VkError):
        vk.Hierarchy(2, 2, 2, host_only=True, cell=vk.vk.VK_CELL_BDM,
                     options=vk.default_options(patch_assembly=vk.vk.VK_ASSEMBLY_MATRIX_FREE))
    # the largest interior patch for k = 5 (165 DoFs) still fits the patch kernels
    h = vk.Hierarchy(4, 2, 5, host_only=True, cell=vk.vk.VK_CELL_BDM)
    ptr, _, _ = h.export_patches(1)
    from oracle import bdm
    assert np.diff(ptr).max() == bdm.interior_patch_size(5) == 165


@pytest.mark.parametrize("N,k", [(4, 1), (4, 2), (2, 3)])
def test_bdm_manufactured_rhs_equals_the_oracle(vk, N, k):
    from oracle import bdm
    h = vk.Hierarchy(N, 1, k, host_only=True, cell=vk.vk.VK_CELL_BDM)
    s = bdm.BDMSpace(N, k)
    want = bdm.load_vector(s)
    want[s.dirichlet_mask()] = 0.0
    assert np.linalg.norm(h.manufactured_rhs() - want) <= 1e-13 * np.linalg.norm(want)


def test_bdm_dof_coords_follow_the_oracle_layout(vk):
    from oracle import bdm
    N, k = 3, 3
    h = vk.Hierarchy(N, 1, k, host_only=True, cell=vk.vk.VK_CELL_BDM)
    xy, kind = h.export_dof_coords(0)
    s = bdm.BDMSpace(N, k)
    assert np.array_equal(kind[:s.n_edge], np.full(s.n_edge, 3))
    assert np.array_equal(kind[s.n_edge:s.n_u], np.full(s.n_u - s.n_edge, 4))
    assert np.array_equal(kind[s.n_u:], np.full(s.n_p, 2))
    for e, (va, vb) in enumerate(s.edges):
        for j in range(k + 1):
            t = (j + 1) / (k + 2)
            want = (np.array(va) + t * (np.array(vb) - np.array(va))) / N
            assert np.allclose(xy[e * (k + 1) + j], want, atol=1e-15)
    for c, cell in enumerate(s.cells):
        _, _, pd = s.cell_dofs(c)
        x0, J = s.geometry(c, 1.0 / N)
        assert np.allclose(xy[s.n_edge + c * (k + 1) * (k - 1)], x0 + J @ [1 / 3, 1 / 3], atol=1e-15)
        for m, (a, b) in enumerate(exact.lattice_nodes(k - 1)):
            assert np.allclose(xy[pd[m]], x0 + J @ [a / (k - 1), b / (k - 1)], atol=1e-15)


def test_bdm_index_bound_and_options_are_checked(vk):
    # (BDM_k, dP_{k-1}) rows couple up to six cells: problems whose matrix would overflow 32-bit
    # indices are refused before any host assembly, and the programmatic-launch option takes 0 or 1
    ok = vk.vk.make_problem(8, 3, 5, cell=vk.vk.VK_CELL_BDM)
    assert _check(vk, ok) == vk.vk.VK_OK
    too_big = vk.vk.make_problem(256, 3, 5, cell=vk.vk.VK_CELL_BDM)    # 1024 x 1024, k = 5
    assert _check(vk, too_big) == vk.vk.VK_ERR_ARG
    assert _check(vk, vk.vk.make_problem(256, 3, 5)) == vk.vk.VK_ERR_ARG   # Taylor-Hood k = 5: no
    assert vk.default_options().graph_pdl == 0
    assert _check(vk, ok, vk.default_options(graph_pdl=1)) == vk.vk.VK_OK
    assert _check(vk, ok, vk.default_options(graph_pdl=2)) == vk.vk.VK_ERR_ARG
