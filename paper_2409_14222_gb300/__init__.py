"""Single-GPU (GB300, sm_103a) matrix-full Vanka multigrid + FGMRES for Stokes: Taylor-Hood on triangles
and quadrilaterals, (BDM_k, dP_{k-1}) with the interior-penalty form on triangles.

Implements the hot path of arXiv 2409.14222 (composite Vanka patches, Chebyshev-accelerated
additive relaxation, V-cycle preconditioned FGMRES) as a C-ABI CUDA library (``libvk.so``, declared in
``include/vk.h``) with this thin binding.  Build the library with ``build.build()``.
"""
from .vk import (Hierarchy, Server, Group, VkError, ndof_of, measure_fma_rate, default_options, footprint, hessenberg_eigenvalues, lib,  # noqa: F401
                 VK_PREC_F32, VK_PREC_F64, VK_PREC_F64E, VK_WEIGHTS_MULTIPLICITY, VK_WEIGHTS_PLAIN, VK_CSR_A, VK_CSR_P, VK_BATCH_NONE, VK_BATCH_BF16, VK_BATCH_FP16,
                 VK_ENGINE_TCGEN05, VK_ENGINE_MMA_SYNC, VK_CELL_TRIANGLE, VK_CELL_QUAD, VK_CELL_BDM,
                 VK_CSR_R, SYMBOLS)
